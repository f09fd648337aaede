// shared.cu -- shared neighbour lists for close pivots.
//
// Paper, "Implementation": pivots close to one another share one neighbour
// list; closeness is a pivot radius set from the mean separation unless the
// user gives one.  Reading implemented here: the points, as stored, are
// grouped by the cubic pivot cell of side h that holds them (cells aligned
// at the origin of coordinates).  A group is represented by its member of
// smallest catalogue index and carries the sum of its members' weights.  The
// pair pipeline then runs over the representatives only, with the group
// weights as primary weights, so every member takes its representative's
// neighbour list and multipoles.
//
// Grouping on the device: a 64-bit pivot-cell key per point (catalogue
// order), a stable LSD radix sort of the catalogue indices by its low 32
// bits and then, when there are more than 2^32 cells, by its high bits;
// segment heads, an exclusive scan of the heads (the group ids), and one
// pass over the segments for the representative and the FP64 weight sum.
#include "ctb_internal.cuh"

namespace ctb {

__global__ void k_pivot_key(const uint4* __restrict__ pts, const uint32_t* __restrict__ i2s, int64_t n,
                            PivotGrid pg, uint32_t* __restrict__ key_lo, uint32_t* __restrict__ key_hi,
                            uint32_t* __restrict__ sort_key, uint32_t* __restrict__ val) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 q = __ldg(pts + __ldg(i2s + i));
    const uint32_t u[3] = {q.x, q.y, q.z};
    uint64_t c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      // the stored coordinate: origin + u * unit (exact for points on the
      // fixed-point grid), then its cell along this axis
      const double x = fma((double)u[k], pg.unit, pg.origin[k]);
      long long ck = (long long)floor(x / pg.h) - pg.k0[k];
      if (ck < 0) ck = 0;
      if (ck >= (long long)pg.n[k]) ck = (long long)pg.n[k] - 1;
      c[k] = (uint64_t)ck;
    }
    const uint64_t key = (c[2] * pg.n[1] + c[1]) * pg.n[0] + c[0];
    key_lo[i] = (uint32_t)key;
    key_hi[i] = (uint32_t)(key >> 32);
    sort_key[i] = (uint32_t)key;
    val[i] = (uint32_t)i;
  }
}

// the high key bits in the order of the first sort pass
__global__ void k_gather_hi(const uint32_t* __restrict__ val, const uint32_t* __restrict__ key_hi, int64_t n,
                            uint32_t* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride)
    out[t] = __ldg(key_hi + __ldg(val + t));
}

__global__ void k_group_heads(const uint32_t* __restrict__ val, const uint32_t* __restrict__ key_lo,
                              const uint32_t* __restrict__ key_hi, int64_t n, uint32_t* __restrict__ head) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    uint32_t h = 1u;
    if (t > 0) {
      const uint32_t a = __ldg(val + t), b = __ldg(val + t - 1);
      h = (__ldg(key_lo + a) != __ldg(key_lo + b) || __ldg(key_hi + a) != __ldg(key_hi + b)) ? 1u : 0u;
    }
    head[t] = h;
  }
}

// One thread per segment head: the representative (smallest catalogue index
// of the segment) as a sorted position, and the weight sum in FP64, members
// in sorted order.
__global__ void k_group_reduce(const uint32_t* __restrict__ val, const uint32_t* __restrict__ head,
                               const uint32_t* __restrict__ gid, int64_t n, const uint4* __restrict__ pts,
                               const uint32_t* __restrict__ i2s, uint32_t* __restrict__ prim_out,
                               float* __restrict__ w_out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    if (!__ldg(head + t)) continue;
    uint32_t rep = __ldg(val + t);
    double W = 0.0;
    int64_t u = t;
    do {
      const uint32_t v = __ldg(val + u);
      rep = min(rep, v);
      W += (double)__uint_as_float(__ldg(pts + __ldg(i2s + v)).w);
      ++u;
    } while (u < n && !__ldg(head + u));
    const uint32_t g = __ldg(gid + t);
    prim_out[g] = __ldg(i2s + rep);
    w_out[g] = (float)W;
  }
}

static int grid_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 65535 * 4) b = 65535 * 4;
  return (int)b;
}

cudaError_t launch_pivot_key(const uint4* pts, const uint32_t* i2s, int64_t n, const PivotGrid& pg,
                             uint32_t* key_lo, uint32_t* key_hi, uint32_t* sort_key, uint32_t* val,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_pivot_key<<<grid_blocks(n), 256, 0, st>>>(pts, i2s, n, pg, key_lo, key_hi, sort_key, val);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_gather_hi(const uint32_t* val, const uint32_t* key_hi, int64_t n, uint32_t* out,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_gather_hi<<<grid_blocks(n), 256, 0, st>>>(val, key_hi, n, out);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_group_heads(const uint32_t* val_sorted, const uint32_t* key_lo, const uint32_t* key_hi,
                               int64_t n, uint32_t* head, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_group_heads<<<grid_blocks(n), 256, 0, st>>>(val_sorted, key_lo, key_hi, n, head);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_group_reduce(const uint32_t* val_sorted, const uint32_t* head, const uint32_t* gid, int64_t n,
                                const uint4* pts, const uint32_t* i2s, uint32_t* prim_out, float* w_out,
                                cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_group_reduce<<<grid_blocks(n), 256, 0, st>>>(val_sorted, head, gid, n, pts, i2s, prim_out, w_out);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ctb
