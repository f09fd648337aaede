// grid.cu -- catalogue ingest and the uniform cell grid (radix sort by cell key).
//
// The paper indexes the catalogue with an octree / kd-tree and prunes empty
// space ("Implementation": octree cells tightened into an "oc-ball-tree" so a
// scan visits only occupied regions).  On the GPU a uniform grid of cubic
// cells, sorted so that each x-row of cells is one contiguous run of points,
// gives the same "visit only what is there" property with coalesced loads:
// a neighbour search becomes a short list of (start, end) ranges.
#include "ctb_internal.cuh"

namespace ctb {

// ---------------------------------------------------------------------------
// ingest: float64 xyz / w  ->  fixed-point uint4 point, cell key, index

__global__ void k_ingest(const double* __restrict__ xyz, const double* __restrict__ w, int64_t n,
                         double box, double ox, double oy, double oz, double inv_unit, Geom g,
                         uint32_t key_base, uint32_t val_base, uint32_t* __restrict__ key,
                         uint32_t* __restrict__ val, uint4* __restrict__ pts, uint32_t* flags) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int neg = 0;  // a negative weight in this thread's points
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double p[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
    double wi = w ? w[i] : 1.0;
    neg |= wi < 0.0;
    bool bad = !isfinite(p[0]) || !isfinite(p[1]) || !isfinite(p[2]) || !isfinite(wi);
    if (bad) {
      atomicOr(flags, 1u);
      p[0] = p[1] = p[2] = 0.0;
      wi = 0.0;
    }
    uint32_t u[3], c[3];
    const double org[3] = {ox, oy, oz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double s;
      if (g.periodic) {
        double t = p[k] / box;               // correctly rounded: a point on the
        t -= floor(t);                       // L/2^32 grid maps to its exact unit
        if (t >= 1.0) t = 0.0;
        s = t * 4294967296.0;                // 2^32 units per side
        if (!(s < 4294967295.0)) s = 4294967295.0;
      } else {
        s = (p[k] - org[k]) * inv_unit;      // bounding cube -> [0, 2^31)
        if (s < 0.0) s = 0.0;
        if (!(s < 2147483647.0)) s = 2147483647.0;
      }
      u[k] = (uint32_t)s;
      c[k] = (uint32_t)(((uint64_t)u[k] * (k == 0 ? g.ncx : g.nc)) >> g.shift);
    }
    key[i] = key_base + (c[2] * g.nc + c[1]) * g.ncx + c[0];
    val[i] = val_base + (uint32_t)i;
    pts[i] = make_uint4(u[0], u[1], u[2], __float_as_uint((float)wi));
  }
  // flags[3]: the catalogue has a negative weight (one vote per block)
  if (__syncthreads_or(neg) && threadIdx.x == 0) atomicOr(flags + 3, 1u);
}

cudaError_t launch_ingest(const double* xyz, const double* w, int64_t n, double box,
                          const double* origin3, double inv_unit, const Geom& g, IngestOut out,
                          uint32_t* d_flags, cudaStream_t st, uint32_t key_base, uint32_t val_base) {
  if (n == 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 65535 * 4) blocks = 65535 * 4;
  double o[3] = {0, 0, 0};
  if (origin3) { o[0] = origin3[0]; o[1] = origin3[1]; o[2] = origin3[2]; }
  k_ingest<<<blocks, 256, 0, st>>>(xyz, w, n, box, o[0], o[1], o[2], inv_unit, g, key_base, val_base,
                                   out.key, out.val, out.pts, d_flags);
  ++g_launches;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// bounding box of finite points (open space): per-block partial min/max

int bbox_blocks(int64_t n) {
  int64_t b = (n + 4095) / 4096;
  if (b < 1) b = 1;
  if (b > 1024) b = 1024;
  return (int)b;
}

__global__ void k_bbox(const double* __restrict__ xyz, int64_t n, double* __restrict__ part,
                       uint32_t* flags) {
  // per block: min x, y, z, |p|^2 and max x, y, z, |p|^2 of the finite points
  double lo[4] = {INFINITY, INFINITY, INFINITY, INFINITY}, hi[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double v[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
    if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2])) {
      atomicOr(flags, 1u);
      continue;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lo[k] = fmin(lo[k], v[k]);
      hi[k] = fmax(hi[k], v[k]);
    }
    const double r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    lo[3] = fmin(lo[3], r2);
    hi[3] = fmax(hi[3], r2);
  }
  __shared__ double s[8][256];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    s[k][threadIdx.x] = lo[k];
    s[4 + k][threadIdx.x] = hi[k];
  }
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        s[k][threadIdx.x] = fmin(s[k][threadIdx.x], s[k][threadIdx.x + h]);
        s[4 + k][threadIdx.x] = fmax(s[4 + k][threadIdx.x], s[4 + k][threadIdx.x + h]);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < 8) part[blockIdx.x * 8 + threadIdx.x] = s[threadIdx.x][0];
}

cudaError_t launch_bbox(const double* xyz, int64_t n, double* d_part, int nblk, uint32_t* d_flags,
                        cudaStream_t st) {
  k_bbox<<<nblk, 256, 0, st>>>(xyz, n, d_part, d_flags);
  ++g_launches;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// device-wide exclusive scan of uint32 (reduce -> scan block sums -> downsweep)

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

size_t scan_tmp_words(size_t len) {
  size_t words = 0;
  while (len > (size_t)kScanTile) {
    len = (len + kScanTile - 1) / kScanTile;
    words += len;
  }
  return words + 1;
}

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t s_warp[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    uint32_t t = lane < nw ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    s_warp[lane] = t;
  }
  __syncthreads();
  uint32_t before = warp > 0 ? s_warp[warp - 1] : 0;
  *total = s_warp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, size_t len, uint32_t* __restrict__ sums) {
  size_t base = (size_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    size_t i = base + (size_t)k * kScanThreads + threadIdx.x;
    if (i < len) s += in[i];
  }
  uint32_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// scans one tile per block; adds offs[blockIdx.x] (offs may be NULL)
__global__ void k_scan_tile(const uint32_t* __restrict__ in, size_t len, const uint32_t* __restrict__ offs,
                            uint32_t* __restrict__ out) {
  size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < len) ? in[base + k] : 0;
    s += v[k];
  }
  uint32_t total;
  uint32_t ex = block_exclusive_scan(s, &total);
  if (offs) ex += offs[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < len) out[base + k] = ex;
    ex += v[k];
  }
}

cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, size_t len, uint32_t* tmp,
                               cudaStream_t st) {
  if (len == 0) return cudaSuccess;
  if (len <= (size_t)kScanTile) {
    k_scan_tile<<<1, kScanThreads, 0, st>>>(in, len, nullptr, out);
    ++g_launches;
    return cudaGetLastError();
  }
  size_t nb = (len + kScanTile - 1) / kScanTile;
  uint32_t* sums = tmp;
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, len, sums);
  ++g_launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // scan the block sums in place (recursively), workspace after them
  e = exclusive_scan_u32(sums, sums, nb, tmp + nb, st);
  if (e != cudaSuccess) return e;
  k_scan_tile<<<(unsigned)nb, kScanThreads, 0, st>>>(in, len, sums, out);
  ++g_launches;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// LSD radix sort of (key, val) pairs, 8-bit digits, stable

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;  // keys per block

int sort_blocks(int64_t n) { return (int)((n + kSortTile - 1) / kSortTile); }
size_t sort_hist_words(int64_t n) { return (size_t)256 * (size_t)(sort_blocks(n) > 0 ? sort_blocks(n) : 1); }

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ key, int64_t n,
                                                             int shift, uint32_t* __restrict__ hist,
                                                             int nblk) {
  __shared__ uint32_t s_h[256];
  s_h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int r = 0; r < kSortRounds; ++r) {
    int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&s_h[(key[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * nblk + blockIdx.x] = s_h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, int64_t n, int shift,
    const uint32_t* __restrict__ offs, int nblk, uint32_t* __restrict__ kout, uint32_t* __restrict__ vout) {
  __shared__ uint32_t s_wc[kSortThreads / 32][256];
  __shared__ uint32_t s_run[256];
  __shared__ uint32_t s_goff[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  s_goff[threadIdx.x] = offs[(size_t)threadIdx.x * nblk + blockIdx.x];
  s_run[threadIdx.x] = 0;
  const unsigned lt = (1u << lane) - 1u;
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) s_wc[w][threadIdx.x] = 0;
    __syncthreads();
    int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
    bool valid = i < n;
    uint32_t k = valid ? kin[i] : 0u;
    uint32_t v = valid ? vin[i] : 0u;
    uint32_t d = (k >> shift) & 255u;
    unsigned act = __ballot_sync(0xffffffffu, valid);
    unsigned rank = 0;
    if (valid) {
      unsigned peers = __match_any_sync(act, d);
      rank = __popc(peers & lt);
      if (rank == 0) s_wc[warp][d] = __popc(peers);
    }
    __syncthreads();
    {
      uint32_t run = s_run[threadIdx.x];
#pragma unroll
      for (int w = 0; w < kSortThreads / 32; ++w) {
        uint32_t c = s_wc[w][threadIdx.x];
        s_wc[w][threadIdx.x] = run;
        run += c;
      }
      s_run[threadIdx.x] = run;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = s_goff[d] + s_wc[warp][d] + rank;
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
  }
}

cudaError_t radix_sort(SortBufs& b, int64_t n, int bits, bool* result_in_1, cudaStream_t st) {
  *result_in_1 = false;
  if (n <= 1 || bits <= 0) return cudaSuccess;
  int nblk = sort_blocks(n);
  uint32_t *ki = b.k0, *vi = b.v0, *ko = b.k1, *vo = b.v1;
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<<<nblk, kSortThreads, 0, st>>>(ki, n, shift, b.hist, nblk);
    ++g_launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan_u32(b.hist, b.hist, (size_t)256 * nblk, b.scan_tmp, st);
    if (e != cudaSuccess) return e;
    k_radix_scatter<<<nblk, kSortThreads, 0, st>>>(ki, vi, n, shift, b.hist, nblk, ko, vo);
    ++g_launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint32_t* t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
    *result_in_1 = !*result_in_1;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// gather into cell order and the cell start table

__global__ void k_gather(const uint32_t* __restrict__ val, const uint4* __restrict__ pin, int64_t n,
                         uint4* __restrict__ pout, uint32_t* __restrict__ s2i, uint32_t* __restrict__ i2s) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint32_t src = val[i];
    pout[i] = pin[src];
    s2i[i] = src;
    i2s[src] = (uint32_t)i;
  }
}

cudaError_t launch_gather(const uint32_t* val_sorted, const uint4* pts_in, int64_t n, uint4* pts_sorted,
                          uint32_t* sorted_to_input, uint32_t* input_to_sorted, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 65535 * 4) blocks = 65535 * 4;
  k_gather<<<blocks, 256, 0, st>>>(val_sorted, pts_in, n, pts_sorted, sorted_to_input, input_to_sorted);
  ++g_launches;
  return cudaGetLastError();
}

// cell_start[c] = first sorted position with key >= c, for c in [0, ncells]:
// the exclusive prefix sum of the points per cell.  The counts are added by
// one atomic per run of equal keys within a warp (the keys are sorted), so
// empty cells cost only the scan, however long the empty stretches.
__global__ void k_cell_count(const uint32_t* __restrict__ key, int64_t n, uint32_t* __restrict__ cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + (threadIdx.x & ~31) + lane;
    const bool ok = i < n;
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const uint32_t k = key[i];
      const unsigned grp = __match_any_sync(act, k);
      if (lane == __ffs(grp) - 1) atomicAdd(cnt + k, (uint32_t)__popc(grp));
    }
  }
}

cudaError_t launch_cell_start(const uint32_t* key_sorted, int64_t n, uint32_t ncells, uint32_t* cell_start,
                              uint32_t* scan_tmp, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(cell_start, 0, ((size_t)ncells + 1) * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  if (n > 0) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 65535 * 4) blocks = 65535 * 4;
    k_cell_count<<<blocks, 256, 0, st>>>(key_sorted, n, cell_start);
    ++g_launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return exclusive_scan_u32(cell_start, cell_start, (size_t)ncells + 1, scan_tmp, st);
}

}  // namespace ctb
