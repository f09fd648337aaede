// sphere.cu -- projected (angular) multipoles on the unit sphere.
//
// Paper, "Statement of need": 3PCF multipoles of scalar fields on the sphere
// (weak-lensing convergence, HEALPix pixels) by a harmonic decomposition of
// one angle of the triangle; "Implementation": each pivot's neighbours fill
// the multipole bins, with sin and cos from a Chebyshev recurrence rather
// than trigonometric calls; "Performance": about two operations per
// multipole for that recurrence.
//
// The neighbour lists come from the same grid and enumeration as the 3-D
// path (chord distance, exact integer bin decisions against chord edges
// 2 sin(theta_b / 2)).  Per neighbour j of pivot p: u, v = the separation
// projected on p's east and north unit vectors, cos(phi) = v / |(u, v)|,
// sin(phi) = u / |(u, v)| (phi = 0 when both vanish), and
//     a_m(p, b) += w_j (cos m phi, sin m phi),   m = 0..K,
// with cos m phi and sin m phi from X_m = 2 cos(phi) X_{m-1} - X_{m-2}
// (two FMAs per m; the weight rides along, as the recurrence is linear).
// Row layout per (primary, bin): [Re a_1, Im a_1, ..., Re a_K, Im a_K, a_0],
// padded to a multiple of 32: each (Re, Im) pair on an even slot, so one
// paired FP32 instruction (FFMA2 / FADD2) advances or accumulates both.
#include "pair.cuh"

namespace ctb {

template <int K>
struct StepSphere {
  static constexpr int NCP = round32(2 * K + 1);
  static constexpr bool kFullLaneLoop = true;
  static constexpr int kConvE = 1;  // the row holds a_m itself: one identity entry per slot
  float ex, ey;      // east unit vector (its z component is zero)
  float nx, ny, nz;  // north unit vector
  __device__ __forceinline__ void operator()(float2* acc, float w, float dx, float dy, float dz) const {
    const float u = fmaf(ex, dx, ey * dy);
    const float v = fmaf(nx, dx, fmaf(ny, dy, nz * dz));
    const float r2 = fmaf(u, u, v * v);
    const bool flat = !(r2 > 0.f);
    const float ir = rsqrtf(flat ? 1.f : r2);
    const float c = flat ? 1.f : v * ir;
    const float s = flat ? 0.f : u * ir;
    slot_ref<2 * K>(acc) += w;
    if constexpr (K >= 1) {
      const float2 c2 = make_float2(c + c, c + c);
      float2 p = make_float2(w, 0.f);          // w (cos, sin) of (m - 2) phi
      float2 q = make_float2(w * c, w * s);    // and of (m - 1) phi
      acc[0] = __fadd2_rn(acc[0], q);
#pragma unroll
      for (int m = 2; m <= K; ++m) {
        const float2 r = __ffma2_rn(c2, q, make_float2(-p.x, -p.y));
        acc[m - 1] = __fadd2_rn(acc[m - 1], r);
        p = q;
        q = r;
      }
    }
  }
};

// East and north unit vectors of the tangent plane at direction (x, y, z):
// e_E = z x n / |z x n|, e_N = n x e_E (n normalised); at a pole e_E = y.
__device__ __forceinline__ StepSphere<0> frame_at(float x, float y, float z) {
  const float il = rsqrtf(fmaf(x, x, fmaf(y, y, z * z)));
  x *= il;
  y *= il;
  z *= il;
  const float rho2 = fmaf(x, x, y * y);
  StepSphere<0> f;
  if (rho2 > 0.f) {
    const float ir = rsqrtf(rho2);
    const float rho = rho2 * ir;
    f.ex = -y * ir;
    f.ey = x * ir;
    f.nx = -z * x * ir;
    f.ny = -z * y * ir;
    f.nz = rho;
  } else {
    f.ex = 0.f;
    f.ey = 1.f;
    f.nx = -z;
    f.ny = 0.f;
    f.nz = x;
  }
  return f;
}

template <int K>
constexpr size_t am_smem_per_warp() {
  return alm_smem_per_warp(StepSphere<K>::NCP);
}
template <int K>
constexpr size_t am_table_bytes() {
  return (size_t)StepSphere<K>::NCP * sizeof(int2);
}

// One warp per primary, one run per non-empty (primary, bin) list, as in k_alm.
template <int K>
__global__ void __launch_bounds__(128) k_am(AlmArgs a) {
  extern __shared__ float s_am[];
  // [identity conversion table | per warp: flush buffers, list offsets, counts]
  int2* s_tab = reinterpret_cast<int2*>(s_am);
  for (int k = threadIdx.x; k < StepSphere<K>::NCP; k += blockDim.x) s_tab[k] = __ldg(a.conv + k);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  char* wbase = reinterpret_cast<char*>(s_am) + am_table_bytes<K>() + (size_t)warp * am_smem_per_warp<K>();
  float* sbuf = reinterpret_cast<float*>(wbase);
  uint32_t* s_off =
      reinterpret_cast<uint32_t*>(wbase + (size_t)(flush_buf_floats(StepSphere<K>::NCP) + StepSphere<K>::NCP) * sizeof(float));
  uint32_t* s_n = s_off + kNbinsCap;
  const int nbins = a.nbins;
  while (true) {
    unsigned long long i = 0;
    if (lane == 0) i = atomicAdd(a.work, 1ull);
    i = __shfl_sync(0xffffffffu, i, 0);
    if (i >= (unsigned long long)a.prim_count) break;
    const uint64_t ib = i * (uint64_t)nbins;
    for (int b = lane; b < nbins; b += 32) {
      const uint32_t n = __ldg(a.counts + ib + b);
      s_n[b] = n;
      s_off[b] = __ldg(a.offsets + ib + b);
      if (n == 0) {
        float4* o = reinterpret_cast<float4*>(a.M + (ib + b) * (uint64_t)a.row);
        for (int k = 0; k < a.row / 4; ++k) o[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    __syncwarp();
    int b = 0;
    while (b < nbins && s_n[b] == 0) ++b;
    if (b < nbins) {
      const int64_t gi = a.prim_begin + (int64_t)i;
      const uint32_t sp = a.prim ? __ldg(a.prim + gi) : (uint32_t)gi;
      const uint4 P = __ldg(a.pts + sp);
      const StepSphere<0> f0 = frame_at(fmaf((float)P.x, a.sph_unit, a.sph_origin[0]),
                                        fmaf((float)P.y, a.sph_unit, a.sph_origin[1]),
                                        fmaf((float)P.z, a.sph_unit, a.sph_origin[2]));
      const StepSphere<K> step{f0.ex, f0.ey, f0.nx, f0.ny, f0.nz};
      int nb = b + 1;
      while (nb < nbins && s_n[nb] == 0) ++nb;
      Run cur{s_off[b], s_n[b]};
      Run nxt = nb < nbins ? Run{s_off[nb], s_n[nb]} : Run{0, 0};
      const uint32_t pe = s_off[nbins - 1] + s_n[nbins - 1];
      if (lane < (int)kListPrefetchLines && cur.off + (uint32_t)lane * 32u < pe)
        prefetch_l2(a.lists + cur.off + (uint32_t)lane * 32u);
      Prefetch pf = prefetch_start(a.lists, a.pts, cur, nxt, P, lane);
      while (true) {
        run_steps(a, step, cur, nxt, P, pf, a.M + (ib + b) * (uint64_t)a.row, s_tab, sbuf, lane, pe);
        b = nb;
        if (b >= nbins) break;
        cur = nxt;
        nb = b + 1;
        while (nb < nbins && s_n[nb] == 0) ++nb;
        nxt = nb < nbins ? Run{s_off[nb], s_n[nb]} : Run{0, 0};
      }
    }
    __syncwarp();
  }
}

template <int K>
static int am_occupancy_K(int wpb) {
  const size_t smem = am_table_bytes<K>() + (size_t)wpb * am_smem_per_warp<K>();
  if (cudaFuncSetAttribute(k_am<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_am<K>, wpb * 32, smem) != cudaSuccess) return 0;
  return nb;
}

template <int K>
static cudaError_t launch_am_K(const AlmArgs& a, int wpb, int nblocks, cudaStream_t st) {
  const size_t smem = am_table_bytes<K>() + (size_t)wpb * am_smem_per_warp<K>();
  cudaError_t e = cudaFuncSetAttribute(k_am<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_am<K><<<nblocks, wpb * 32, smem, st>>>(a);
  ++g_launches;
  return cudaGetLastError();
}

#define CTB_SPHERE_CASES(X) \
  X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

int am_blocks_per_sm(int mmax, int wpb) {
  switch (mmax) {
#define CASE(K) \
  case K:       \
    return am_occupancy_K<K>(wpb);
    CTB_SPHERE_CASES(CASE)
#undef CASE
    default:
      return 0;
  }
}

cudaError_t launch_am(const AlmArgs& a, int mmax, int wpb, int nblocks, cudaStream_t st) {
  switch (mmax) {
#define CASE(K) \
  case K:       \
    return launch_am_K<K>(a, wpb, nblocks, st);
    CTB_SPHERE_CASES(CASE)
#undef CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace ctb
