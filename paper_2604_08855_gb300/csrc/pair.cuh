// pair.cuh -- harmonic accumulation of the pair multipoles (template;
// instantiated per ell_max in pair_[a-f].cu so they compile in parallel).
//
// Paper, "Implementation": pick a pivot, find all its neighbours inside the
// search range, fill the multipole bins; sin/cos of the angle are replaced by
// a polynomial recurrence because evaluating trigonometric functions is slow.
// "Performance": the time goes into scanning for neighbours and updating the
// histograms, with a per-multipole recurrence cost.
//
// GB300 design.  The neighbour lists of a primary are grouped by bin
// (stream.cu).  One warp owns one primary: for each of its (primary, bin)
// lists each lane takes one neighbour per step, evaluates the (l, m)
// coefficients of the direction by recurrences in float32 registers and
// accumulates them (one FMA per coefficient).  Up to l_max 10 one kernel
// holds all coefficients; above, the m columns are split into passes of at
// most 128 accumulators, each its own kernel and launch (see k_alm).  At the end of the list the 32
// lanes' accumulators are summed through a shared-memory transpose, scaled by
// the per-(l, m) normalisation and stored as the (primary, bin) row of M.
// Each list is one run, so the cross-lane reduction happens once per
// (primary, bin), and the first loads of the next list are issued while the
// current one is still being accumulated.
//
// Recurrence (real Y_lm up to a constant per (l, m), applied at the flush):
//   (c_m + i s_m) = w (x + i y)^m           complex power, 4 FLOPs per m
//   p_m^m = 1,  p_{m+1}^m = z,  p_l^m = z p_{l-1}^m - beta_lm p_{l-2}^m
// p_l^m is the associated Legendre function with the (1 - z^2)^{m/2} factor
// absorbed in (x + i y)^m and rescaled to a monic recurrence (2 FLOPs per step).
#pragma once

#include "ctb_internal.cuh"

namespace ctb {

constexpr uint32_t kNone = 0xffffffffu;
// The list words of one primary are one contiguous range; the read position
// is kept this many 128-byte lines ahead of use in L2.  The list buffer is
// allocated with kListSlackBytes past its last entry for prefetches that run
// beyond it.
constexpr uint32_t kListPrefetchLines = 6;

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}


// Column m >= 1 of the Legendre recurrence, l = LL..L (template recursion keeps
// every accumulator index a compile-time constant, so the array stays in
// registers).
template <int L, int M0, int M1, int M, int LL>
__device__ __forceinline__ void column_rec(const AlmArgs& a, float* acc, float z, float cr, float ci, float p2,
                                           float p1) {
  if constexpr (LL <= L) {
    const float p = fmaf(z, p1, -(a.beta[LL * (kLmaxCap + 1) + M] * p2));
    acc[local_slot(LL, M, M0, M1)] = fmaf(p, cr, acc[local_slot(LL, M, M0, M1)]);
    acc[local_slot(LL, -M, M0, M1)] = fmaf(p, ci, acc[local_slot(LL, -M, M0, M1)]);
    column_rec<L, M0, M1, M, LL + 1>(a, acc, z, cr, ci, p1, p);
  }
}

// Chebyshev column m: moments S_{m,k} += c T_k, k = K..L-m, stored in slot (m + k, +-m).
template <int L, int M0, int M1, int M, int K>
__device__ __forceinline__ void cheb_col(float* acc, const float* T, float cr, float ci) {
  if constexpr (K <= L - M) {
    if constexpr (M == 0) {
      acc[local_slot(K, 0, M0, M1)] = fmaf(cr, T[K], acc[local_slot(K, 0, M0, M1)]);
    } else {
      acc[local_slot(M + K, M, M0, M1)] = fmaf(cr, T[K], acc[local_slot(M + K, M, M0, M1)]);
      acc[local_slot(M + K, -M, M0, M1)] = fmaf(ci, T[K], acc[local_slot(M + K, -M, M0, M1)]);
    }
    cheb_col<L, M0, M1, M, K + 1>(acc, T, cr, ci);
  }
}

// Columns m = M..ME with (cr, ci) = w (x + i y)^M on entry.
template <int L, int M0, int M1, int M, int ME>
__device__ __forceinline__ void columns_rec(const AlmArgs& a, float* acc, const float* T, float x, float y, float z,
                                            float cr, float ci) {
  if constexpr (M <= ME) {
    if constexpr (M <= cheb_max_m(L)) {
      acc[local_slot(M, M, M0, M1)] += cr;  // T_0 = 1
      acc[local_slot(M, -M, M0, M1)] += ci;
      cheb_col<L, M0, M1, M, 1>(acc, T, cr, ci);
    } else {
      acc[local_slot(M, M, M0, M1)] += cr;
      acc[local_slot(M, -M, M0, M1)] += ci;
      if constexpr (M + 1 <= L) {
        acc[local_slot(M + 1, M, M0, M1)] = fmaf(z, cr, acc[local_slot(M + 1, M, M0, M1)]);
        acc[local_slot(M + 1, -M, M0, M1)] = fmaf(z, ci, acc[local_slot(M + 1, -M, M0, M1)]);
      }
      column_rec<L, M0, M1, M, M + 2>(a, acc, z, cr, ci, 1.f, z);
    }
    if constexpr (M + 1 <= ME) {
      const float nr = fmaf(cr, x, -(ci * y));
      const float ni = fmaf(cr, y, ci * x);
      columns_rec<L, M0, M1, M + 1, ME>(a, acc, T, x, y, z, nr, ni);
    }
  }
}

// T_k(z), k = K..KMAX, by T_k = 2z T_{k-1} - T_{k-2}: one FMA per degree.
template <int K, int KMAX>
__device__ __forceinline__ void cheb_seq(float* T, float z2) {
  if constexpr (K <= KMAX) {
    T[K] = fmaf(z2, T[K - 1], -T[K - 2]);
    cheb_seq<K + 1, KMAX>(T, z2);
  }
}

// (x + i y)^E, E >= 1, by repeated squaring: a pass that starts at column
// m0 needs the power m0, in about 4 log2(m0) instructions instead of 4 m0.
template <int E>
__device__ __forceinline__ void cpow(float x, float y, float& r, float& i) {
  if constexpr (E == 1) {
    r = x;
    i = y;
  } else if constexpr (E % 2 == 0) {
    float a, b;
    cpow<E / 2>(x, y, a, b);
    r = fmaf(a, a, -(b * b));
    i = (a + a) * b;
  } else {
    float a, b;
    cpow<E - 1>(x, y, a, b);
    r = fmaf(a, x, -(b * y));
    i = fmaf(a, y, b * x);
  }
}

// Add one neighbour (weight w, unit direction x, y, z) to the pass's
// accumulators: one FMA per coefficient, plus the Chebyshev sequence (shared
// by all Chebyshev columns), the Legendre recurrences of the other columns,
// and the complex power.
template <int L, int M0, int M1>
__device__ __forceinline__ void accum_pass(const AlmArgs& a, float* acc, float w, float x, float y, float z) {
  constexpr int MC = cheb_max_m(L);
  constexpr int KMAX = M0 <= MC ? L - M0 : 1;  // highest Chebyshev degree this pass needs
  float T[KMAX + 1 > 2 ? KMAX + 1 : 2];
  if constexpr (M0 <= MC) {
    T[0] = 1.f;
    T[1] = z;
    cheb_seq<2, KMAX>(T, z + z);
  }
  if constexpr (M0 == 0) {
    if constexpr (MC >= 0) {
      acc[local_slot(0, 0, M0, M1)] += w;
      cheb_col<L, M0, M1, 0, 1>(acc, T, w, 0.f);
    }
  }
  constexpr int MS = M0 < 1 ? 1 : M0;
  constexpr int ME = M1 < L ? M1 : L;
  if constexpr (MS <= ME) {
    float pr, pi;
    cpow<MS>(x, y, pr, pi);  // (x + i y)^MS by squaring
    columns_rec<L, M0, M1, MS, ME>(a, acc, T, x, y, z, w * pr, w * pi);
  }
}

// Cross-lane sum of the NCP accumulators through shared memory: every lane
// writes its row (stride NCP + 4 floats, so 16-byte stores of 8 consecutive
// lanes cover all 32 banks), then lane l sums column block
// [l * NCP/32, (l+1) * NCP/32) over the 32 rows.  Afterwards acc[0 .. NCP/32)
// of lane l holds the warp totals of those slots.
template <int NCP>
__device__ __forceinline__ void smem_transpose_reduce(float* acc, float* buf, int lane) {
  constexpr int S = NCP + 4;
  constexpr int V = NCP / 32;
  float* row = buf + lane * S;
#pragma unroll
  for (int i = 0; i < NCP; i += 4)
    *reinterpret_cast<float4*>(row + i) = make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
  __syncwarp();
  if constexpr (V == 4) {
    float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
#pragma unroll
    for (int r = 0; r < 32; r += 2) {
      const float4 u = *reinterpret_cast<const float4*>(buf + r * S + 4 * lane);
      const float4 v = *reinterpret_cast<const float4*>(buf + (r + 1) * S + 4 * lane);
      s0.x += u.x; s0.y += u.y; s0.z += u.z; s0.w += u.w;
      s1.x += v.x; s1.y += v.y; s1.z += v.z; s1.w += v.w;
    }
    acc[0] = s0.x + s1.x; acc[1] = s0.y + s1.y; acc[2] = s0.z + s1.z; acc[3] = s0.w + s1.w;
  } else if constexpr (V == 2) {
    float2 s0 = make_float2(0.f, 0.f), s1 = s0;
#pragma unroll
    for (int r = 0; r < 32; r += 2) {
      const float2 u = *reinterpret_cast<const float2*>(buf + r * S + 2 * lane);
      const float2 v = *reinterpret_cast<const float2*>(buf + (r + 1) * S + 2 * lane);
      s0.x += u.x; s0.y += u.y;
      s1.x += v.x; s1.y += v.y;
    }
    acc[0] = s0.x + s1.x; acc[1] = s0.y + s1.y;
  } else {
    float s[V];
#pragma unroll
    for (int c = 0; c < V; ++c) s[c] = 0.f;
#pragma unroll
    for (int r = 0; r < 32; ++r)
#pragma unroll
      for (int c = 0; c < V; ++c) s[c] += buf[r * S + V * lane + c];
#pragma unroll
    for (int c = 0; c < V; ++c) acc[c] = s[c];
  }
  __syncwarp();
}

// One neighbour list run: records [off, off + n) of the lists buffer.
struct Run {
  uint32_t off, n;
};

// Loads in flight for the next iteration: two record words and one neighbour.
struct Prefetch {
  uint32_t j0, j1;
  uint4 q0;
};

// Record of iteration t of the concatenated runs [cur | nxt] (T = iterations of cur).
__device__ __forceinline__ uint32_t rec_at(const uint32_t* __restrict__ lists, Run cur, Run nxt, uint32_t T,
                                           uint32_t t, int lane) {
  if (t < T) {
    const uint32_t k = t * 32 + lane;
    return k < cur.n ? __ldcs(lists + cur.off + k) : kNone;
  }
  const uint32_t k = (t - T) * 32 + lane;
  return k < nxt.n ? __ldcs(lists + nxt.off + k) : kNone;
}

// Loads of the first two iterations of the concatenated runs [r | nxt].
__device__ __forceinline__ Prefetch prefetch_start(const uint32_t* lists, const uint4* pts, Run r, Run nxt,
                                                   uint4 P, int lane) {
  Prefetch pf;
  const uint32_t T = (r.n + 31u) / 32u;
  pf.j0 = rec_at(lists, r, nxt, T, 0, lane);
  pf.j1 = rec_at(lists, r, nxt, T, 1, lane);
  pf.q0 = pf.j0 != kNone ? __ldg(pts + pf.j0) : P;
  return pf;
}

// The per-neighbour work of one m-range pass of the 3-D harmonics: the unit
// direction, then the pass's recurrences and one FMA per coefficient.
template <int L, int M0, int M1>
struct Step3D {
  static constexpr int NCP = round32(coef_count(L, M0, M1));
  // Each launch runs one m-pass, so the full-lane copy of the step and the
  // general one are the only code in the instruction cache.
  static constexpr bool kFullLaneLoop = true;
  const AlmArgs& a;
  __device__ __forceinline__ void operator()(float* acc, float w, float dx, float dy, float dz) const {
    const float ir = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    accum_pass<L, M0, M1>(a, acc, w, dx * ir, dy * ir, dz * ir);
  }
};

// Accumulate one pass over one run and store it to the row; the loads for
// the first iterations of `nxt` are issued inside the loop, so the next run
// starts without a memory bubble.  `step` adds one neighbour (weight and
// separation in units; a lane without a neighbour passes w = 0) to the
// Step::NCP accumulators.
template <class Step>
__device__ __forceinline__ void run_steps(const AlmArgs& a, const Step& step, Run cur, Run nxt, const uint4 P,
                                          Prefetch& pf, float* __restrict__ out, int base, float* sbuf, int lane,
                                          uint32_t pe) {
  constexpr int NCP = Step::NCP;
  const uint32_t* __restrict__ lists = a.lists;
  const uint4* __restrict__ pts = a.pts;
  float acc[NCP];
#pragma unroll
  for (int i = 0; i < NCP; ++i) acc[i] = 0.f;
  const uint32_t T = (cur.n + 31u) / 32u;
  // the second record word: the previous run could not see past this run
  // when it is a single step long, so take it from (cur, nxt)
  pf.j1 = rec_at(lists, cur, nxt, T, 1, lane);
  uint32_t t = 0;
  // Steps whose lanes all hold a neighbour and whose look-ahead words are in
  // this run: no validity tests, no run switch.  (The list buffer has slack
  // past its last entry, so the L2 prefetch needs no bound here.)
  if constexpr (Step::kFullLaneLoop) {
    const uint32_t full = cur.n >> 5;
    if (t + 3u < full) {
      // two gathers in flight: q0 = point(t), q1 = point(t + 1), j1 = word(t + 2)
      uint4 q1 = __ldg(pts + pf.j1);
      pf.j1 = __ldcs(lists + cur.off + 64u + (uint32_t)lane);
      const uint32_t* __restrict__ wp = lists + cur.off + 96u + (uint32_t)lane;
      const uint32_t* pp = lists + cur.off + kListPrefetchLines * 32u;
      const bool lane0 = lane == 0;
#pragma unroll 1
      for (; t + 3u < full; ++t) {
        if (lane0) prefetch_l2(pp);
        pp += 32;
        const uint4 q = pf.q0;
        pf.q0 = q1;
        q1 = __ldg(pts + pf.j1);
        pf.j1 = __ldcs(wp);
        wp += 32;
        const float dx = __int2float_rn((int)(q.x - P.x));
        const float dy = __int2float_rn((int)(q.y - P.y));
        const float dz = __int2float_rn((int)(q.z - P.z));
        step(acc, __uint_as_float(q.w), dx, dy, dz);
      }
      // back to one gather in flight: q0 = point(t) (valid), j1 = word(t + 1)
      pf.j0 = 0u;
      pf.j1 = rec_at(lists, cur, nxt, T, t + 1, lane);
    }
  }
  // the last steps of the run: partial lanes, look-ahead into the next run
  for (; t < T; ++t) {
    const uint32_t pa = cur.off + (t + kListPrefetchLines) * 32u;
    if (lane == 0 && pa < pe) prefetch_l2(lists + pa);
    const uint4 q = pf.q0;
    const bool valid = pf.j0 != kNone;
    pf.j0 = pf.j1;
    pf.q0 = pf.j0 != kNone ? __ldg(pts + pf.j0) : P;
    pf.j1 = rec_at(lists, cur, nxt, T, t + 2, lane);
    float dx = __int2float_rn((int)(q.x - P.x));
    float dy = __int2float_rn((int)(q.y - P.y));
    float dz = __int2float_rn((int)(q.z - P.z));
    float w = __uint_as_float(q.w);
    if (!valid) {
      dx = 1.f;
      dy = 0.f;
      dz = 0.f;
      w = 0.f;
    }
    step(acc, w, dx, dy, dz);
  }
  smem_transpose_reduce<NCP>(acc, sbuf, lane);
  // lane holds the warp totals of local slots [lane * V, lane * V + V); turn
  // them into normalised a_lm: out[s] = sum_e coef_e * total[src_e]
  // (Chebyshev moments -> Legendre values; one entry, the normalisation, for
  // slots accumulated by the Legendre recurrence)
  constexpr int V = NCP / 32;
#pragma unroll
  for (int i = 0; i < V; ++i) sbuf[lane * V + i] = acc[i];
  __syncwarp();
  float* o = out + lane * V;
#pragma unroll
  for (int i = 0; i < V; ++i) {
    const int sl = base + lane * V + i;
    const int e0 = __ldg(a.conv_off + sl), e1 = __ldg(a.conv_off + sl + 1);
    float v = 0.f;
    for (int e = e0; e < e1; ++e) v = fmaf(__ldg(a.conv_coef + e), sbuf[__ldg(a.conv_src + e) - base], v);
    acc[i] = v;
  }
  __syncwarp();
  if constexpr (V == 4) {
    __stcs(reinterpret_cast<float4*>(o), make_float4(acc[0], acc[1], acc[2], acc[3]));
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) __stcs(o + i, acc[i]);
  }
}

template <int L, int M0, int M1>
__device__ __forceinline__ void run_pass(const AlmArgs& a, Run cur, Run nxt, const uint4 P, Prefetch& pf,
                                         float* __restrict__ out, int base, float* sbuf, int lane, uint32_t pe) {
  run_steps(a, Step3D<L, M0, M1>{a}, cur, nxt, P, pf, out, base, sbuf, lane, pe);
}

// number of m-passes of kernel L, and the columns and row offset of pass P
__host__ __device__ constexpr int pass_count(int L) {
  int n = 0;
  for (int m0 = 0; m0 <= L; m0 = pass_end(L, m0, pass_cap(L, m0)) + 1) ++n;
  return n;
}
__host__ __device__ constexpr int pass_m0(int L, int P) {
  int m0 = 0;
  for (int p = 0; p < P; ++p) m0 = pass_end(L, m0, pass_cap(L, m0)) + 1;
  return m0;
}
__host__ __device__ constexpr int pass_m1(int L, int P) { return pass_end(L, pass_m0(L, P), pass_cap(L, pass_m0(L, P))); }
__host__ __device__ constexpr int pass_ncp(int L, int P) { return round32(coef_count(L, pass_m0(L, P), pass_m1(L, P))); }
__host__ __device__ constexpr int pass_base(int L, int P) {
  int b = 0;
  for (int p = 0; p < P; ++p) b += pass_ncp(L, p);
  return b;
}

// resident blocks of 4 warps the register budget of a pass is sized for
__host__ __device__ constexpr int alm_min_blocks(int ncp) { return ncp <= 64 ? 5 : (ncp <= 96 ? 4 : 3); }

__host__ __device__ constexpr size_t alm_smem_per_warp(int ncp) {
  return (size_t)32 * (ncp + 4) * sizeof(float) + 2 * kNbinsCap * sizeof(uint32_t);
}

// One warp per primary: its (primary, bin) lists are consecutive runs of the
// lists buffer; each list is accumulated in registers for m-pass P of kernel
// L and flushed once, with the next list's first loads already in flight.
//
// The passes of a kernel with several (l_max > 10) are separate kernels,
// launched one after another.  With all passes in one launch, warps in
// different passes overflowed the instruction cache; as separate kernels
// every warp on the GPU runs the same pass body, and each pass gets its own
// register budget (a pass with fewer accumulators runs more warps per SM).
// The lists are re-read once per pass; the points stay in L2.
template <int L, int P>
__global__ void __launch_bounds__(128, alm_min_blocks(pass_ncp(L, P))) k_alm(AlmArgs a) {
  constexpr int M0 = pass_m0(L, P), M1 = pass_m1(L, P), NCP = pass_ncp(L, P), BASE = pass_base(L, P);
  extern __shared__ float s_alm[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  char* wbase = reinterpret_cast<char*>(s_alm) + (size_t)warp * alm_smem_per_warp(NCP);
  float* sbuf = reinterpret_cast<float*>(wbase);
  uint32_t* s_off = reinterpret_cast<uint32_t*>(wbase + (size_t)32 * (NCP + 4) * sizeof(float));
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
      if (P == 0 && n == 0) {
        // empty bin: its row is zero (all passes' slots)
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
      const uint4 Pt = __ldg(a.pts + sp);
      int nb = b + 1;
      while (nb < nbins && s_n[nb] == 0) ++nb;
      Run cur{s_off[b], s_n[b]};
      Run nxt = nb < nbins ? Run{s_off[nb], s_n[nb]} : Run{0, 0};
      // end of this primary's list range; its first lines go to L2 now
      const uint32_t pe = s_off[nbins - 1] + s_n[nbins - 1];
      if (lane < (int)kListPrefetchLines && cur.off + (uint32_t)lane * 32u < pe)
        prefetch_l2(a.lists + cur.off + (uint32_t)lane * 32u);
      Prefetch pf = prefetch_start(a.lists, a.pts, cur, nxt, Pt, lane);
      while (true) {
        run_pass<L, M0, M1>(a, cur, nxt, Pt, pf, a.M + (ib + b) * (uint64_t)a.row + BASE, BASE, sbuf, lane, pe);
        b = nb;
        if (b >= nbins) break;
        cur = nxt;
        nb = b + 1;
        while (nb < nbins && s_n[nb] == 0) ++nb;
        nxt = nb < nbins ? Run{s_off[nb], s_n[nb]} : Run{0, 0};
      }
    }
    __syncwarp();  // s_n / s_off are rewritten for the next primary
  }
}

template <int L, int P>
int alm_occupancy_pass(int wpb) {
  const size_t smem = (size_t)wpb * alm_smem_per_warp(pass_ncp(L, P));
  if (cudaFuncSetAttribute(k_alm<L, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_alm<L, P>, wpb * 32, smem) != cudaSuccess) return 0;
  return nb;
}

// passes P.. of kernel L: each launch resident-sized from its own occupancy,
// the work counter zeroed before every pass after the first
template <int L, int P>
cudaError_t launch_passes(const AlmArgs& a, int wpb, int nsm, cudaStream_t st) {
  if constexpr (P >= pass_count(L)) {
    return cudaSuccess;
  } else {
    const size_t smem = (size_t)wpb * alm_smem_per_warp(pass_ncp(L, P));
    cudaError_t e = cudaFuncSetAttribute(k_alm<L, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int bps = alm_occupancy_pass<L, P>(wpb);
    if (bps < 1) return cudaErrorInvalidConfiguration;
    if (P > 0) {
      e = cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), st);
      if (e != cudaSuccess) return e;
    }
    k_alm<L, P><<<bps * nsm, wpb * 32, smem, st>>>(a);
    ++g_launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_passes<L, P + 1>(a, wpb, nsm, st);
  }
}

template <int L>
cudaError_t launch_alm_L(const AlmArgs& a, int wpb, int nsm, cudaStream_t st) {
  return launch_passes<L, 0>(a, wpb, nsm, st);
}

// the smallest occupancy over the passes (0: some pass cannot be resident)
template <int L, int P>
int alm_occupancy_from(int wpb) {
  if constexpr (P >= pass_count(L)) {
    return 1 << 30;
  } else {
    const int o = alm_occupancy_pass<L, P>(wpb);
    const int r = alm_occupancy_from<L, P + 1>(wpb);
    return o < r ? o : r;
  }
}

template <int L>
int alm_occupancy_L(int wpb) {
  return alm_occupancy_from<L, 0>(wpb);
}

}  // namespace ctb
