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
// lists each lane takes one neighbour per step, evaluates polynomial moments
// of the direction by recurrences in float32 registers and accumulates them
// (one paired FMA per (+m, -m) pair of moments).  Up to l_max 10 one kernel
// holds all coefficients; above, the m columns are split into passes of at
// most kPassCap accumulators, each its own kernel and launch (see k_alm).  At
// the end of the list the 32 lanes' accumulators are summed through a
// shared-memory transpose, mapped to normalised a_lm and stored as the
// (primary, bin) row of M.
// Each list is one run, so the cross-lane reduction happens once per
// (primary, bin), and the first loads of the next list are issued while the
// current one is still being accumulated.
//
// Moments (real Y_lm up to a fixed linear map per (l, m), applied at the flush):
//   (c_m + i s_m) = w (x + i y)^m        one paired FMUL + FFMA per m
//   q_k(z)        = the pass's basis: Chebyshev T_k (T_0 = 1, T_1 = z,
//                   T_k = 2z T_{k-1} - T_{k-2}: one FMA per degree) for the
//                   pass that starts at m = 0, else the monic recurrence
//                   polynomials of the pass's first column m0 (q_0 = 1,
//                   q_1 = z, q_k = z q_{k-1} - beta q_{k-2}: two per degree)
//   S_{m,k}      += q_k (c_m, s_m)       one paired FFMA per (k, +-m)
// The (1 - z^2)^{m/2} factor of the associated Legendre function is absorbed
// in (x + i y)^m.  Blackwell's paired FP32 instructions (FFMA2 / FMUL2 /
// FADD2) update the (+m, -m) accumulator pair in one issue slot; in a stream
// of independent accumulations they reach about 1.5x the FMA throughput of
// scalar FFMA on this part.
#pragma once

#include <type_traits>

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

// accumulator slot S of a float2 array: the even slot is .x, the odd .y
template <int S>
__device__ __forceinline__ float& slot_ref(float2* acc) {
  if constexpr ((S & 1) == 0) return acc[S >> 1].x;
  else return acc[S >> 1].y;
}

// Pair (k, +-M) of column M: acc += q_k (c, s) for k = K..L-M (k = 0: q_0 = 1).
template <int L, int M0, int M1, int M, int K>
__device__ __forceinline__ void column_pairs(float2* acc, const float* Q, float2 cs) {
  if constexpr (K <= L - M) {
    constexpr int i = local_slot(L, M + K, M, M0, M1) >> 1;
    if constexpr (K == 0) acc[i] = __fadd2_rn(acc[i], cs);
    else acc[i] = __ffma2_rn(make_float2(Q[K], Q[K]), cs, acc[i]);
    column_pairs<L, M0, M1, M, K + 1>(acc, Q, cs);
  }
}

// Column 0 (first pass only): acc(k, 0) += w q_k.
template <int L, int M0, int M1, int K>
__device__ __forceinline__ void column_zero(float2* acc, const float* Q, float w) {
  if constexpr (K <= L) {
    float& a = slot_ref<local_slot(L, K, 0, M0, M1)>(acc);
    a = K == 0 ? a + w : fmaf(w, Q[K], a);
    column_zero<L, M0, M1, K + 1>(acc, Q, w);
  }
}

// Columns M..ME with cs = w (x + i y)^M on entry; xy = (x, y), myx = (-y, x),
// so cs (x + i y) = cs.x xy + cs.y myx.
template <int L, int M0, int M1, int M, int ME>
__device__ __forceinline__ void columns(float2* acc, const float* Q, float2 xy, float2 myx, float2 cs) {
  if constexpr (M <= ME) {
    column_pairs<L, M0, M1, M, 0>(acc, Q, cs);
    if constexpr (M + 1 <= ME) {
      const float2 nx = __ffma2_rn(make_float2(cs.x, cs.x), xy, __fmul2_rn(make_float2(cs.y, cs.y), myx));
      columns<L, M0, M1, M + 1, ME>(acc, Q, xy, myx, nx);
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

// q_k = p^{M0}_{M0+k}(z), k = K..KMAX: q_k = z q_{k-1} - beta_{M0+k, M0} q_{k-2}.
template <int M0, int K, int KMAX>
__device__ __forceinline__ void basis_seq(const AlmArgs& a, float* Q, float z) {
  if constexpr (K <= KMAX) {
    Q[K] = fmaf(z, Q[K - 1], -(a.beta[(M0 + K) * (kLmaxCap + 1) + M0] * Q[K - 2]));
    basis_seq<M0, K + 1, KMAX>(a, Q, z);
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

// Degree-major order for passes of few columns: the powers of all columns
// first, then per degree k the next basis polynomial and the moments of
// every column that reaches degree k.  Only three basis values are live at a
// time (against all L - m0 + 1 in column-major order), which keeps the wide
// passes of l_max 20 within their register budget.
template <int L, int M0, int M1, int K, int KMAX, int MS, int ME>
__device__ __forceinline__ void degrees(const AlmArgs& a, float2* acc, const float2* cs, float w, float z, float z2,
                                        float q2, float q1) {
  if constexpr (K <= KMAX) {
    float q;
    if constexpr (K == 0) q = 1.f;
    else if constexpr (K == 1) q = z;
    else if constexpr (M0 == 0) q = fmaf(z2, q1, -q2);
    else q = fmaf(z, q1, -(a.beta[(M0 + K) * (kLmaxCap + 1) + M0] * q2));
    if constexpr (M0 == 0) {
      float& c0 = slot_ref<local_slot(L, K, 0, M0, M1)>(acc);
      c0 = K == 0 ? c0 + w : fmaf(w, q, c0);
    }
#pragma unroll
    for (int m = MS; m <= ME; ++m) {
      if (K <= L - m) {
        const int i = local_slot(L, m + K, m, M0, M1) >> 1;
        if (K == 0) acc[i] = __fadd2_rn(acc[i], cs[m - MS]);
        else acc[i] = __ffma2_rn(make_float2(q, q), cs[m - MS], acc[i]);
      }
    }
    degrees<L, M0, M1, K + 1, KMAX, MS, ME>(a, acc, cs, w, z, z2, q1, q);
  }
}

// columns of a pass that is accumulated degree-major
__host__ __device__ constexpr bool degree_major(int L, int m0, int m1) {
  return (m1 < L ? m1 : L) - (m0 < 1 ? 1 : m0) + 1 <= 5;
}

// Add one neighbour (weight w, unit direction x, y, z) to the pass's
// accumulators: the pass's basis sequence, the complex powers, and one
// paired FMA per (k, +-m) moment (one FMA per moment of column 0).
template <int L, int M0, int M1>
__device__ __forceinline__ void accum_pass(const AlmArgs& a, float2* acc, float w, float x, float y, float z) {
  constexpr int KMAX = L - M0;  // highest basis degree this pass needs
  constexpr int MS = M0 < 1 ? 1 : M0;
  constexpr int ME = M1 < L ? M1 : L;
  if constexpr (degree_major(L, M0, M1)) {
    constexpr int NC = ME >= MS ? ME - MS + 1 : 1;
    float2 cs[NC];
    if constexpr (MS <= ME) {
      float pr, pi;
      cpow<MS>(x, y, pr, pi);
      cs[0] = make_float2(w * pr, w * pi);
      const float2 xy = make_float2(x, y), myx = make_float2(-y, x);
#pragma unroll
      for (int c = 1; c < NC; ++c)
        cs[c] = __ffma2_rn(make_float2(cs[c - 1].x, cs[c - 1].x), xy, __fmul2_rn(make_float2(cs[c - 1].y, cs[c - 1].y), myx));
    }
    degrees<L, M0, M1, 0, KMAX, MS, ME>(a, acc, cs, w, z, z + z, 0.f, 0.f);
  } else {
    float Q[KMAX + 1 > 2 ? KMAX + 1 : 2];
    Q[0] = 1.f;
    Q[1] = z;
    if constexpr (M0 == 0) cheb_seq<2, KMAX>(Q, z + z);
    else basis_seq<M0, 2, KMAX>(a, Q, z);
    if constexpr (M0 == 0) column_zero<L, M0, M1, 0>(acc, Q, w);
    if constexpr (MS <= ME) {
      float pr, pi;
      cpow<MS>(x, y, pr, pi);  // (x + i y)^MS by squaring
      columns<L, M0, M1, MS, ME>(acc, Q, make_float2(x, y), make_float2(-y, x), make_float2(w * pr, w * pi));
    }
  }
}

// Cross-lane sum of the accumulators through shared memory, in chunks of
// at most kFlushChunk slots: every lane writes its chunk (stride W + 4 floats,
// so 16-byte stores of 8 consecutive lanes cover all 32 banks), then lane l
// sums the chunk's column block [l * W/32, (l+1) * W/32) over the 32 rows and
// writes the totals to tot[chunk start + that block].
constexpr int kFlushChunk = 64;
__host__ __device__ constexpr int flush_buf_floats(int ncp) {
  return 32 * ((ncp < kFlushChunk ? ncp : kFlushChunk) + 4);
}

template <int NCP, int C0>
__device__ __forceinline__ void flush_chunks(const float2* acc, float* buf, float* tot, int lane) {
  if constexpr (C0 < NCP) {
    constexpr int W = NCP - C0 < kFlushChunk ? NCP - C0 : kFlushChunk;
    constexpr int S = W + 4;
    constexpr int V = W / 32;
    float* row = buf + lane * S;
#pragma unroll
    for (int i = 0; i < W / 2; i += 2)
      *reinterpret_cast<float4*>(row + 2 * i) =
          make_float4(acc[C0 / 2 + i].x, acc[C0 / 2 + i].y, acc[C0 / 2 + i + 1].x, acc[C0 / 2 + i + 1].y);
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
      *reinterpret_cast<float4*>(tot + C0 + 4 * lane) =
          make_float4(s0.x + s1.x, s0.y + s1.y, s0.z + s1.z, s0.w + s1.w);
    } else if constexpr (V == 2) {
      float2 s0 = make_float2(0.f, 0.f), s1 = s0;
#pragma unroll
      for (int r = 0; r < 32; r += 2) {
        const float2 u = *reinterpret_cast<const float2*>(buf + r * S + 2 * lane);
        const float2 v = *reinterpret_cast<const float2*>(buf + (r + 1) * S + 2 * lane);
        s0.x += u.x; s0.y += u.y;
        s1.x += v.x; s1.y += v.y;
      }
      *reinterpret_cast<float2*>(tot + C0 + 2 * lane) = make_float2(s0.x + s1.x, s0.y + s1.y);
    } else {
      float sm[V];
#pragma unroll
      for (int c = 0; c < V; ++c) sm[c] = 0.f;
#pragma unroll
      for (int r = 0; r < 32; ++r)
#pragma unroll
        for (int c = 0; c < V; ++c) sm[c] += buf[r * S + V * lane + c];
#pragma unroll
      for (int c = 0; c < V; ++c) tot[C0 + V * lane + c] = sm[c];
    }
    __syncwarp();  // the buffer is rewritten by the next chunk
    flush_chunks<NCP, C0 + W>(acc, buf, tot, lane);
  }
}

// Flush conversion of one pass, padded to E entries per slot and stored
// entry-major in shared memory: entry e of local slot s at tab[e * NCP + s],
// as (source local slot, coefficient bits); unused entries have coefficient
// 0.  Lane l maps slots l, l + 32, ...: out[s] = sum_e coef * tot[src], the
// loads of every entry independent of each other.
template <int NCP, int E>
__device__ __forceinline__ void flush_store(const int2* tab, const float* tot, float* __restrict__ out, int lane) {
#pragma unroll
  for (int i = 0; i < NCP / 32; ++i) {
    const int s = lane + 32 * i;
    float v = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int2 t = tab[e * NCP + s];
      v = fmaf(__int_as_float(t.y), tot[t.x], v);
    }
    __stcs(out + s, v);
  }
}

// One neighbour list run: records [off, off + n) of the lists buffer.
struct Run {
  uint32_t off, n;
};

// Loads in flight, for steps t, t + 1 and t + 2 of the concatenated runs:
// the neighbours of the next two steps (q0, q1; j0, j1 their record words,
// kNone for a lane without one) and the record word of the step after.
struct Prefetch {
  uint32_t j0, j1, j2;
  uint4 q0, q1;
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

__device__ __forceinline__ uint4 gather(const uint4* __restrict__ pts, uint32_t j, uint4 P) {
  return j != kNone ? __ldg(pts + j) : P;
}

// Loads of the first three iterations of the concatenated runs [r | nxt].
__device__ __forceinline__ Prefetch prefetch_start(const uint32_t* lists, const uint4* pts, Run r, Run nxt,
                                                   uint4 P, int lane) {
  Prefetch pf;
  const uint32_t T = (r.n + 31u) / 32u;
  pf.j0 = rec_at(lists, r, nxt, T, 0, lane);
  pf.j1 = rec_at(lists, r, nxt, T, 1, lane);
  pf.j2 = rec_at(lists, r, nxt, T, 2, lane);
  pf.q0 = gather(pts, pf.j0, P);
  pf.q1 = gather(pts, pf.j1, P);
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
  // flush conversion entries per slot: moment degrees of the same parity
  static constexpr int kConvE = conv_entries(L, M0);
  const AlmArgs& a;
  __device__ __forceinline__ void operator()(float2* acc, float w, float dx, float dy, float dz) const {
    const float ir = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    accum_pass<L, M0, M1>(a, acc, w, dx * ir, dy * ir, dz * ir);
  }
  // The unit direction and weight of a neighbour, ahead of its
  // accumulation.  The full-lane loop of a single-pass kernel (l_max <= 10)
  // prepares each step's direction one iteration ahead (5 % faster at
  // l_max 10); in the 255-register passes of l_max 20 the extra live state
  // made the pass slower, so they keep the plain step.
  __device__ __forceinline__ float4 prep(uint4 q, uint4 P) const {
    const float dx = __int2float_rn((int)(q.x - P.x));
    const float dy = __int2float_rn((int)(q.y - P.y));
    const float dz = __int2float_rn((int)(q.z - P.z));
    const float ir = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    return make_float4(dx * ir, dy * ir, dz * ir, __uint_as_float(q.w));
  }
  __device__ __forceinline__ void accum(float2* acc, float4 s) const { accum_pass<L, M0, M1>(a, acc, s.w, s.x, s.y, s.z); }
  static constexpr bool kPrep = L <= kSinglePassLmax;
};

template <class S, class = void>
struct has_prep : std::false_type {};
template <class S>
struct has_prep<S, std::void_t<decltype(&S::prep)>> : std::true_type {};
template <class S>
__host__ __device__ constexpr bool use_prep() {
  if constexpr (has_prep<S>::value) return S::kPrep;
  else return false;
}

// Accumulate one pass over one run and store it to the row; the loads for
// the first iterations of `nxt` are issued inside the loop, so the next run
// starts without a memory bubble.  `step` adds one neighbour (weight and
// separation in units; a lane without a neighbour passes w = 0) to the
// Step::NCP accumulators.
template <class Step>
__device__ __forceinline__ void run_steps(const AlmArgs& a, const Step& step, Run cur, Run nxt, const uint4 P,
                                          Prefetch& pf, float* __restrict__ out, const int2* ctab, float* sbuf,
                                          int lane, uint32_t pe) {
  constexpr int NCP = Step::NCP;
  const uint32_t* __restrict__ lists = a.lists;
  const uint4* __restrict__ pts = a.pts;
  float2 acc[NCP / 2];
#pragma unroll
  for (int i = 0; i < NCP / 2; ++i) acc[i] = make_float2(0.f, 0.f);
  const uint32_t T = (cur.n + 31u) / 32u;
  // Steps 1 and 2 of [cur | nxt]: the previous run looked only one run
  // ahead, so when cur is shorter than that they are taken again here.
  {
    const uint32_t w1 = rec_at(lists, cur, nxt, T, 1, lane);
    if (w1 != pf.j1) {
      pf.j1 = w1;
      pf.q1 = gather(pts, w1, P);
    }
    pf.j2 = rec_at(lists, cur, nxt, T, 2, lane);
  }
  uint32_t t = 0;
  // Steps whose lanes all hold a neighbour and whose look-ahead words are in
  // this run: no validity tests, no run switch.  (The list buffer has slack
  // past its last entry, so the L2 prefetch needs no bound here.)  Two
  // neighbour gathers are in flight and the record word one step before
  // its gather.
  if constexpr (Step::kFullLaneLoop) {
    const uint32_t full = cur.n >> 5;
    if (t + 3u < full) {
      const uint32_t* __restrict__ wp = lists + cur.off + 96u + (uint32_t)lane;
      const uint32_t* pp = lists + cur.off + kListPrefetchLines * 32u;
      const bool lane0 = lane == 0;
      uint4 q0 = pf.q0, q1 = pf.q1;
      uint32_t j2 = pf.j2;
      if constexpr (use_prep<Step>()) {
        // each step's direction is prepared one iteration ahead, so its
        // dependent chain overlaps the previous step's accumulation
        float4 S = step.prep(q0, P);
#pragma unroll 1
        for (; t + 3u < full; ++t) {
          if (lane0) prefetch_l2(pp);
          pp += 32;
          const float4 Sn = step.prep(q1, P);
          q0 = q1;
          q1 = __ldg(pts + j2);
          j2 = __ldcs(wp);
          wp += 32;
          step.accum(acc, S);
          S = Sn;
        }
      } else {
#pragma unroll 1
        for (; t + 3u < full; ++t) {
          if (lane0) prefetch_l2(pp);
          pp += 32;
          const uint4 q = q0;
          q0 = q1;
          q1 = __ldg(pts + j2);
          j2 = __ldcs(wp);
          wp += 32;
          const float dx = __int2float_rn((int)(q.x - P.x));
          const float dy = __int2float_rn((int)(q.y - P.y));
          const float dz = __int2float_rn((int)(q.z - P.z));
          step(acc, __uint_as_float(q.w), dx, dy, dz);
        }
      }
      // t + 1 and t + 2 are full-lane steps of this run
      pf.q0 = q0;
      pf.q1 = q1;
      pf.j0 = 0u;
      pf.j1 = 0u;
      pf.j2 = j2;
    }
  }
  // the last steps of the run: partial lanes, look-ahead into the next run,
  // the same two gathers in flight
  for (; t < T; ++t) {
    const uint32_t pa = cur.off + (t + kListPrefetchLines) * 32u;
    if (lane == 0 && pa < pe) prefetch_l2(lists + pa);
    const uint4 q = pf.q0;
    const bool valid = pf.j0 != kNone;
    pf.q0 = pf.q1;
    pf.j0 = pf.j1;
    pf.q1 = gather(pts, pf.j2, P);
    pf.j1 = pf.j2;
    pf.j2 = rec_at(lists, cur, nxt, T, t + 3, lane);
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
  // Warp totals, in chunks of at most kFlushChunk slots through the
  // transpose buffer, into tot[slot]; then every lane maps its slots' totals
  // to normalised a_lm: out[s] = sum_e coef_e * tot[src_e] (moments in the
  // pass's basis -> the Legendre values of their column).
  float* tot = sbuf + flush_buf_floats(NCP);
  flush_chunks<NCP, 0>(acc, sbuf, tot, lane);
  __syncwarp();
  flush_store<NCP, Step::kConvE>(ctab, tot, out, lane);
  __syncwarp();
}

template <int L, int M0, int M1>
__device__ __forceinline__ void run_pass(const AlmArgs& a, Run cur, Run nxt, const uint4 P, Prefetch& pf,
                                         float* __restrict__ out, const int2* ctab, float* sbuf, int lane,
                                         uint32_t pe) {
  run_steps(a, Step3D<L, M0, M1>{a}, cur, nxt, P, pf, out, ctab, sbuf, lane, pe);
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
// entries of the padded conversion tables of the passes before P
__host__ __device__ constexpr int conv_pass_offset(int L, int P) {
  int b = 0;
  for (int p = 0; p < P; ++p) b += pass_ncp(L, p) * conv_entries(L, pass_m0(L, p));
  return b;
}
__host__ __device__ constexpr size_t alm_table_bytes(int L, int P) {
  return (size_t)pass_ncp(L, P) * conv_entries(L, pass_m0(L, P)) * sizeof(int2);
}

// resident blocks of 4 warps the register budget of a pass is sized for
// (each of the SM's four schedulers holds a quarter of the registers: 2
// warps per scheduler allow 255 registers a thread, 3 allow 168, 4 allow 128)
__host__ __device__ constexpr int alm_min_blocks(int ncp) { return ncp <= 32 ? 5 : (ncp <= 64 ? 4 : (ncp <= 136 ? 3 : 2)); }

// per warp: the flush's transpose buffer, the slot totals, then the
// primary's list offsets and counts
__host__ __device__ constexpr size_t alm_smem_per_warp(int ncp) {
  return (size_t)(flush_buf_floats(ncp) + ncp) * sizeof(float) + 2 * kNbinsCap * sizeof(uint32_t);
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
  constexpr int NTAB = NCP * conv_entries(L, M0);
  extern __shared__ float s_alm[];
  // [the pass's conversion table | per warp: flush buffers, list offsets, counts]
  int2* s_tab = reinterpret_cast<int2*>(s_alm);
  for (int k = threadIdx.x; k < NTAB; k += blockDim.x) s_tab[k] = __ldg(a.conv + conv_pass_offset(L, P) + k);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  char* wbase = reinterpret_cast<char*>(s_alm) + alm_table_bytes(L, P) + (size_t)warp * alm_smem_per_warp(NCP);
  float* sbuf = reinterpret_cast<float*>(wbase);
  uint32_t* s_off = reinterpret_cast<uint32_t*>(wbase + (size_t)(flush_buf_floats(NCP) + NCP) * sizeof(float));
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
        run_pass<L, M0, M1>(a, cur, nxt, Pt, pf, a.M + (ib + b) * (uint64_t)a.row + BASE, s_tab, sbuf, lane, pe);
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
  const size_t smem = alm_table_bytes(L, P) + (size_t)wpb * alm_smem_per_warp(pass_ncp(L, P));
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
    const size_t smem = alm_table_bytes(L, P) + (size_t)wpb * alm_smem_per_warp(pass_ncp(L, P));
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
