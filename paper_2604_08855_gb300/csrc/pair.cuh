// pair.cuh -- the pair-multipole kernel (template; instantiated per ell_max in
// pair_[a-f].cu so the instantiations compile in parallel).
//
// Paper, "Implementation": pick a pivot, find all its neighbours inside the
// search range, fill the multipole bins; sin/cos of the angle are replaced by
// a polynomial recurrence because evaluating trigonometric functions is slow.
// "Performance": the time goes into scanning for neighbours and updating the
// histograms, with a per-multipole recurrence cost.
//
// GB300 design.  One warp owns one primary p at a time (persistent warps fetch
// primaries from a global counter).  For p it
//   1. walks the x-rows of grid cells that intersect the ball r < r_max
//      (each row is one contiguous run of cell-sorted points: coalesced
//      16-byte loads, 32 candidates per step);
//   2. bins every candidate (exact fixed-point separation, float32 r^2) and
//      appends its index to a per-warp, per-bin list in global scratch, in
//      stream order (match_any ranks lanes with equal bins);
//   3. when a list is nearly full, and at the end, processes one bin: each lane
//      takes one neighbour per step, evaluates all (l, m) coefficients of the
//      direction by recurrences in float32 registers and accumulates them
//      (one FMA per coefficient); a transposing butterfly of warp shuffles
//      then sums the 32 lanes' accumulators and the lane-owned slices are
//      scaled by the normalisation and written to the primary's row of M.
// Processing a bin as one long run is what keeps the accumulators in
// registers: the cross-lane reduction happens once per (primary, bin) run,
// not once per neighbour.
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

// Column m >= 1 of the recurrence, l = LL..L (template recursion keeps every
// accumulator index a compile-time constant, so the array stays in registers).
template <int L, int M0, int M1, int M, int LL>
__device__ __forceinline__ void column_rec(const PairArgs& a, float* acc, float z, float cr, float ci, float p2,
                                           float p1) {
  if constexpr (LL <= L) {
    const float p = fmaf(z, p1, -(a.beta[LL * (kLmaxCap + 1) + M] * p2));
    acc[local_slot(LL, M, M0, M1)] = fmaf(p, cr, acc[local_slot(LL, M, M0, M1)]);
    acc[local_slot(LL, -M, M0, M1)] = fmaf(p, ci, acc[local_slot(LL, -M, M0, M1)]);
    column_rec<L, M0, M1, M, LL + 1>(a, acc, z, cr, ci, p1, p);
  }
}

// Column m = 0, l = LL..L.
template <int L, int M0, int M1, int LL>
__device__ __forceinline__ void column0_rec(const PairArgs& a, float* acc, float w, float z, float p2, float p1) {
  if constexpr (LL <= L) {
    const float p = fmaf(z, p1, -(a.beta[LL * (kLmaxCap + 1)] * p2));
    acc[local_slot(LL, 0, M0, M1)] = fmaf(w, p, acc[local_slot(LL, 0, M0, M1)]);
    column0_rec<L, M0, M1, LL + 1>(a, acc, w, z, p1, p);
  }
}

// Columns m = M..ME with (cr, ci) = w (x + i y)^M on entry.
template <int L, int M0, int M1, int M, int ME>
__device__ __forceinline__ void columns_rec(const PairArgs& a, float* acc, float x, float y, float z, float cr,
                                            float ci) {
  if constexpr (M <= ME) {
    acc[local_slot(M, M, M0, M1)] += cr;
    acc[local_slot(M, -M, M0, M1)] += ci;
    if constexpr (M + 1 <= L) {
      acc[local_slot(M + 1, M, M0, M1)] = fmaf(z, cr, acc[local_slot(M + 1, M, M0, M1)]);
      acc[local_slot(M + 1, -M, M0, M1)] = fmaf(z, ci, acc[local_slot(M + 1, -M, M0, M1)]);
    }
    column_rec<L, M0, M1, M, M + 2>(a, acc, z, cr, ci, 1.f, z);
    if constexpr (M + 1 <= ME) {
      const float nr = fmaf(cr, x, -(ci * y));
      const float ni = fmaf(cr, y, ci * x);
      columns_rec<L, M0, M1, M + 1, ME>(a, acc, x, y, z, nr, ni);
    }
  }
}

// Add one neighbour (weight w, unit direction x, y, z) to the pass's
// accumulators: one FMA per coefficient plus the recurrences.
template <int L, int M0, int M1>
__device__ __forceinline__ void accum_pass(const PairArgs& a, float* acc, float w, float x, float y, float z) {
  if constexpr (M0 == 0) {
    acc[local_slot(0, 0, M0, M1)] += w;
    if constexpr (L >= 1) acc[local_slot(1, 0, M0, M1)] = fmaf(w, z, acc[local_slot(1, 0, M0, M1)]);
    column0_rec<L, M0, M1, 2>(a, acc, w, z, 1.f, z);
  }
  constexpr int MS = M0 < 1 ? 1 : M0;
  constexpr int ME = M1 < L ? M1 : L;
  if constexpr (MS <= ME) {
    float cr = w * x, ci = w * y;  // w (x + i y)^1
#pragma unroll
    for (int k = 1; k < MS; ++k) {
      const float t = fmaf(cr, x, -(ci * y));
      ci = fmaf(cr, y, ci * x);
      cr = t;
    }
    columns_rec<L, M0, M1, MS, ME>(a, acc, x, y, z, cr, ci);
  }
}

// One butterfly level: lanes with (lane & mask) keep the upper half of v and
// send the lower half to their partner, and vice versa; V values -> V/2.
template <int V>
__device__ __forceinline__ void bfly(float* v, int lane, int mask) {
  const bool up = (lane & mask) != 0;
#pragma unroll
  for (int i = 0; i < V / 2; ++i) {
    float send = up ? v[i] : v[i + V / 2];
    float keep = up ? v[i + V / 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
  }
}

// Sum NCP values over the warp; afterwards lane l holds the totals of slots
// [l * NCP/32, (l+1) * NCP/32) in v[0 .. NCP/32).
template <int NCP>
__device__ __forceinline__ void warp_transpose_reduce(float* v, int lane) {
  bfly<NCP>(v, lane, 16);
  bfly<NCP / 2>(v, lane, 8);
  bfly<NCP / 4>(v, lane, 4);
  bfly<NCP / 8>(v, lane, 2);
  bfly<NCP / 16>(v, lane, 1);
}

// Accumulate one m-range pass of one bin run and write/add it to the row.
template <int L, int M0, int M1>
__device__ __forceinline__ void run_pass(const PairArgs& a, const uint32_t* __restrict__ list, uint32_t n,
                                         const uint4 P,
                                         const uint4* __restrict__ pts, float* __restrict__ out,
                                         const float* __restrict__ norm, bool first, int lane) {
  constexpr int NCP = round32(coef_count(L, M0, M1));
  float acc[NCP];
#pragma unroll
  for (int i = 0; i < NCP; ++i) acc[i] = 0.f;
  const uint32_t nr = (n + 31u) & ~31u;
  uint32_t k = lane;
  uint32_t j0 = k < n ? __ldcg(list + k) : kNone;
  uint32_t j1 = k + 32 < n ? __ldcg(list + k + 32) : kNone;
  uint4 q0 = j0 != kNone ? __ldg(pts + j0) : P;
  for (; k < nr; k += 32) {
    const uint4 q = q0;
    const bool valid = j0 != kNone;
    j0 = j1;
    q0 = j0 != kNone ? __ldg(pts + j0) : P;
    j1 = k + 64 < n ? __ldcg(list + k + 64) : kNone;
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
    const float ir = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    accum_pass<L, M0, M1>(a, acc, w, dx * ir, dy * ir, dz * ir);
  }
  warp_transpose_reduce<NCP>(acc, lane);
  constexpr int V = NCP / 32;
  float* o = out + lane * V;
  const float* nm = norm + lane * V;
  if constexpr (V % 4 == 0) {
#pragma unroll
    for (int i = 0; i < V; i += 4) {
      float4 s = __ldg(reinterpret_cast<const float4*>(nm + i));
      float4 r = make_float4(acc[i] * s.x, acc[i + 1] * s.y, acc[i + 2] * s.z, acc[i + 3] * s.w);
      if (first)
        *reinterpret_cast<float4*>(o + i) = r;
      else
        atomicAdd(reinterpret_cast<float4*>(o + i), r);
    }
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) {
      float r = acc[i] * __ldg(nm + i);
      if (first)
        o[i] = r;
      else
        atomicAdd(o + i, r);
    }
  }
}

template <int L, int M0, int BASE>
struct PassChain {
  static constexpr int M1 = pass_end(L, M0, kPassCap);
  static constexpr int NCP = round32(coef_count(L, M0, M1));
  __device__ static __forceinline__ void run(const PairArgs& a, const uint32_t* list, uint32_t n, const uint4 P,
                                             const uint4* pts, float* out, const float* norm, bool first,
                                             int lane) {
    run_pass<L, M0, M1>(a, list, n, P, pts, out + BASE, norm + BASE, first, lane);
    if constexpr (M1 + 1 <= L) PassChain<L, M1 + 1, BASE + NCP>::run(a, list, n, P, pts, out, norm, first, lane);
  }
};

__device__ __forceinline__ float slab_dist(int d, float fr) {
  return d > 0 ? (float)d - fr : (d < 0 ? (float)(-d - 1) + fr : 0.f);
}

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

template <int L>
__global__ void __launch_bounds__(128, 3) k_pair(PairArgs a) {
  extern __shared__ uint32_t s_dyn[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const Geom g = a.g;
  const int nbins = g.nbins;
  uint32_t* cnt = s_dyn + warp * kNbinsCap;
  const uint64_t gw = (uint64_t)blockIdx.x * wpb + warp;
  uint32_t* lists = a.lists + gw * (uint64_t)nbins * a.cap;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t nc = g.nc;
  const float R2 = g.rcell * g.rcell;
  const int K = (int)floorf(g.rcell) + 1;
  int W = 2 * K + 1, off0 = -K;
  bool fullwin = false;
  if (g.periodic && W >= (int)nc) {
    W = (int)nc;
    off0 = -(((int)nc - 1) / 2);
    fullwin = true;
  }
  const int nrows = W * W;
  const uint64_t lowmask = (1ull << g.shift) - 1ull;
  const float frac_scale = 1.0f / (float)(1ull << g.shift);
  unsigned long long my_pairs = 0;

  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.work, 2ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= (unsigned long long)a.prim_count) break;
    const int64_t iend = min((int64_t)base + 2, a.prim_count);
    for (int64_t i = (int64_t)base; i < iend; ++i) {
      const int64_t gi = a.prim_begin + i;
      const uint32_t sp = a.prim ? a.prim[gi] : (uint32_t)gi;
      const uint4 P = __ldg(a.pts + sp);
      if (lane == 0) a.wprim[i] = __uint_as_float(P.w);
      if (lane < nbins) cnt[lane] = 0;
      if (lane + 32 < nbins) cnt[lane + 32] = 0;
      __syncwarp();
      float* Mrow = a.M + (uint64_t)i * nbins * a.row;

      // primary position in cell units
      const uint64_t sx = (uint64_t)P.x * nc, sy = (uint64_t)P.y * nc, sz = (uint64_t)P.z * nc;
      const int cxp = (int)(sx >> g.shift), cyp = (int)(sy >> g.shift), czp = (int)(sz >> g.shift);
      const float frx = (float)(sx & lowmask) * frac_scale;
      const float fry = (float)(sy & lowmask) * frac_scale;
      const float frz = (float)(sz & lowmask) * frac_scale;
      const float fx = (float)cxp + frx;

      // stream state
      int t0 = 0;
      uint32_t s0 = 0, e0 = 0, s1 = 0, e1 = 0;  // this lane's row segments
      unsigned pend = 0;                         // lanes with unconsumed segments
      uint32_t cs = 0, ce = 0;                   // current segment (warp-uniform)
      bool streaming = true;
      int drain = 0;
      uint64_t pending_bins = 0, flushed = 0;

      while (true) {
        int pb = -1;
        if (pending_bins) {
          pb = __ffsll((long long)pending_bins) - 1;
          pending_bins &= pending_bins - 1;
        } else if (streaming) {
          // ---- advance to a non-empty segment
          while (cs >= ce) {
            if (pend == 0) {
              if (t0 >= nrows) break;
              const int t = t0 + lane;
              s0 = e0 = s1 = e1 = 0;
              if (t < nrows) {
                const int dy = t % W + off0, dz = t / W + off0;
                float gy = slab_dist(dy, fry), gz = slab_dist(dz, frz);
                if (fullwin) {
                  gy = fminf(gy, fminf(slab_dist(dy - (int)nc, fry), slab_dist(dy + (int)nc, fry)));
                  gz = fminf(gz, fminf(slab_dist(dz - (int)nc, frz), slab_dist(dz + (int)nc, frz)));
                }
                const float rho2 = gy * gy + gz * gz;
                int cy = cyp + dy, cz = czp + dz;
                bool ok = rho2 < R2;
                if (g.periodic) {
                  cy = pmod(cy, (int)nc);
                  cz = pmod(cz, (int)nc);
                } else {
                  ok = ok && cy >= 0 && cy < (int)nc && cz >= 0 && cz < (int)nc;
                }
                if (ok) {
                  const float hw = sqrtf(R2 - rho2);
                  int lo = (int)floorf(fx - hw), hi = (int)floorf(fx + hw);
                  const uint32_t rb = ((uint32_t)cz * nc + (uint32_t)cy) * nc;
                  int a0 = 1, b0 = 0, a1 = 1, b1 = 0;
                  if (g.periodic) {
                    if (hi - lo + 1 >= (int)nc) {
                      a0 = 0;
                      b0 = (int)nc - 1;
                    } else {
                      const int lm = pmod(lo, (int)nc), hm = pmod(hi, (int)nc);
                      if (lm <= hm) {
                        a0 = lm;
                        b0 = hm;
                      } else {
                        a0 = lm;
                        b0 = (int)nc - 1;
                        a1 = 0;
                        b1 = hm;
                      }
                    }
                  } else {
                    lo = max(lo, 0);
                    hi = min(hi, (int)nc - 1);
                    a0 = lo;
                    b0 = hi;
                  }
                  if (a0 <= b0) {
                    s0 = __ldg(a.cell_start + rb + a0);
                    e0 = __ldg(a.cell_start + rb + b0 + 1);
                  }
                  if (a1 <= b1) {
                    s1 = __ldg(a.cell_start + rb + a1);
                    e1 = __ldg(a.cell_start + rb + b1 + 1);
                  }
                }
              }
              t0 += 32;
              pend = __ballot_sync(0xffffffffu, s0 < e0 || s1 < e1);
              continue;
            }
            const int src = __ffs(pend) - 1;
            const bool h0 = __shfl_sync(0xffffffffu, s0 < e0, src);
            const uint32_t ns = __shfl_sync(0xffffffffu, h0 ? s0 : s1, src);
            const uint32_t ne = __shfl_sync(0xffffffffu, h0 ? e0 : e1, src);
            if (lane == src) {
              if (h0) s0 = e0;
              else s1 = e1;
            }
            cs = ns;
            ce = ne;
            pend = __ballot_sync(0xffffffffu, s0 < e0 || s1 < e1);
          }
          if (cs >= ce) {
            streaming = false;
            continue;
          }
          // ---- one step of 32 candidates
          const uint32_t j = cs + lane;
          const bool valid = j < ce;
          const uint4 q = valid ? __ldg(a.pts + j) : P;
          const float dx = __int2float_rn((int)(q.x - P.x));
          const float dy = __int2float_rn((int)(q.y - P.y));
          const float dz = __int2float_rn((int)(q.z - P.z));
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          bool inb = valid && r2 > 0.f && r2 >= g.rlo2_u && r2 < g.rhi2_u;
          int b = 0;
          if (inb) {
            const float r = r2 * rsqrtf(r2);
            const float t = (r - g.rmin_u) * g.inv_dr_u;
            b = (int)floorf(t);
            const float fr = t - (float)b;
            if (b < 0 || b >= nbins || fr < 1e-4f || fr > 1.f - 1e-4f) {
              // within float rounding of an edge: decide on the exact squared
              // separation (integer units^2) against the exact thresholds
              const long long ix = (int)(q.x - P.x), iy = (int)(q.y - P.y), iz = (int)(q.z - P.z);
              const unsigned long long e2 = (unsigned long long)(ix * ix + iy * iy + iz * iz);
              if (e2 == 0ull || e2 < __ldg(a.thr) || e2 >= __ldg(a.thr + nbins)) {
                inb = false;
              } else {
                b = min(max(b, 0), nbins - 1);
                while (e2 < __ldg(a.thr + b)) --b;
                while (e2 >= __ldg(a.thr + b + 1)) ++b;
              }
            }
          }
          const unsigned act = __ballot_sync(0xffffffffu, inb);
          bool full = false;
          if (inb) {
            const unsigned grp = __match_any_sync(act, b);
            const unsigned rank = __popc(grp & lt);
            const uint32_t c0 = cnt[b];
            __syncwarp(act);
            lists[(uint64_t)b * a.cap + c0 + rank] = j;
            const uint32_t c1 = c0 + __popc(grp);
            if (rank == 0) cnt[b] = c1;
            full = c1 + 32 > a.cap;
          }
          __syncwarp();
          my_pairs += __popc(act);
          const unsigned flo = __reduce_or_sync(0xffffffffu, (full && b < 32) ? (1u << b) : 0u);
          const unsigned fhi = __reduce_or_sync(0xffffffffu, (full && b >= 32) ? (1u << (b - 32)) : 0u);
          pending_bins |= ((uint64_t)fhi << 32) | flo;
          cs += 32;
          continue;
        } else {
          // ---- drain the remaining bins in order
          while (drain < nbins && cnt[drain] == 0) {
            if (!((flushed >> drain) & 1ull)) {
              float4* o = reinterpret_cast<float4*>(Mrow + (uint64_t)drain * a.row);
              for (int k = lane; k < a.row / 4; k += 32) o[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            ++drain;
          }
          if (drain >= nbins) break;
          pb = drain++;
        }
        // ---- process bin pb
        const uint32_t n = cnt[pb];
        const bool first = !((flushed >> pb) & 1ull);
        PassChain<L, 0, 0>::run(a, lists + (uint64_t)pb * a.cap, n, P, a.pts, Mrow + (uint64_t)pb * a.row, a.norm,
                                first, lane);
        __syncwarp();
        if (lane == 0) cnt[pb] = 0;
        __syncwarp();
        flushed |= 1ull << pb;
      }
    }
  }
  if (lane == 0 && my_pairs) atomicAdd(a.npairs, my_pairs);
}

template <int L>
cudaError_t launch_pair_L(const PairArgs& a, int wpb, int nblocks, cudaStream_t st) {
  size_t smem = (size_t)wpb * kNbinsCap * sizeof(uint32_t);
  k_pair<L><<<nblocks, wpb * 32, smem, st>>>(a);
  ++g_launches;
  return cudaGetLastError();
}

template <int L>
int pair_occupancy_L(int wpb) {
  int nb = 0;
  size_t smem = (size_t)wpb * kNbinsCap * sizeof(uint32_t);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pair<L>, wpb * 32, smem) != cudaSuccess) return 0;
  return nb;
}

}  // namespace ctb
