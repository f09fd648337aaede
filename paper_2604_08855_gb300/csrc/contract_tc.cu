// contract_tc.cu -- the zeta contraction on the fifth-generation tensor cores.
//
// For each l the contraction  zeta~_l(b1,b2) = sum_p w_p sum_m a_lm(p,b1) a_lm(p,b2)
// is a tall-skinny symmetric rank-k update with K = (primary, m) running
// over p * (2l+1) + (m + l).  With C = sqrt|w_p| a it is
//   D_l = sum_k s_k C[b1][k] C[b2][k],   s_k = sign w_p.
// The pack kernel writes, per l, H = the BF16 rounding of C and L2 =
// 2 (C - H) in BF16 (exact: C - H fits BF16, doubling is exact), and S = s H
// when some weight is negative (else S is H itself).  The MMAs form
//   Z = S H^T + S L2^T = sum s (H H^T + 2 H L^T),
// and the FP64 finalisation symmetrises: (Z + Z^T) / 2 = sum s (H H^T + H L^T
// + L H^T) = D up to the dropped L L^T term (relative error ~2^-16, as a
// three-product hi/lo split).  TF32: Z = S T^T with T = tf32(C).
// Operands are K-major in tiles of one 128-byte row per bin (64 BF16 or 32
// TF32 elements), tile-major in HBM, so one TMA box (a 3-D box: 128 bytes x
// npad bins x one tile) reads a contiguous block; npad = nbins padded to a
// multiple of 16, rows past nbins zero-filled by TMA.  The tiles of a
// pipeline stage are contiguous in shared memory, [S] H [L2], and one MMA of
// M = 64, N = 2 npad (H and L2 side by side; TF32: N = npad) covers a
// 16-element K step: its A view starts at the stage's first tile and runs 64
// rows on into the next tiles (or the ring's slack), so rows past npad of D
// are products of other rows and are ignored.  The K steps of a tile
// alternate between two accumulators (one when TMEM is short: 64 bins).
// Two CTAs share an SM.  FP32 accumulation happens in TMEM;
// every kTcFlushTiles K tiles the accumulators are drained to FP64 registers
// (double buffered in TMEM so the MMA issue never waits for the drain), and
// the FP64 totals go to a per-CTA partial that a fixed-order FP64 reduction
// sums.
//
// Persistent over l: one wave of CTAs splits the concatenation of every
// l's K tiles into equal contiguous ranges, so each CTA allocates TMEM and
// sets up its pipeline once per launch and crosses l boundaries in its range
// (each boundary ends an accumulator flush and the partial row of that l).
//
// Roles per CTA (192 threads): warps 0-3 drain TMEM (warp w reads TMEM lanes
// 32w..32w+31 = rows of D), warp 4 issues the TMA loads, warp 5 issues the
// MMAs from one elected thread.  Every mbarrier wait is bounded: on timeout
// the CTA records an error, stops issuing, waits (bounded) for its own
// outstanding copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctb_internal.cuh"

namespace ctb {

constexpr int kTcThreads = 192;
constexpr int kTcFlushTiles = 64;
// CTAs resident per SM, each with its own TMA pipeline (shared memory and
// TMEM split between them): one CTA's ring of 16 stages kept the loads
// latency-bound at about 2.5 TB/s; two per SM doubled the throughput
constexpr int kTcCtasPerSm = 2;
constexpr long long kTcTimeoutCycles = 4000000000ll;  // about 2 s

struct TcMaps {
  CUtensorMap m[kLmaxCap + 1][3];  // per l: A (S, or H), B = H, B_lo = L2  (TF32: S or T, T, -)
};

struct TcArgs {
  int nl;
  int nbins;
  int npad;
  int nsplit;
  int stages;
  int ncols;                          // TMEM columns allocated
  int ncol_d;                         // columns of one accumulator (the MMA's N)
  int nchain;                         // accumulator chains the K steps of a tile take in turn (1 or 2)
  unsigned int cum[kLmaxCap + 2];     // 128-byte K tiles of the l before l (cum[nl] = all)
  double* partial;                    // [nl][nsplit][nbins][nbins]
  unsigned int* err;                  // bit 0: a bounded wait timed out
  long long timeout_cycles;           // limit of every mbarrier wait
  int inject_stall;                   // test hook: the MMA thread first waits on a barrier nothing signals
  int signed_a;                       // 1: the A operand is its own tensor S (some weight is negative)
};

struct TcArgsMaps {
  TcMaps maps;
  TcArgs args;
};

// ---------------------------------------------------------------------------
// PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of `bar` with parity `parity`; false if this CTA has
// given up (timeout here or elsewhere in the CTA).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, unsigned int* err,
                                          long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      atomicOr(err, 1u);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

template <bool TF32>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  if constexpr (TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3);
  v[4] = __uint_as_float(r4);
  v[5] = __uint_as_float(r5);
  v[6] = __uint_as_float(r6);
  v[7] = __uint_as_float(r7);
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
//   bits  0-13  start address >> 4        bits 16-29  leading byte offset >> 4 (unused here)
//   bits 32-45  stride byte offset >> 4   bits 46-47  descriptor version (1)
//   bits 61-63  layout: 2 = 128-byte swizzle
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: D f32, A/B K-major, M = 64, N = n.
//   bits 4-5 D format (1 = f32); 7-9 A format, 10-12 B format (kind::f16: 1 = bf16;
//   kind::tf32: 2 = tf32); 15/16 A/B major (0 = K); 17-22 N >> 3; 24-28 M >> 4.
constexpr int kTcM = 64;
__host__ __device__ constexpr uint32_t make_idesc(bool tf32, int n) {
  return (1u << 4) | ((tf32 ? 2u : 1u) << 7) | ((tf32 ? 2u : 1u) << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kTcM >> 4) << 24);
}

// ---------------------------------------------------------------------------
// contraction kernel: gridDim.x CTAs, each a contiguous range of the
// concatenated (l, K tile) sequence; partial row blockIdx.x of each l

template <bool TF32, int NCH>
__global__ void __launch_bounds__(kTcThreads, kTcCtasPerSm) k_contract_tc(const __grid_constant__ TcArgsMaps am) {
  const TcMaps& maps = am.maps;
  const TcArgs& a = am.args;
  extern __shared__ uint8_t s_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(s_raw) + 1023) & ~(uintptr_t)1023);
  const int split = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t total = a.cum[a.nl];
  const uint32_t per = (total + gridDim.x - 1) / gridDim.x;
  const uint32_t t0 = (uint32_t)split * per;
  const uint32_t t1 = min(total, t0 + per);
  if (t0 >= t1) return;  // uniform for the whole CTA
  const int S = a.stages;
  constexpr int NB = TF32 ? 1 : 2;  // B operands: H (and L2)
  const uint32_t T_BYTES = (uint32_t)a.npad * 128u;  // one operand tile
  const uint32_t A_BYTES = a.signed_a ? T_BYTES : 0u;  // S, else A is the H tile
  const uint32_t STAGE = A_BYTES + NB * T_BYTES;
  // after the stages: the A view's overrun (64 rows), then the barriers
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)S * STAGE + (size_t)kTcM * 128u);
  uint64_t* empty = full + S;
  uint64_t* accfull = empty + S;
  uint64_t* accempty = accfull + 2;
  uint64_t* done = accempty + 2;
  uint64_t* never = done + 1;  // no thread ever arrives here (fault-injection hook)
  uint32_t* s_taddr = reinterpret_cast<uint32_t*>(never + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(s_taddr + 1);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accfull + b, 1);
      mbar_init(accempty + b, 128);
    }
    mbar_init(done, 1);
    mbar_init(never, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_taddr)),
                 "r"(a.ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *s_taddr;
  // the l segments of [t0, t1): [max(t0, cum[l]), min(t1, cum[l+1]))
  int lfirst = 0;
  while (a.cum[lfirst + 1] <= t0) ++lfirst;

  if (warp == 4) {
    // ---- TMA producer
    if (lane == 0) {
      uint32_t issued = 0, it = 0;
      bool ok = true;
      for (int l = lfirst; ok && l < a.nl && a.cum[l] < t1; ++l) {
        const uint32_t sb = max(t0, a.cum[l]), se = min(t1, a.cum[l + 1]);
        for (uint32_t t = sb; t < se; ++t, ++it) {
          const int s = (int)(it % S);
          const uint32_t ph = (it / S) & 1u;
          if (!mbar_wait(empty + s, ph ^ 1u, s_abort, a.err, a.timeout_cycles)) {
            ok = false;
            break;
          }
          uint8_t* st = sm + (size_t)s * STAGE;
          mbar_expect_tx(full + s, STAGE);
          const int z = (int)(t - a.cum[l]);  // K tile: one contiguous block of nbins rows
          if (a.signed_a) tma_load_3d(st, &maps.m[l][0], 0, 0, z, full + s);
          tma_load_3d(st + A_BYTES, &maps.m[l][1], 0, 0, z, full + s);
          if (!TF32) tma_load_3d(st + A_BYTES + T_BYTES, &maps.m[l][2], 0, 0, z, full + s);
          ++issued;
        }
      }
      // bounded wait for this CTA's copies still in flight (the consumer may
      // give up later than this loop ends); on the normal path these phases
      // have completed and each test passes at once
      const uint32_t first = issued > (uint32_t)S ? issued - S : 0;
      for (uint32_t k = first; k < issued; ++k) {
        const long long tw = clock64();
        while (!mbar_try_wait(full + (k % S), (k / S) & 1u) && clock64() - tw < a.timeout_cycles) {
        }
      }
    }
  } else if (warp == 5) {
    // ---- MMA issuer
    if (lane == 0) {
      // N = the B view: H and L2 side by side (BF16), or T (TF32)
      const uint32_t idesc = make_idesc(TF32, a.ncol_d);
      // fault injection: a wait that runs out, then the ordinary abort path
      bool go = !a.inject_stall || mbar_wait(never, 0, s_abort, a.err, a.timeout_cycles);
      uint32_t it = 0, f = 0;  // f: accumulator flushes so far (buffer f & 1)
      for (int l = lfirst; go && l < a.nl && a.cum[l] < t1; ++l) {
        const uint32_t sb = max(t0, a.cum[l]), se = min(t1, a.cum[l + 1]);
        for (uint32_t t = sb; go && t < se; ++t, ++it) {
          const int s = (int)(it % S);
          const uint32_t ph = (it / S) & 1u;
          const uint32_t buf = f & 1u;
          const bool first_of_flush = ((t - sb) % kTcFlushTiles) == 0;
          const bool last_of_flush = ((t - sb) % kTcFlushTiles) == kTcFlushTiles - 1 || t + 1 == se;
          if (first_of_flush && f >= 2 &&
              !mbar_wait(accempty + buf, ((f >> 1) - 1) & 1u, s_abort, a.err, a.timeout_cycles)) {
            go = false;
            break;
          }
          if (!mbar_wait(full + s, ph, s_abort, a.err, a.timeout_cycles)) {
            go = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(sm + (size_t)s * STAGE);
          const uint32_t b_hi = sa + A_BYTES;
          // NCH accumulator chains (the 16-element K steps in turn)
          constexpr uint32_t nch = NCH;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t acc0 = (first_of_flush && (uint32_t)kk < nch) ? 0u : 1u;
            const uint32_t ko = (uint32_t)kk * 32u;  // 32 bytes of K per MMA
            const uint32_t d = taddr + (buf * nch + (uint32_t)kk % nch) * (uint32_t)a.ncol_d;
            tc_mma<TF32>(d, sw128_desc(sa + ko), sw128_desc(b_hi + ko), idesc, acc0);
          }
          tc_commit(empty + s);
          if (last_of_flush) {
            tc_commit(accfull + buf);
            ++f;
          }
        }
      }
      // all MMAs issued by this thread complete before TMEM is released
      tc_commit(done);
      const long long tw = clock64();
      while (!mbar_try_wait(done, 0) && clock64() - tw < a.timeout_cycles) {
      }
    }
  } else {
    // ---- drain TMEM to FP64 (warps 0-3).  With M = 64 row i of D lives in
    // TMEM lane 32 (i / 16) + i % 16: warp w reads lanes 32w.. and its lanes
    // 0-15 hold rows 16w..16w+15.  One FP64 row sum per l segment, added to
    // partial row `split` of that l.
    const uint32_t row_addr = taddr + ((uint32_t)(warp * 32) << 16);
    const int r = lane < 16 ? warp * 16 + lane : 1 << 20;
    uint32_t f = 0;
    bool ok = true;
    for (int l = lfirst; ok && l < a.nl && a.cum[l] < t1; ++l) {
      const uint32_t sb = max(t0, a.cum[l]), se = min(t1, a.cum[l + 1]);
      const uint32_t nflush = (se - sb + kTcFlushTiles - 1) / kTcFlushTiles;
      double acc[64];
#pragma unroll
      for (int c = 0; c < 64; ++c) acc[c] = 0.0;
      for (uint32_t k = 0; k < nflush; ++k, ++f) {
        const uint32_t buf = f & 1u;
        if (!mbar_wait(accfull + buf, (f >> 1) & 1u, s_abort, a.err, a.timeout_cycles)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          if (c * 8 < a.npad) {
            // Z[r][col] = the chains' S H^T plus their S L2^T (BF16)
            const uint32_t col = buf * (uint32_t)NCH * (uint32_t)a.ncol_d + (uint32_t)(c * 8);
            float v[8], u[8];
            tmem_ld8(row_addr + col, v);
            if constexpr (NCH > 1) {
              tmem_ld8(row_addr + col + (uint32_t)a.ncol_d, u);
#pragma unroll
              for (int q = 0; q < 8; ++q) v[q] += u[q];
            }
            if (!TF32) {
              tmem_ld8(row_addr + col + (uint32_t)a.npad, u);
#pragma unroll
              for (int q = 0; q < 8; ++q) v[q] += u[q];
              if constexpr (NCH > 1) {
                tmem_ld8(row_addr + col + (uint32_t)a.ncol_d + (uint32_t)a.npad, u);
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] += u[q];
              }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[c * 8 + q] += (double)v[q];
          }
        }
        tc_fence_before();
        mbar_arrive(accempty + buf);
      }
      if (ok && r < a.nbins && !*s_abort) {
        double* out = a.partial + (((size_t)l * a.nsplit + split) * a.nbins + r) * a.nbins;
#pragma unroll
        for (int c = 0; c < 64; ++c)
          if (c < a.nbins) out[c] += acc[c];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(a.ncols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// pack: coefficient rows -> K-major operands per l

// A block takes kPackPrims consecutive primaries.  For each bin, one thread
// copies their rows (contiguous, row * 4 bytes each) into shared memory with
// TMA bulk copies completing on an mbarrier, two bins ahead in a two-stage
// ring, so the copies of the next bin overlap the conversion of this one.
// For each l the block's operands of one bin are a contiguous span of
// kPackPrims * (2l+1) elements starting at a multiple of 16 elements; span l
// starts at 16 l^2 of the bin's concatenated spans.  Each thread converts
// chunks of 8 consecutive elements (chunk k lies in span l = floor(sqrt(k/2)))
// and writes them with 16-byte stores: C = sqrt|w_p| a as H (BF16) and
// L2 = 2 (C - H) (BF16), or as TF32; and S = sign(w_p) H when outS is set.
// A partial last block converts element by element; block 0 also writes the
// zeros of the K padding.
constexpr int kPackPrims = 16;
constexpr int kPackThreads = 256;

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_elem, float hi_elem) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);  // .x = lo_elem (lower address)
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float flip(float v, bool neg) { return neg ? -v : v; }

// Operand layout of one l: K tiles of KT elements (one 128-byte row each),
// tile-major: element k of bin b at ((k / KT) nbins + b) KT + k % KT, so a
// K tile of every bin is one contiguous block that one TMA box reads.
template <bool TF32>
__device__ __forceinline__ unsigned long long op_index(unsigned long long lbase, int nbins, int b, unsigned long long k) {
  constexpr unsigned long long KT = TF32 ? 32 : 64;
  return lbase + ((k / KT) * (unsigned long long)nbins + (unsigned long long)b) * KT + k % KT;
}

// 8 consecutive elements c[i] (already scaled by sqrt|w|) with signs neg[i]
template <bool TF32>
__device__ __forceinline__ void pack_store(void* outS, void* outH, void* outL, unsigned long long idx, const float* c,
                                           const bool* neg) {
  if constexpr (TF32) {
    uint32_t t[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t[i]) : "f"(c[i]));
    uint4* H = reinterpret_cast<uint4*>(reinterpret_cast<uint32_t*>(outH) + idx);
    H[0] = make_uint4(t[0], t[1], t[2], t[3]);
    H[1] = make_uint4(t[4], t[5], t[6], t[7]);
    if (outS) {
      uint32_t u[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) u[i] = t[i] ^ (neg[i] ? 0x80000000u : 0u);
      uint4* Sp = reinterpret_cast<uint4*>(reinterpret_cast<uint32_t*>(outS) + idx);
      Sp[0] = make_uint4(u[0], u[1], u[2], u[3]);
      Sp[1] = make_uint4(u[4], u[5], u[6], u[7]);
    }
  } else {
    float h[8], l2[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      h[i] = __bfloat162float(__float2bfloat16_rn(c[i]));
      l2[i] = 2.f * (c[i] - h[i]);
    }
    const unsigned long long o = idx / 8;  // 8 BF16 = 16 bytes
    reinterpret_cast<uint4*>(outH)[o] = make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]),
                                                   pack_bf16x2(h[4], h[5]), pack_bf16x2(h[6], h[7]));
    reinterpret_cast<uint4*>(outL)[o] = make_uint4(pack_bf16x2(l2[0], l2[1]), pack_bf16x2(l2[2], l2[3]),
                                                   pack_bf16x2(l2[4], l2[5]), pack_bf16x2(l2[6], l2[7]));
    if (outS)
      reinterpret_cast<uint4*>(outS)[o] = make_uint4(
          pack_bf16x2(flip(h[0], neg[0]), flip(h[1], neg[1])), pack_bf16x2(flip(h[2], neg[2]), flip(h[3], neg[3])),
          pack_bf16x2(flip(h[4], neg[4]), flip(h[5], neg[5])), pack_bf16x2(flip(h[6], neg[6]), flip(h[7], neg[7])));
  }
}

template <bool TF32>
__device__ __forceinline__ void pack_store1(void* outS, void* outH, void* outL, unsigned long long idx, float c,
                                            bool neg) {
  if constexpr (TF32) {
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(c));
    reinterpret_cast<uint32_t*>(outH)[idx] = t;
    if (outS) reinterpret_cast<uint32_t*>(outS)[idx] = t ^ (neg ? 0x80000000u : 0u);
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn(c);
    const float hf = __bfloat162float(h);
    reinterpret_cast<__nv_bfloat16*>(outH)[idx] = h;
    reinterpret_cast<__nv_bfloat16*>(outL)[idx] = __float2bfloat16_rn(2.f * (c - hf));
    if (outS) reinterpret_cast<__nv_bfloat16*>(outS)[idx] = __float2bfloat16_rn(flip(hf, neg));
  }
}

template <bool TF32>
__global__ void __launch_bounds__(kPackThreads) k_pack(const float* __restrict__ M, const float* __restrict__ wprim,
                                                       int64_t np, int nbins, int row, int lmax,
                                                       const int* __restrict__ slot,
                                                       const unsigned long long* __restrict__ lbase,
                                                       const unsigned long long* __restrict__ kp,
                                                       void* __restrict__ outS, void* __restrict__ outH,
                                                       void* __restrict__ outL, unsigned int* err,
                                                       long long timeout_cycles) {
  extern __shared__ __align__(16) float s_pack[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ int s_abort;
  __shared__ unsigned long long s_lbase[kLmaxCap + 1], s_kp[kLmaxCap + 1];
  float* stage0 = s_pack;                                  // [kPackPrims][row], two stages
  float* s_w = stage0 + 2 * kPackPrims * row;              // [kPackPrims] sqrt|w|, sign bit = sign w
  int* s_slot = reinterpret_cast<int*>(s_w + kPackPrims);  // [(lmax+1)^2]
  const int nc = (lmax + 1) * (lmax + 1);
  const int64_t p0 = (int64_t)blockIdx.x * kPackPrims;
  const int pt = (int)min((int64_t)kPackPrims, np - p0);
  const uint32_t rowbytes = (uint32_t)row * 4u;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) s_slot[c] = slot[c];
  for (int q = threadIdx.x; q < pt; q += blockDim.x) {
    const float wq = __ldg(wprim + p0 + q);
    s_w[q] = copysignf(sqrtf(fabsf(wq)), wq);
  }
  for (int l = threadIdx.x; l <= lmax; l += blockDim.x) {
    s_lbase[l] = lbase[l];
    s_kp[l] = kp[l];
  }
  if (threadIdx.x == 0) {
    s_abort = 0;
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // stage s holds bin b (s = b & 1); its copies complete phase (b >> 1) of s_bar[s]
  auto issue = [&](int b) {
    float* dst = stage0 + (b & 1) * kPackPrims * row;
    uint64_t* bar = &s_bar[b & 1];
    mbar_expect_tx(bar, rowbytes * (uint32_t)pt);
    for (int q = 0; q < pt; ++q) bulk_g2s(dst + q * row, M + ((p0 + q) * nbins + b) * (int64_t)row, rowbytes, bar);
  };
  if (threadIdx.x == 0) {
    issue(0);
    if (nbins > 1) issue(1);
  }
  if (blockIdx.x == 0) {
    // zeros in the K padding of every (l, bin): elements [np (2l+1), kp[l]) of its region
    for (int l = 0; l <= lmax; ++l) {
      const unsigned long long used = (unsigned long long)np * (2 * l + 1);
      const int tail = (int)(s_kp[l] - used);
      for (int e = threadIdx.x; e < nbins * tail; e += blockDim.x) {
        const int bb = e / tail, t = e - bb * tail;
        pack_store1<TF32>(outS, outH, outL, op_index<TF32>(s_lbase[l], nbins, bb, used + (unsigned long long)t), 0.f,
                          false);
      }
    }
  }
  int b = 0;
  for (; b < nbins; ++b) {
    mbar_wait(&s_bar[b & 1], (uint32_t)(b >> 1) & 1u, &s_abort, err, timeout_cycles);
    __syncthreads();
    if (s_abort) break;
    const float* rows = stage0 + (b & 1) * kPackPrims * row;
    if (pt == kPackPrims) {
      const int nchunks = 2 * nc;  // 16 (l+1)^2 elements per bin, 8 per chunk
      for (int k = threadIdx.x; k < nchunks; k += blockDim.x) {
        const int t = k >> 1;
        int l = (int)sqrtf((float)t);
        while ((l + 1) * (l + 1) <= t) ++l;
        while (l * l > t) --l;
        const int nl = 2 * l + 1;
        const int e0 = 8 * k - 16 * l * l;  // first element of the chunk in span l
        int q = e0 / nl;
        int mi = e0 - q * nl;
        float cv[8];
        bool ng[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float sw = s_w[q];
          cv[i] = fabsf(sw) * rows[q * row + s_slot[l * l + mi]];
          ng[i] = signbit(sw);
          if (++mi == nl) {
            mi = 0;
            ++q;
          }
        }
        const unsigned long long idx =
            op_index<TF32>(s_lbase[l], nbins, b, (unsigned long long)p0 * nl + (unsigned long long)e0);
        pack_store<TF32>(outS, outH, outL, idx, cv, ng);
      }
    } else {
      for (int l = 0; l <= lmax; ++l) {
        const int nl = 2 * l + 1;
        const unsigned long long k0 = (unsigned long long)p0 * nl;
        for (int e = threadIdx.x; e < pt * nl; e += blockDim.x) {
          const int q = e / nl, mi = e - q * nl;
          const float sw = s_w[q];
          pack_store1<TF32>(outS, outH, outL, op_index<TF32>(s_lbase[l], nbins, b, k0 + (unsigned long long)e),
                            fabsf(sw) * rows[q * row + s_slot[l * l + mi]], signbit(sw));
        }
      }
    }
    __syncthreads();  // stage (b & 1) is consumed
    if (threadIdx.x == 0 && b + 2 < nbins) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(b + 2);
    }
  }
  if (s_abort && threadIdx.x == 0) {
    // bounded wait for this block's own copies still in flight: bins b .. min(b + 1, nbins - 1)
    int dummy = 0;
    for (int c = b; c < nbins && c < b + 2; ++c)
      mbar_wait(&s_bar[c & 1], (uint32_t)(c >> 1) & 1u, &dummy, err, timeout_cycles);
  }
}

// zeta_l(b1,b2) = 4 pi/(2l+1) * sum_split (D(b1,b2) + D(b2,b1)) / 2, in split order
__global__ void k_finalize_tc(const double* __restrict__ partial, int nl, int nsplit, int nb,
                              double* __restrict__ zeta) {
  const int total = nl * nb * nb;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < total; o += gridDim.x * blockDim.x) {
    const int l = o / (nb * nb), r = o % (nb * nb);
    const int b1 = r / nb, b2 = r % nb;
    double s = 0.0;
    for (int c = 0; c < nsplit; ++c) {
      const double* blk = partial + ((size_t)l * nsplit + c) * nb * nb;
      s += 0.5 * (blk[b1 * nb + b2] + blk[b2 * nb + b1]);
    }
    zeta[o] = s * (4.0 * 3.14159265358979323846 / (2.0 * l + 1.0));
  }
}

// ---------------------------------------------------------------------------
// host side

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

int tc_npad(int nbins) { return std::max(16, (nbins + 15) / 16 * 16); }

size_t tc_stage_bytes(bool tf32, bool signed_a, int nbins) {
  return ((signed_a ? 1 : 0) + (tf32 ? 1 : 2)) * (size_t)tc_npad(nbins) * 128;
}

void tc_layout(bool tf32, int64_t np, int nbins, int lmax, std::vector<unsigned long long>& lbase,
               std::vector<unsigned long long>& kp, size_t* elems) {
  const unsigned long long kt = tf32 ? 32 : 64;  // elements per 128-byte K tile
  lbase.assign(lmax + 1, 0);
  kp.assign(lmax + 1, 0);
  unsigned long long acc = 0;
  for (int l = 0; l <= lmax; ++l) {
    kp[l] = ((unsigned long long)np * (2 * l + 1) + kt - 1) / kt * kt;
    lbase[l] = acc;
    acc += (unsigned long long)nbins * kp[l];
  }
  *elems = (size_t)acc;
}

cudaError_t launch_pack(bool tf32, const float* M, const float* wprim, int64_t np, int nbins, int row, int lmax,
                        const int* slot, const unsigned long long* lbase, const unsigned long long* kp, void* outS,
                        void* outH, void* outL, unsigned int* err, cudaStream_t st) {
  if (np == 0) return cudaSuccess;
  const int64_t blocks = (np + kPackPrims - 1) / kPackPrims;
  const size_t smem = ((size_t)2 * kPackPrims * row + kPackPrims + (size_t)(lmax + 1) * (lmax + 1)) * 4;
  cudaError_t e;
  if (tf32) {
    e = cudaFuncSetAttribute(k_pack<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_pack<true><<<(unsigned)blocks, kPackThreads, smem, st>>>(M, wprim, np, nbins, row, lmax, slot, lbase, kp, outS,
                                                               outH, outL, err, kTcTimeoutCycles);
  } else {
    e = cudaFuncSetAttribute(k_pack<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_pack<false><<<(unsigned)blocks, kPackThreads, smem, st>>>(M, wprim, np, nbins, row, lmax, slot, lbase, kp, outS,
                                                                outH, outL, err, kTcTimeoutCycles);
  }
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_contract_tc(bool tf32, int64_t np, int nbins, int lmax, const unsigned long long* h_lbase,
                               const unsigned long long* h_kp, void* opA, void* opH, void* opL, double* partial,
                               int nsplit, unsigned int* err, bool inject_stall, cudaStream_t st) {
  if (np == 0) return cudaSuccess;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const int npad = tc_npad(nbins);
  const size_t esz = tf32 ? 4 : 2;
  const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  TcArgsMaps am;
  std::memset(&am, 0, sizeof(am));
  TcMaps& maps = am.maps;
  TcArgs& a = am.args;
  a.nl = lmax + 1;
  a.nbins = nbins;
  a.npad = npad;
  a.nsplit = nsplit;
  a.partial = partial;
  a.err = err;
  // about 2 s per wait; an injected stall gives up after about 10 ms
  a.timeout_cycles = inject_stall ? 20000000ll : kTcTimeoutCycles;
  a.inject_stall = inject_stall ? 1 : 0;
  void* bases[3] = {opA, opH, opL};
  a.signed_a = opA != opH ? 1 : 0;
  a.cum[0] = 0;
  for (int l = 0; l <= lmax; ++l) {
    a.cum[l + 1] = a.cum[l] + (unsigned int)(h_kp[l] / (tf32 ? 32 : 64));
    for (int k = 0; k < 3; ++k) {
      if ((tf32 && k == 2) || (k == 0 && !a.signed_a)) continue;
      // [K tile][bin][128 bytes]: a box is one K tile of npad rows (rows past
      // nbins zero-filled)
      void* gaddr = static_cast<char*>(bases[k]) + h_lbase[l] * esz;
      const cuuint64_t kt = 128 / esz;
      cuuint64_t gdim[3] = {kt, (cuuint64_t)nbins, (cuuint64_t)(h_kp[l] / kt)};
      cuuint64_t gstride[2] = {128, (cuuint64_t)nbins * 128};
      cuuint32_t box[3] = {(cuuint32_t)kt, (cuuint32_t)npad, 1};
      cuuint32_t estr[3] = {1, 1, 1};
      CUresult r = enc(&maps.m[l][k], dt, 3, gaddr, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
  }
  const size_t stage = tc_stage_bytes(tf32, a.signed_a != 0, nbins);
  const size_t slack = (size_t)kTcM * 128;  // the A view's overrun past the last stage
  const size_t budget = (220 * 1024) / kTcCtasPerSm;
  a.stages = (int)std::max<size_t>(2, std::min<size_t>(16, (budget - 1024 - slack - 256) / stage));
  // accumulators: 2 flush buffers x nchain chains x N columns, within this
  // CTA's share of the SM's 512 TMEM columns
  a.ncol_d = tf32 ? npad : 2 * npad;
  a.nchain = 2 * 2 * a.ncol_d * kTcCtasPerSm <= 512 ? 2 : 1;
  int ncols = 32;
  while (ncols < 2 * a.nchain * a.ncol_d) ncols *= 2;
  a.ncols = ncols;
  const size_t smem = 1024 + a.stages * stage + slack + 256;
  // one wave: kTcCtasPerSm CTAs per SM, at most one per partial row
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorInvalidValue;
  const int grid = std::max(1, std::min(kTcCtasPerSm * nsm, nsplit));
  void (*fn)(const TcArgsMaps) = tf32 ? (a.nchain == 2 ? k_contract_tc<true, 2> : k_contract_tc<true, 1>)
                                     : (a.nchain == 2 ? k_contract_tc<false, 2> : k_contract_tc<false, 1>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, kTcThreads, smem, st>>>(am);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_finalize_tc(const double* partial, int lmax, int nsplit, int nbins, double* zeta, cudaStream_t st) {
  const int total = (lmax + 1) * nbins * nbins;
  k_finalize_tc<<<(total + 255) / 256, 256, 0, st>>>(partial, lmax + 1, nsplit, nbins, zeta);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ctb
