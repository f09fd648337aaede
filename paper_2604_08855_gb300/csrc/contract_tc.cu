// contract_tc.cu -- the zeta contraction on the fifth-generation tensor cores.
//
// For each l the contraction  zeta~_l(b1,b2) = sum_p w_p sum_m a_lm(p,b1) a_lm(p,b2)
// is a tall-skinny product  D_l = A_l B_l^T  with K = (primary, m) running over
// p * (2l+1) + (m + l):
//   A_l[b][k] = w_p a_lm(p,b)      (rows = bins, zero-padded to M = 128)
//   B_l[b][k] =     a_lm(p,b)      (rows = bins, zero-padded to N = npad)
// Both operands are K-major; the pack kernel writes them from the coefficient
// rows either as a BF16 hi/lo split (a = hi + lo; D = Ah Bh + Ah Bl + Al Bh,
// three kind::f16 products, relative error ~2^-16) or rounded to TF32 (one
// kind::tf32 product).  FP32 accumulation happens in TMEM; every
// kTcFlushTiles K tiles the accumulator is drained to FP64 registers (double
// buffered in TMEM so the MMA issue never waits for the drain), and the FP64
// totals go to a per-CTA partial that a fixed-order FP64 reduction sums.
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
constexpr int kTcFlushTiles = 16;
constexpr long long kTcTimeoutCycles = 4000000000ll;  // about 2 s

struct TcMaps {
  CUtensorMap m[kLmaxCap + 1][4];  // per l: A_hi, A_lo, B_hi, B_lo  (TF32: A, -, B, -)
};

struct TcArgs {
  int nl;
  int nbins;
  int npad;
  int nsplit;
  int stages;
  int ncols;                          // TMEM columns allocated
  unsigned int ktiles[kLmaxCap + 1];  // 128-byte K tiles per l
  double* partial;                    // [nl][nsplit][nbins][nbins]
  unsigned int* err;                  // bit 0: a bounded wait timed out
  long long timeout_cycles;           // limit of every mbarrier wait
  int inject_stall;                   // test hook: the MMA thread first waits on a barrier nothing signals
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

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
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

// Instruction descriptor: D f32, A/B K-major, M = 128, N = npad.
//   bits 4-5 D format (1 = f32); 7-9 A format, 10-12 B format (kind::f16: 1 = bf16;
//   kind::tf32: 2 = tf32); 15/16 A/B major (0 = K); 17-22 N >> 3; 24-28 M >> 4.
__host__ __device__ constexpr uint32_t make_idesc(bool tf32, int n) {
  return (1u << 4) | ((tf32 ? 2u : 1u) << 7) | ((tf32 ? 2u : 1u) << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

// ---------------------------------------------------------------------------
// contraction kernel: grid (nsplit, nl), one K range of one l per CTA

template <bool TF32>
__global__ void __launch_bounds__(kTcThreads, 1) k_contract_tc(const __grid_constant__ TcMaps maps, TcArgs a) {
  extern __shared__ uint8_t s_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(s_raw) + 1023) & ~(uintptr_t)1023);
  const int l = blockIdx.y;
  const int split = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t total = a.ktiles[l];
  const uint32_t per = (total + a.nsplit - 1) / a.nsplit;
  const uint32_t t0 = (uint32_t)split * per;
  const uint32_t t1 = min(total, t0 + per);
  if (t0 >= t1) return;  // uniform for the whole CTA
  const uint32_t ntiles = t1 - t0;
  const int S = a.stages;
  constexpr int NA = TF32 ? 1 : 2;
  const uint32_t A_BYTES = 128u * 128u;
  const uint32_t B_BYTES = (uint32_t)a.npad * 128u;
  const uint32_t STAGE = NA * (A_BYTES + B_BYTES);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)S * STAGE);
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
  const uint32_t nflush = (ntiles + kTcFlushTiles - 1) / kTcFlushTiles;

  if (warp == 4) {
    // ---- TMA producer
    if (lane == 0) {
      uint32_t issued = 0;
      for (uint32_t it = 0; it < ntiles; ++it) {
        const int s = (int)(it % S);
        const uint32_t ph = (it / S) & 1u;
        if (!mbar_wait(empty + s, ph ^ 1u, s_abort, a.err, a.timeout_cycles)) break;
        uint8_t* st = sm + (size_t)s * STAGE;
        mbar_expect_tx(full + s, STAGE);
        const int x = (int)((t0 + it) * (TF32 ? 32u : 64u));
        tma_load_2d(st, &maps.m[l][0], x, 0, full + s);
        if (!TF32) tma_load_2d(st + A_BYTES, &maps.m[l][1], x, 0, full + s);
        tma_load_2d(st + NA * A_BYTES, &maps.m[l][2], x, 0, full + s);
        if (!TF32) tma_load_2d(st + NA * A_BYTES + B_BYTES, &maps.m[l][3], x, 0, full + s);
        ++issued;
      }
      // bounded wait for this CTA's copies still in flight (the consumer may
      // give up later than this loop ends); on the normal path these phases
      // have completed and each test passes at once
      const uint32_t first = issued > (uint32_t)S ? issued - S : 0;
      for (uint32_t it = first; it < issued; ++it) {
        const long long tw = clock64();
        while (!mbar_try_wait(full + (it % S), (it / S) & 1u) && clock64() - tw < a.timeout_cycles) {
        }
      }
    }
  } else if (warp == 5) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = make_idesc(TF32, a.npad);
      // fault injection: a wait that runs out, then the ordinary abort path
      const bool go = !a.inject_stall || mbar_wait(never, 0, s_abort, a.err, a.timeout_cycles);
      for (uint32_t it = 0; go && it < ntiles; ++it) {
        const int s = (int)(it % S);
        const uint32_t ph = (it / S) & 1u;
        const uint32_t f = it / kTcFlushTiles;
        const uint32_t buf = f & 1u;
        const bool first_of_flush = (it % kTcFlushTiles) == 0;
        if (first_of_flush && f >= 2 && !mbar_wait(accempty + buf, ((f >> 1) - 1) & 1u, s_abort, a.err, a.timeout_cycles)) break;
        if (!mbar_wait(full + s, ph, s_abort, a.err, a.timeout_cycles)) break;
        tc_fence_after();
        const uint32_t sa = smem_u32(sm + (size_t)s * STAGE);
        const uint32_t a_hi = sa, a_lo = sa + A_BYTES;
        const uint32_t b_hi = sa + NA * A_BYTES, b_lo = b_hi + B_BYTES;
        const uint32_t d = taddr + buf * (uint32_t)a.npad;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t acc0 = (first_of_flush && kk == 0) ? 0u : 1u;
          const uint32_t ko = (uint32_t)kk * 32u;  // 32 bytes of K per MMA
          tc_mma<TF32>(d, sw128_desc(a_hi + ko), sw128_desc(b_hi + ko), idesc, acc0);
          if (!TF32) {
            tc_mma<TF32>(d, sw128_desc(a_hi + ko), sw128_desc(b_lo + ko), idesc, 1u);
            tc_mma<TF32>(d, sw128_desc(a_lo + ko), sw128_desc(b_hi + ko), idesc, 1u);
          }
        }
        tc_commit(empty + s);
        if ((it % kTcFlushTiles) == kTcFlushTiles - 1 || it + 1 == ntiles) tc_commit(accfull + buf);
      }
      // all MMAs issued by this thread complete before TMEM is released
      tc_commit(done);
      const long long tw = clock64();
      while (!mbar_try_wait(done, 0) && clock64() - tw < a.timeout_cycles) {
      }
    }
  } else {
    // ---- drain TMEM to FP64 (warps 0-3; warp w owns rows 32w..32w+31)
    double acc[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) acc[c] = 0.0;
    const uint32_t row_addr = taddr + ((uint32_t)(warp * 32) << 16);
    for (uint32_t f = 0; f < nflush; ++f) {
      const uint32_t buf = f & 1u;
      if (!mbar_wait(accfull + buf, (f >> 1) & 1u, s_abort, a.err, a.timeout_cycles)) break;
      tc_fence_after();
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (c * 8 < a.npad) {
          float v[8];
          tmem_ld8(row_addr + buf * (uint32_t)a.npad + (uint32_t)(c * 8), v);
#pragma unroll
          for (int q = 0; q < 8; ++q) acc[c * 8 + q] += (double)v[q];
        }
      }
      tc_fence_before();
      mbar_arrive(accempty + buf);
    }
    const int r = warp * 32 + lane;
    if (r < a.nbins && !*s_abort) {
      double* out = a.partial + (((size_t)l * a.nsplit + split) * a.nbins + r) * a.nbins;
#pragma unroll
      for (int c = 0; c < 64; ++c)
        if (c < a.nbins) out[c] += acc[c];
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
// and writes them with 16-byte stores.  A = w_p a and B = a, each as a BF16
// hi + lo pair (or rounded to TF32).  A partial last block converts element
// by element; block 0 also writes the zeros of the K padding.
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

template <bool TF32>
__device__ __forceinline__ void pack_store(void* outA_hi, void* outA_lo, void* outB_hi, void* outB_lo,
                                           unsigned long long idx, const float* av, const float* v) {
  if constexpr (TF32) {
    uint32_t ta[8], tb[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(ta[i]) : "f"(av[i]));
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(tb[i]) : "f"(v[i]));
    }
    uint4* A = reinterpret_cast<uint4*>(reinterpret_cast<uint32_t*>(outA_hi) + idx);
    uint4* B = reinterpret_cast<uint4*>(reinterpret_cast<uint32_t*>(outB_hi) + idx);
    A[0] = make_uint4(ta[0], ta[1], ta[2], ta[3]);
    A[1] = make_uint4(ta[4], ta[5], ta[6], ta[7]);
    B[0] = make_uint4(tb[0], tb[1], tb[2], tb[3]);
    B[1] = make_uint4(tb[4], tb[5], tb[6], tb[7]);
  } else {
    float ah[8], al[8], bh[8], bl[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      ah[i] = __bfloat162float(__float2bfloat16_rn(av[i]));
      al[i] = av[i] - ah[i];
      bh[i] = __bfloat162float(__float2bfloat16_rn(v[i]));
      bl[i] = v[i] - bh[i];
    }
    const unsigned long long o = idx / 8;  // 8 BF16 = 16 bytes
    reinterpret_cast<uint4*>(outA_hi)[o] = make_uint4(pack_bf16x2(ah[0], ah[1]), pack_bf16x2(ah[2], ah[3]),
                                                      pack_bf16x2(ah[4], ah[5]), pack_bf16x2(ah[6], ah[7]));
    reinterpret_cast<uint4*>(outA_lo)[o] = make_uint4(pack_bf16x2(al[0], al[1]), pack_bf16x2(al[2], al[3]),
                                                      pack_bf16x2(al[4], al[5]), pack_bf16x2(al[6], al[7]));
    reinterpret_cast<uint4*>(outB_hi)[o] = make_uint4(pack_bf16x2(bh[0], bh[1]), pack_bf16x2(bh[2], bh[3]),
                                                      pack_bf16x2(bh[4], bh[5]), pack_bf16x2(bh[6], bh[7]));
    reinterpret_cast<uint4*>(outB_lo)[o] = make_uint4(pack_bf16x2(bl[0], bl[1]), pack_bf16x2(bl[2], bl[3]),
                                                      pack_bf16x2(bl[4], bl[5]), pack_bf16x2(bl[6], bl[7]));
  }
}

template <bool TF32>
__device__ __forceinline__ void pack_store1(void* outA_hi, void* outA_lo, void* outB_hi, void* outB_lo,
                                            unsigned long long idx, float av, float v) {
  if constexpr (TF32) {
    uint32_t ta, tb;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(ta) : "f"(av));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(tb) : "f"(v));
    reinterpret_cast<uint32_t*>(outA_hi)[idx] = ta;
    reinterpret_cast<uint32_t*>(outB_hi)[idx] = tb;
  } else {
    const __nv_bfloat16 ah = __float2bfloat16_rn(av);
    const __nv_bfloat16 bh = __float2bfloat16_rn(v);
    reinterpret_cast<__nv_bfloat16*>(outA_hi)[idx] = ah;
    reinterpret_cast<__nv_bfloat16*>(outA_lo)[idx] = __float2bfloat16_rn(av - __bfloat162float(ah));
    reinterpret_cast<__nv_bfloat16*>(outB_hi)[idx] = bh;
    reinterpret_cast<__nv_bfloat16*>(outB_lo)[idx] = __float2bfloat16_rn(v - __bfloat162float(bh));
  }
}

template <bool TF32>
__global__ void __launch_bounds__(kPackThreads) k_pack(const float* __restrict__ M, const float* __restrict__ wprim,
                                                       int64_t np, int nbins, int row, int lmax,
                                                       const int* __restrict__ slot,
                                                       const unsigned long long* __restrict__ lbase,
                                                       const unsigned long long* __restrict__ kp,
                                                       void* __restrict__ outA_hi, void* __restrict__ outA_lo,
                                                       void* __restrict__ outB_hi, void* __restrict__ outB_lo,
                                                       unsigned int* err, long long timeout_cycles) {
  extern __shared__ __align__(16) float s_pack[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ int s_abort;
  __shared__ unsigned long long s_lbase[kLmaxCap + 1], s_kp[kLmaxCap + 1];
  float* stage0 = s_pack;                                  // [kPackPrims][row], two stages
  float* s_w = stage0 + 2 * kPackPrims * row;              // [kPackPrims]
  int* s_slot = reinterpret_cast<int*>(s_w + kPackPrims);  // [(lmax+1)^2]
  const int nc = (lmax + 1) * (lmax + 1);
  const int64_t p0 = (int64_t)blockIdx.x * kPackPrims;
  const int pt = (int)min((int64_t)kPackPrims, np - p0);
  const uint32_t rowbytes = (uint32_t)row * 4u;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) s_slot[c] = slot[c];
  for (int q = threadIdx.x; q < pt; q += blockDim.x) s_w[q] = __ldg(wprim + p0 + q);
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
        pack_store1<TF32>(outA_hi, outA_lo, outB_hi, outB_lo,
                          s_lbase[l] + (unsigned long long)bb * s_kp[l] + used + (unsigned long long)t, 0.f, 0.f);
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
        float v[8], av[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          v[i] = rows[q * row + s_slot[l * l + mi]];
          av[i] = s_w[q] * v[i];
          if (++mi == nl) {
            mi = 0;
            ++q;
          }
        }
        const unsigned long long idx = s_lbase[l] + (unsigned long long)b * s_kp[l] +
                                       (unsigned long long)p0 * nl + (unsigned long long)e0;
        pack_store<TF32>(outA_hi, outA_lo, outB_hi, outB_lo, idx, av, v);
      }
    } else {
      for (int l = 0; l <= lmax; ++l) {
        const int nl = 2 * l + 1;
        const unsigned long long base = s_lbase[l] + (unsigned long long)b * s_kp[l] + (unsigned long long)p0 * nl;
        for (int e = threadIdx.x; e < pt * nl; e += blockDim.x) {
          const int q = e / nl, mi = e - q * nl;
          const float v = rows[q * row + s_slot[l * l + mi]];
          pack_store1<TF32>(outA_hi, outA_lo, outB_hi, outB_lo, base + (unsigned long long)e, s_w[q] * v, v);
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

size_t tc_stage_bytes(bool tf32, int nbins) {
  const size_t nA = tf32 ? 1 : 2;
  return nA * (128 * 128 + (size_t)tc_npad(nbins) * 128);
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
                        const int* slot, const unsigned long long* lbase, const unsigned long long* kp, void* ahi,
                        void* alo, void* bhi, void* blo, unsigned int* err, cudaStream_t st) {
  if (np == 0) return cudaSuccess;
  const int64_t blocks = (np + kPackPrims - 1) / kPackPrims;
  const size_t smem = ((size_t)2 * kPackPrims * row + kPackPrims + (size_t)(lmax + 1) * (lmax + 1)) * 4;
  cudaError_t e;
  if (tf32) {
    e = cudaFuncSetAttribute(k_pack<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_pack<true><<<(unsigned)blocks, kPackThreads, smem, st>>>(M, wprim, np, nbins, row, lmax, slot, lbase, kp, ahi,
                                                               alo, bhi, blo, err, kTcTimeoutCycles);
  } else {
    e = cudaFuncSetAttribute(k_pack<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_pack<false><<<(unsigned)blocks, kPackThreads, smem, st>>>(M, wprim, np, nbins, row, lmax, slot, lbase, kp, ahi,
                                                                alo, bhi, blo, err, kTcTimeoutCycles);
  }
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_contract_tc(bool tf32, int64_t np, int nbins, int lmax, const unsigned long long* h_lbase,
                               const unsigned long long* h_kp, void* ahi, void* alo, void* bhi, void* blo,
                               double* partial, int nsplit, unsigned int* err, bool inject_stall,
                               cudaStream_t st) {
  if (np == 0) return cudaSuccess;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const int npad = tc_npad(nbins);
  const size_t esz = tf32 ? 4 : 2;
  const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  TcArgs a{};
  a.nl = lmax + 1;
  a.nbins = nbins;
  a.npad = npad;
  a.nsplit = nsplit;
  a.partial = partial;
  a.err = err;
  // about 2 s per wait; an injected stall gives up after about 10 ms
  a.timeout_cycles = inject_stall ? 20000000ll : kTcTimeoutCycles;
  a.inject_stall = inject_stall ? 1 : 0;
  void* bases[4] = {ahi, alo, bhi, blo};
  for (int l = 0; l <= lmax; ++l) {
    a.ktiles[l] = (unsigned int)(h_kp[l] / (tf32 ? 32 : 64));
    for (int k = 0; k < 4; ++k) {
      if (tf32 && (k == 1 || k == 3)) continue;
      void* gaddr = static_cast<char*>(bases[k]) + h_lbase[l] * esz;
      cuuint64_t gdim[2] = {(cuuint64_t)h_kp[l], (cuuint64_t)nbins};
      cuuint64_t gstride[1] = {(cuuint64_t)(h_kp[l] * esz)};
      cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)(k < 2 ? 128 : npad)};
      cuuint32_t estr[2] = {1, 1};
      CUresult r = enc(&maps.m[l][k], dt, 2, gaddr, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
  }
  const size_t stage = tc_stage_bytes(tf32, nbins);
  const size_t budget = 220 * 1024;
  a.stages = (int)std::max<size_t>(2, std::min<size_t>(8, (budget - 1024 - 256) / stage));
  int ncols = 32;
  while (ncols < 2 * npad) ncols *= 2;
  a.ncols = ncols;
  const size_t smem = 1024 + a.stages * stage + 256;
  cudaError_t e;
  if (tf32) {
    e = cudaFuncSetAttribute(k_contract_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_contract_tc<true><<<dim3(nsplit, lmax + 1), kTcThreads, smem, st>>>(maps, a);
  } else {
    e = cudaFuncSetAttribute(k_contract_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_contract_tc<false><<<dim3(nsplit, lmax + 1), kTcThreads, smem, st>>>(maps, a);
  }
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
