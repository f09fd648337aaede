// contract.cu -- the zeta contraction on the CUDA cores (plain FP32 form) and
// the FP64 cross-block reduction + normalisation.
//
//   zeta~_l(b1,b2) = sum_p w_p sum_{m=-l..l} a_lm(p,b1) a_lm(p,b2)
//   zeta_l(b1,b2)  = 4 pi / (2l+1) zeta~_l(b1,b2)
// (the estimator the paper's "Implementation" section fills bin by bin; its
// normalisation is the triplet-sum one, so that zeta_0 = sum_p w_p N_p N_p).
#include "ctb_internal.cuh"

namespace ctb {

constexpr int kConThreads = 512;
constexpr int kConMaxPer = 24;       // entries per thread (registers)
constexpr int kConFlush = 64;        // primaries per FP32 partial before FP64
constexpr int kConSmemFloats = 24576;  // 96 KB of staged rows
constexpr int kConGroup = kConThreads * kConMaxPer;  // entries per block (grid.y splits more)

// Block (x, y) owns partial row (part0 + x), a contiguous range of primaries,
// and entries [y * kConGroup, (y+1) * kConGroup) of the upper triangle
// (l, b1 <= b2); each thread owns up to kConMaxPer of them.  Staged rows use
// an odd smem stride (row + 1 floats) so that lanes reading the same slot of
// different bins hit different banks.  FP32 sums over kConFlush primaries,
// then FP64.
__global__ void __launch_bounds__(kConThreads) k_contract_fp32(ContractArgs a) {
  extern __shared__ float s_dyn[];
  __shared__ int s_slot[(kLmaxCap + 1) * (kLmaxCap + 1)];
  const int nb = a.nbins, row = a.row, srow = a.row + 1;
  const int rowsz = nb * row, srowsz = nb * srow;
  const int rows_cap = srowsz > kConSmemFloats ? srowsz : kConSmemFloats;
  float* s_rows = s_dyn;
  const int T = nb * (nb + 1) / 2;
  const int e_lo = blockIdx.y * kConGroup;
  const int E = min((a.lmax + 1) * T - e_lo, kConGroup);
  const int nc = (a.lmax + 1) * (a.lmax + 1);
  for (int c = threadIdx.x; c < nc; c += blockDim.x) s_slot[c] = a.slot[c];
  uint32_t md[kConMaxPer];
#pragma unroll
  for (int k = 0; k < kConMaxPer; ++k) {
    const int e = threadIdx.x + k * kConThreads;
    md[k] = 0;
    if (e < E) {
      int l = (e + e_lo) / T, r = (e + e_lo) % T, b1 = 0;
      while (r >= nb - b1) {
        r -= nb - b1;
        ++b1;
      }
      const int b2 = b1 + r;
      md[k] = (uint32_t)l | ((uint32_t)b1 << 5) | ((uint32_t)b2 << 11);
    }
  }
  const int64_t per = (a.np + gridDim.x - 1) / gridDim.x;
  const int64_t p0 = (int64_t)blockIdx.x * per;
  const int64_t p1 = min(a.np, p0 + per);
  const int stage = rows_cap / srowsz;
  float acc[kConMaxPer];
  double acc64[kConMaxPer];
#pragma unroll
  for (int k = 0; k < kConMaxPer; ++k) {
    acc[k] = 0.f;
    acc64[k] = 0.0;
  }
  int since = 0;
  __syncthreads();
  for (int64_t pb = p0; pb < p1; pb += stage) {
    const int cnt = (int)min((int64_t)stage, p1 - pb);
    const float* src = a.M + (uint64_t)pb * rowsz;
    for (int k = threadIdx.x; k < cnt * rowsz; k += blockDim.x) {
      const int rr = k / row, cc = k - rr * row;  // rr = primary * nb + bin
      s_rows[rr * srow + cc] = __ldcs(src + k);
    }
    __syncthreads();
    for (int q = 0; q < cnt; ++q) {
      const float wp = a.wprim[pb + q];
      const float* A = s_rows + q * srowsz;
#pragma unroll
      for (int k = 0; k < kConMaxPer; ++k) {
        const int e = threadIdx.x + k * kConThreads;
        if (e < E) {
          const uint32_t m = md[k];
          const int l = m & 31, b1 = (m >> 5) & 63, b2 = (m >> 11) & 63;
          const float* A1 = A + b1 * srow;
          const float* A2 = A + b2 * srow;
          const int c0 = l * l;
          float s = 0.f;
          for (int c = c0; c <= c0 + 2 * l; ++c) {
            const int sl = s_slot[c];
            s = fmaf(A1[sl], A2[sl], s);
          }
          acc[k] = fmaf(wp, s, acc[k]);
        }
      }
      if (++since == kConFlush) {
        since = 0;
#pragma unroll
        for (int k = 0; k < kConMaxPer; ++k) {
          acc64[k] += (double)acc[k];
          acc[k] = 0.f;
        }
      }
    }
    __syncthreads();
  }
  double* out = a.partial + (size_t)(a.part0 + blockIdx.x) * (a.lmax + 1) * nb * nb;
#pragma unroll
  for (int k = 0; k < kConMaxPer; ++k) {
    const int e = threadIdx.x + k * kConThreads;
    if (e < E) {
      const uint32_t m = md[k];
      const int l = m & 31, b1 = (m >> 5) & 63, b2 = (m >> 11) & 63;
      out[((size_t)l * nb + b1) * nb + b2] += acc64[k] + (double)acc[k];
    }
  }
}

cudaError_t launch_contract_fp32(const ContractArgs& a, int nparts, cudaStream_t st) {
  const int E = (a.lmax + 1) * a.nbins * (a.nbins + 1) / 2;
  const int groups = (E + kConGroup - 1) / kConGroup;
  if (a.np == 0) return cudaSuccess;
  const int srowsz = a.nbins * (a.row + 1);
  const int rows_cap = srowsz > kConSmemFloats ? srowsz : kConSmemFloats;
  const size_t smem = (size_t)rows_cap * sizeof(float);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_contract_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_contract_fp32<<<dim3(nparts, groups), kConThreads, smem, st>>>(a);
  ++g_launches;
  return cudaGetLastError();
}

// zeta_l(b1,b2) = 4 pi/(2l+1) * sum_parts partial[part][l][min b][max b], in part order.
__global__ void k_finalize(const double* __restrict__ partial, int nparts, int lmax, int nb,
                           double* __restrict__ zeta) {
  const int total = (lmax + 1) * nb * nb;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < total; o += gridDim.x * blockDim.x) {
    const int l = o / (nb * nb), r = o % (nb * nb);
    int b1 = r / nb, b2 = r % nb;
    if (b1 > b2) {
      int t = b1;
      b1 = b2;
      b2 = t;
    }
    const size_t idx = ((size_t)l * nb + b1) * nb + b2;
    const size_t stride = (size_t)(lmax + 1) * nb * nb;
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += partial[(size_t)p * stride + idx];
    zeta[o] = s * (4.0 * 3.14159265358979323846 / (2.0 * l + 1.0));
  }
}

cudaError_t launch_finalize(const double* partial, int nparts, int lmax, int nbins, double* zeta,
                            cudaStream_t st) {
  const int total = (lmax + 1) * nbins * nbins;
  const int blocks = (total + 255) / 256;
  k_finalize<<<blocks, 256, 0, st>>>(partial, nparts, lmax, nbins, zeta);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ctb
