// contract.cu -- the zeta contraction on the CUDA cores (plain FP32 form) and
// the FP64 cross-block reduction + normalisation.
//
//   zeta~_l(b1,b2) = sum_p w_p sum_{m=-l..l} a_lm(p,b1) a_lm(p,b2)
//   zeta_l(b1,b2)  = 4 pi / (2l+1) zeta~_l(b1,b2)
// (the estimator the paper's "Implementation" section fills bin by bin; its
// normalisation is the triplet-sum one, so that zeta_0 = sum_p w_p N_p N_p).
#include "ctb_internal.cuh"

namespace ctb {

// Register-tiled form.  For one l, zeta~_l restricted to bins [4B1, 4B1+4) x
// [4B2, 4B2+4) is a 4x4 tile: per primary and per m, one 16-byte shared load
// of each side (bins contiguous) and 16 FMAs.  Work split of a block:
//   warp  -> a multipole pair (l, L - l) (one l when l = L - l), so every warp
//            does 2L + 2 m-steps per primary and no lane diverges on l;
//            pairs with more than 32 tiles take several warps
//   lane  -> a tile B1 <= B2 and an m-group g: lanes of the same tile split the
//            m-steps (m = g, g + G, ...) and are added in group order at the end
// The block stages a few primaries' rows transposed to [primary][l^2+l+m][bin]
// (bins padded to a multiple of 4 with zeros).  FP32 over the block's slice of
// the launch's primaries, then one FP64 add per (l, b1 <= b2) entry, whose
// owner is a single lane: the partial sums are deterministic.
constexpr int kConTile = 4;
constexpr int kConMaxThreads = 512;
constexpr int kConStageFloats = 10240;  // 40 KB of staged rows: several blocks per SM

struct ConShape {
  int nbb, tiles, G, warps_per_pair, pairs, pairs_per_block, ny, threads, Q, per, red_floats, tab_ints,
      smem_floats;
};

__host__ __device__ inline ConShape con_shape(int nbins, int lmax, int row, int sphere) {
  ConShape c{};
  c.nbb = (nbins + kConTile - 1) / kConTile;
  c.tiles = c.nbb * (c.nbb + 1) / 2;
  c.warps_per_pair = (c.tiles + 31) / 32;
  c.G = c.tiles >= 32 ? 1 : 32 / c.tiles;
  c.pairs = lmax / 2 + 1;
  // at most kConMaxThreads a block: more pairs go to further blocks in y
  c.pairs_per_block = kConMaxThreads / (32 * c.warps_per_pair);
  if (c.pairs_per_block > c.pairs) c.pairs_per_block = c.pairs;
  c.ny = (c.pairs + c.pairs_per_block - 1) / c.pairs_per_block;
  c.threads = 32 * c.warps_per_pair * c.pairs_per_block;
  const int nc = sphere ? 2 * lmax + 1 : (lmax + 1) * (lmax + 1);
  c.per = nc * c.nbb * kConTile;
  c.Q = c.per >= kConStageFloats ? 1 : kConStageFloats / c.per;
  c.red_floats = c.G > 1 ? (c.threads / 32) * 32 * 17 : 0;
  c.tab_ints = (row + 3) & ~3;  // row slot -> l^2 + l + m, or -1
  c.smem_floats = c.tab_ints + c.Q * c.per + c.red_floats;
  return c;
}

// 4x4 tile of one group (a multipole l: components l^2 .. l^2 + 2l; on the
// sphere, m: component 0, or 2m-1 and 2m): acc[i][j] += w * sum_{c in group} x_i y_j,
// the lanes of the tile's m-groups taking every G-th component.
__device__ __forceinline__ void con_tile(const float* __restrict__ S, int nbp, int s0, int nc, int g, int G, int B1,
                                         int B2, float w, float (&acc)[16]) {
  for (int m = g; m < nc; m += G) {
    const float4 x = *reinterpret_cast<const float4*>(S + (s0 + m) * nbp + 4 * B1);
    const float4 y = *reinterpret_cast<const float4*>(S + (s0 + m) * nbp + 4 * B2);
    const float xs[4] = {w * x.x, w * x.y, w * x.z, w * x.w};
    const float ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i * 4 + j] = fmaf(xs[i], ys[j], acc[i * 4 + j]);
  }
}

__device__ __forceinline__ int group_start(int l, int sphere) { return sphere ? (l == 0 ? 0 : 2 * l - 1) : l * l; }
__device__ __forceinline__ int group_size(int l, int sphere) { return sphere ? (l == 0 ? 1 : 2) : 2 * l + 1; }

__device__ __forceinline__ void con_flush(const ConShape& sh, const float (&acc)[16], int l, int tile, int g, int B1,
                                          int B2, int nb, int lmax, double* __restrict__ out, float* s_red,
                                          int lane) {
  // lanes of one tile: add the m-groups in order through shared memory
  float* mine = s_red + lane * 17;
  if (sh.G > 1) {
#pragma unroll
    for (int k = 0; k < 16; ++k) mine[k] = acc[k];
  }
  __syncwarp();
  if (g == 0 && tile < sh.tiles && l <= lmax) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      float v = acc[k];
      for (int h = 1; h < sh.G; ++h) v += s_red[(lane + h * sh.tiles) * 17 + k];
      const int b1 = 4 * B1 + k / 4, b2 = 4 * B2 + k % 4;
      if (b1 < nb && b2 < nb && b1 <= b2) out[((size_t)l * nb + b1) * nb + b2] += (double)v;
    }
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kConMaxThreads, 1) k_contract_fp32(ContractArgs a) {
  extern __shared__ float s_dyn[];
  const int nb = a.nbins, L = a.lmax;
  const int nc = a.sphere ? 2 * L + 1 : (L + 1) * (L + 1);  // coefficients per (primary, bin)
  const ConShape sh = con_shape(nb, L, a.row, a.sphere);
  const int nbp = sh.nbb * kConTile;
  const int per = sh.per;
  // [row slot -> coefficient table | Q staged primaries | per-warp m-group combine buffers]
  int* s_inv = reinterpret_cast<int*>(s_dyn);
  float* s_rows = s_dyn + sh.tab_ints;
  float* s_red_all = s_rows + sh.Q * per;
  for (int k = threadIdx.x; k < a.row; k += blockDim.x) s_inv[k] = -1;
  for (int k = threadIdx.x; k < sh.Q * per; k += blockDim.x) s_rows[k] = 0.f;  // bin padding stays zero
  __syncthreads();
  for (int c = threadIdx.x; c < nc; c += blockDim.x) s_inv[a.slot[c]] = c;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int pair = blockIdx.y * sh.pairs_per_block + warp / sh.warps_per_pair;
  const int part = warp % sh.warps_per_pair;
  const int la = pair, lb = L - pair;
  const int tl = lane % (sh.G == 1 ? 32 : sh.tiles);
  const int g = sh.G == 1 ? 0 : lane / sh.tiles;
  const int tile = part * 32 + tl;
  const bool active = pair < sh.pairs && tile < sh.tiles && g < sh.G;
  int B1 = 0, B2 = 0;
  {
    int r = active ? tile : 0;
    while (r >= sh.nbb - B1) {
      r -= sh.nbb - B1;
      ++B1;
    }
    B2 = B1 + r;
  }
  float acc_a[16], acc_b[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc_a[k] = acc_b[k] = 0.f;
  const int64_t slice = (a.np + gridDim.x - 1) / gridDim.x;
  const int64_t p0 = (int64_t)blockIdx.x * slice;
  const int64_t p1 = min(a.np, p0 + slice);
  const int rowsz = nb * a.row;
  const bool vec4 = (a.row & 3) == 0 && (reinterpret_cast<uintptr_t>(a.M) & 15) == 0;
  for (int64_t pb = p0; pb < p1; pb += sh.Q) {
    const int cnt = (int)min((int64_t)sh.Q, p1 - pb);
    __syncthreads();  // the previous primaries are done (and the tables / zero fill on entry)
    // coalesced loads of the rows (16 bytes when rows and base allow it),
    // scattered to [primary][coefficient][bin]
    if (vec4) {
      // consecutive lanes take consecutive bins of the same four slots: their
      // transposed stores land in consecutive words (no bank conflicts)
      const float4* src = reinterpret_cast<const float4*>(a.M + (uint64_t)pb * rowsz);
      const int row4 = a.row >> 2;
      for (int k = threadIdx.x; k < cnt * nb * row4; k += blockDim.x) {
        const int r = k / nb, b = k - r * nb;  // r = primary * row4 + c4
        const int q = r / row4, c4 = r - q * row4;
        const float4 v = __ldcs(src + ((q * nb + b) * row4 + c4));
        const float e[4] = {v.x, v.y, v.z, v.w};
        float* dst = s_rows + q * per + b;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = s_inv[4 * c4 + i];
          if (c >= 0) dst[c * nbp] = e[i];
        }
      }
    } else {
      const float* src = a.M + (uint64_t)pb * rowsz;
      for (int k = threadIdx.x; k < cnt * nb * a.row; k += blockDim.x) {
        const int pr = k / a.row, sl = k - pr * a.row;
        const int q = pr / nb, b = pr - q * nb;
        const int c = s_inv[sl];
        if (c >= 0) s_rows[q * per + c * nbp + b] = __ldcs(src + k);
      }
    }
    __syncthreads();
    if (active) {
      for (int q = 0; q < cnt; ++q) {
        const float w = a.wprim[pb + q];
        const float* S = s_rows + q * per;
        con_tile(S, nbp, group_start(la, a.sphere), group_size(la, a.sphere), g, sh.G, B1, B2, w, acc_a);
        if (lb != la)
          con_tile(S, nbp, group_start(lb, a.sphere), group_size(lb, a.sphere), g, sh.G, B1, B2, w, acc_b);
      }
    }
  }
  if (pair >= sh.pairs) return;
  double* out = a.partial + (size_t)(a.part0 + blockIdx.x) * (L + 1) * nb * nb;
  float* s_red = s_red_all + warp * 32 * 17;
  con_flush(sh, acc_a, la, tile, g, B1, B2, nb, L, out, s_red, lane);
  if (lb != la) con_flush(sh, acc_b, lb, tile, g, B1, B2, nb, L, out, s_red, lane);
}

// Resident blocks per SM of the contraction for this shape (0 if it cannot run).
int contract_fp32_blocks_per_sm(int nbins, int lmax, int row, int sphere) {
  const ConShape sh = con_shape(nbins, lmax, row, sphere);
  const size_t smem = (size_t)sh.smem_floats * sizeof(float);
  if (smem > 200 * 1024) return 0;
  if (cudaFuncSetAttribute(k_contract_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_contract_fp32, sh.threads, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_contract_fp32(const ContractArgs& a, int nparts, cudaStream_t st) {
  if (a.np == 0) return cudaSuccess;
  const ConShape sh = con_shape(a.nbins, a.lmax, a.row, a.sphere);
  const size_t smem = (size_t)sh.smem_floats * sizeof(float);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_contract_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_contract_fp32<<<dim3(nparts, sh.ny), sh.threads, smem, st>>>(a);
  ++g_launches;
  return cudaGetLastError();
}

// zeta_l(b1,b2) = f_l * sum_parts partial[part][l][min b][max b], in part
// order; f_l = 4 pi/(2l+1) for the 3-D multipoles, 1 on the sphere.
__global__ void k_finalize(const double* __restrict__ partial, int nparts, int lmax, int nb, int sphere,
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
    zeta[o] = sphere ? s : s * (4.0 * 3.14159265358979323846 / (2.0 * l + 1.0));
  }
}

cudaError_t launch_finalize(const double* partial, int nparts, int lmax, int nbins, double* zeta, bool sphere,
                            cudaStream_t st) {
  const int total = (lmax + 1) * nbins * nbins;
  const int blocks = (total + 255) / 256;
  k_finalize<<<blocks, 256, 0, st>>>(partial, nparts, lmax, nbins, sphere ? 1 : 0, zeta);
  ++g_launches;
  return cudaGetLastError();
}

// Weighted pair sums of the two-point function from the same pass:
// sum_p w_p sum_{j in b} w_j = sqrt(4 pi) sum_p w_p a_00(p, b), the a_00 column
// of the M rows (col).  Block bx takes a fixed slice of the primaries, four
// thread groups interleave over it, and the groups are added in a fixed order
// to partial[bx][b] (FP64; accumulated over the chunks of one compute).
__global__ void __launch_bounds__(256) k_pair_sums(const float* __restrict__ M, const float* __restrict__ w,
                                                   int64_t np, int nbins, int row, int col,
                                                   double* __restrict__ partial) {
  __shared__ double s[4][kNbinsCap];
  const int64_t nparts = gridDim.x, bx = blockIdx.x;
  const int64_t p0 = np * bx / nparts, p1 = np * (bx + 1) / nparts;
  const int g = threadIdx.x >> 6, b = threadIdx.x & 63;
  double acc = 0.0;
  if (b < nbins)
    for (int64_t p = p0 + g; p < p1; p += 4) acc += (double)w[p] * (double)M[(p * nbins + b) * row + col];
  s[g][b] = acc;
  __syncthreads();
  if (threadIdx.x < nbins) {
    const int bb = threadIdx.x;
    partial[bx * nbins + bb] += (s[0][bb] + s[1][bb]) + (s[2][bb] + s[3][bb]);
  }
}

cudaError_t launch_pair_sums(const float* M, const float* w, int64_t np, int nbins, int row, int col,
                             double* partial, int nparts, cudaStream_t st) {
  k_pair_sums<<<nparts, 256, 0, st>>>(M, w, np, nbins, row, col, partial);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ctb
