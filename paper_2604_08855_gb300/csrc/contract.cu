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
// of each side (four bins contiguous) and eight paired FMAs.  Work split of a
// block: every (multipole pair (l, L - l), tile B1 <= B2) is a task, and G
// consecutive threads share a task, splitting its m-steps (m = g, g + G,
// ...) and adding their partial tiles in thread order at the end.  A pair
// does 2L + 2 m-steps per primary whatever its l (one l when l = L - l), so
// the threads of a warp stay in step.  All pairs of a primary fit one block
// (up to 512 threads), so each row is read from HBM once; larger shapes
// split the pairs over blockIdx.y.
//
// Staging: the block walks its slice of the launch's primaries in stages of
// Q primaries, double-buffered in shared memory.  While the FMAs run on one
// buffer, the next stage's rows are in flight in registers: a warp loads 4
// bins x 8 float4 (one 128-byte line per bin), and each thread scatters its
// float4 to the staged layout [slot][bin], slot s at row s * nbp + 4 (s / 8):
// the 4 (s / 8) shift puts the 32 scalar stores of a warp (8 consecutive
// slots x 4 bins) in 32 distinct banks when nbp = 4 mod 32.  Bins are padded
// to a multiple of 4 with zeros.  Shapes whose tasks fit 256 threads (short
// rows: the sphere's, l_max 10) run two such blocks per SM with half-size
// stages; the stage size of short rows is raised with extra loader warps so
// that a stage still fits the registers.  When two buffers do not fit (64 bins at
// l_max 20), one buffer is staged between two barriers, the next stage's
// loads still in flight during the FMAs.  FP32 over the block's slice, then one FP64
// add per (l, b1 <= b2) entry, whose owner is a single thread: the partial
// sums are deterministic.
constexpr int kConTile = 4;
constexpr int kConMaxThreads = 512;
constexpr int kConStageFloats = 20480;  // one staged buffer at most (80 KB; two are used)
constexpr int kConPF = 8;              // float4 loads a thread keeps in flight per stage
constexpr size_t kConSmemCap = 220 * 1024;
constexpr int kConMaxQ = 64;            // primaries per stage at most
// shapes whose tasks fit this many threads run two blocks per SM (half the
// threads, half the staged rows each: 2 x 256 threads x 128 registers)
constexpr int kConSmallThreads = 256;

struct ConShape {
  int nbb;           // bin quads
  int nbp;           // floats per staged slot row
  int tiles;         // 4x4 tiles B1 <= B2
  int pairs;         // multipole pairs (l, L - l)
  int G;             // threads per task
  int ppb, ny;       // pairs per block, blocks in y
  int threads;
  int nch;           // load chunks of 8 float4 along a row
  int srow;          // floats per staged primary
  int Q;             // primaries per stage
  int nbuf;          // staged buffers: 2, or 1 when two do not fit
  int tab_ints;      // coefficient -> slot table
  int stage_floats;  // all buffers
  int red_floats;    // the end-of-kernel combine buffer (aliases the stages)
  int smem_floats;
};

__host__ __device__ inline ConShape con_shape(int nbins, int lmax, int row, int sphere) {
  ConShape c{};
  c.nbb = (nbins + kConTile - 1) / kConTile;
  c.nbp = kConTile * c.nbb;
  if (c.nbp % 32 == 0) c.nbp += 4;
  c.tiles = c.nbb * (c.nbb + 1) / 2;
  c.pairs = lmax / 2 + 1;
  const int nc = sphere ? 2 * lmax + 1 : (lmax + 1) * (lmax + 1);
  const int msteps = sphere ? 4 : 2 * lmax + 2;  // m-steps of the longest pair
  const bool small = c.pairs * c.tiles <= kConSmallThreads;
  const int tmax = small ? kConSmallThreads : kConMaxThreads;
  if (c.pairs * c.tiles <= kConMaxThreads) {
    c.ppb = c.pairs;
    c.G = tmax / (c.pairs * c.tiles);
    if (c.G > msteps) c.G = msteps;
    if (c.G > 32) c.G = 32;
  } else {
    c.G = 1;
    c.ppb = kConMaxThreads / c.tiles;
  }
  c.ny = (c.pairs + c.ppb - 1) / c.ppb;
  c.threads = (c.ppb * c.tiles * c.G + 31) / 32 * 32;
  c.nch = ((row + 3) / 4 + 7) / 8;
  {
    // enough warps that one primary's rows are in flight in registers
    const int wl = (c.nbb * c.nch + kConPF - 1) / kConPF;
    if (c.threads < 32 * wl) c.threads = 32 * wl < tmax ? 32 * wl : tmax;
  }
  c.srow = (row * c.nbp + 4 * ((row + 7) / 8) + 3) & ~3;
  const int units1 = c.nbb * c.nch;  // load units of one primary
  int q = (small ? kConStageFloats / 2 : kConStageFloats) / c.srow;
  if (q > kConMaxQ) q = kConMaxQ;
  if (q < 1) q = 1;
  {
    // short rows: more warps (idle in the FMAs) so that a stage of q
    // primaries is still loaded from registers
    const int wq = (q * units1 + kConPF - 1) / kConPF;
    if (c.threads < 32 * wq) c.threads = 32 * wq < tmax ? 32 * wq : tmax;
  }
  const int warps = c.threads / 32;
  c.Q = q;
  if (c.Q * units1 > kConPF * warps) c.Q = kConPF * warps / units1;  // keep a stage's loads in registers
  if (c.Q < 1) c.Q = 1;
  // coefficient -> staged row offset, then the staged primaries' weights
  c.tab_ints = ((nc + 3) & ~3) + 2 * kConMaxQ;
  c.nbuf = (size_t)(c.tab_ints + 2 * c.Q * c.srow) * 4 <= kConSmemCap ? 2 : 1;
  c.stage_floats = c.nbuf * c.Q * c.srow;
  c.red_floats = c.threads * 17;
  c.smem_floats = c.tab_ints + (c.stage_floats > c.red_floats ? c.stage_floats : c.red_floats);
  (void)nc;
  return c;
}

__device__ __forceinline__ int group_start(int l, int sphere) { return sphere ? (l == 0 ? 0 : 2 * l - 1) : l * l; }
__device__ __forceinline__ int group_size(int l, int sphere) { return sphere ? (l == 0 ? 1 : 2) : 2 * l + 1; }

// offset of slot s of staged primary q
__device__ __forceinline__ int con_off(const ConShape& sh, int q, int s) { return q * sh.srow + s * sh.nbp + 4 * (s >> 3); }

// 4x4 tile of one group (a multipole l: components l^2 .. l^2 + 2l; on the
// sphere, m: component 0, or 2m-1 and 2m): acc += w x y^T summed over the
// group's components, the task's threads taking every G-th component.
// acc[2 i + j] holds entries (i, 2j) and (i, 2j + 1).
__device__ __forceinline__ void con_tile(const float* __restrict__ S, int G, const int* s_offc, int c0, int nc, int g,
                                         int B1, int B2, float w, float2 (&acc)[8]) {
  const float* Sx = S + 4 * B1;
  const float* Sy = S + 4 * B2;
#pragma unroll 2
  for (int m = g; m < nc; m += G) {
    const int off = s_offc[c0 + m];
    const float4 x = *reinterpret_cast<const float4*>(Sx + off);
    const float4 y = *reinterpret_cast<const float4*>(Sy + off);
    const float2 y01 = make_float2(y.x, y.y), y23 = make_float2(y.z, y.w);
    const float2 x01 = __fmul2_rn(make_float2(w, w), make_float2(x.x, x.y));
    const float2 x23 = __fmul2_rn(make_float2(w, w), make_float2(x.z, x.w));
    acc[0] = __ffma2_rn(make_float2(x01.x, x01.x), y01, acc[0]);
    acc[1] = __ffma2_rn(make_float2(x01.x, x01.x), y23, acc[1]);
    acc[2] = __ffma2_rn(make_float2(x01.y, x01.y), y01, acc[2]);
    acc[3] = __ffma2_rn(make_float2(x01.y, x01.y), y23, acc[3]);
    acc[4] = __ffma2_rn(make_float2(x23.x, x23.x), y01, acc[4]);
    acc[5] = __ffma2_rn(make_float2(x23.x, x23.x), y23, acc[5]);
    acc[6] = __ffma2_rn(make_float2(x23.y, x23.y), y01, acc[6]);
    acc[7] = __ffma2_rn(make_float2(x23.y, x23.y), y23, acc[7]);
  }
}

// The G threads of a task add their tiles in thread order (through shared
// memory), and the first adds the result to the block's FP64 partial.
__device__ __forceinline__ void con_flush(const ConShape& sh, const float2 (&acc)[8], bool own, int l, int g,
                                          int B1, int B2, int nb, double* __restrict__ out, float* s_red) {
  float* mine = s_red + threadIdx.x * 17;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    mine[2 * k] = acc[k].x;
    mine[2 * k + 1] = acc[k].y;
  }
  __syncthreads();
  if (own && g == 0) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      float v = mine[k];
      for (int h = 1; h < sh.G; ++h) v += s_red[(threadIdx.x + h) * 17 + k];
      // k = 2 (2 i + j') + e: entry (i, 2 j' + e)
      const int i = k >> 2, j = k & 3;
      const int b1 = 4 * B1 + i, b2 = 4 * B2 + j;
      if (b1 < nb && b2 < nb && b1 <= b2) out[((size_t)l * nb + b1) * nb + b2] += (double)v;
    }
  }
  __syncthreads();
}

// Load units: 4 bins x 8 float4 of a row (lane l: bin 4 bq + l / 8, float4
// 8 ch + l % 8) of staged primary q, u = (q nbb + bq) nch + ch.  Warp w owns
// units [w upw, (w + 1) upw) of a stage, walked by incrementing (q, bq, ch).
struct ConUnit {
  int q, bq, ch;
};
__device__ __forceinline__ void con_next(const ConShape& sh, ConUnit& t) {
  if (++t.ch == sh.nch) {
    t.ch = 0;
    if (++t.bq == sh.nbb) {
      t.bq = 0;
      ++t.q;
    }
  }
}

__device__ __forceinline__ void con_store4(float* buf, const ConShape& sh, int q, int b, int c4, float4 v) {
  const int s = 4 * c4;
  float* d = buf + con_off(sh, q, s) + b;
  // slots s .. s + 3 share s / 8
  d[0] = v.x;
  d[sh.nbp] = v.y;
  d[2 * sh.nbp] = v.z;
  d[3 * sh.nbp] = v.w;
}

__global__ void __launch_bounds__(kConMaxThreads, 1) k_contract_fp32(ContractArgs a) {
  extern __shared__ __align__(16) float s_dyn[];
  const int nb = a.nbins, L = a.lmax;
  const int nc = a.sphere ? 2 * L + 1 : (L + 1) * (L + 1);  // coefficients per (primary, bin)
  const ConShape sh = con_shape(nb, L, a.row, a.sphere);
  // [coefficient -> staged row offset | weights of the staged primaries, per
  //  buffer | staged buffers (the combine buffer at the end)]
  int* s_offc = reinterpret_cast<int*>(s_dyn);
  float* s_w = s_dyn + (sh.tab_ints - 2 * kConMaxQ);
  float* s_stage = s_dyn + sh.tab_ints;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    const int sl = a.slot[c];
    s_offc[c] = sl * sh.nbp + 4 * (sl >> 3);
  }
  for (int k = threadIdx.x; k < sh.stage_floats; k += blockDim.x) s_stage[k] = 0.f;  // bin padding stays zero
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int task = tid / sh.G, g = tid - task * sh.G;
  const int pair = blockIdx.y * sh.ppb + task / sh.tiles;
  const int tile = task % sh.tiles;
  const bool active = task < sh.ppb * sh.tiles && pair < sh.pairs;
  int B1 = 0, B2 = 0;
  {
    int r = active ? tile : 0;
    while (r >= sh.nbb - B1) {
      r -= sh.nbb - B1;
      ++B1;
    }
    B2 = B1 + r;
  }
  const int la = pair, lb = L - pair;
  float2 acc_a[8], acc_b[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc_a[k] = acc_b[k] = make_float2(0.f, 0.f);
  const int64_t slice = (a.np + gridDim.x - 1) / gridDim.x;
  const int64_t p0 = (int64_t)blockIdx.x * slice;
  const int64_t p1 = min(a.np, p0 + slice);
  const int64_t rowsz = (int64_t)nb * a.row;
  const bool vec4 = (a.row & 3) == 0 && (reinterpret_cast<uintptr_t>(a.M) & 15) == 0;
  const int row4 = a.row >> 2;
  const int units = sh.Q * sh.nbb * sh.nch;  // load units of a full stage
  const int upw = (units + nwarps - 1) / nwarps;   // units per warp
  ConUnit t0;  // this warp's first unit
  {
    const int u0 = warp * upw, per = sh.nbb * sh.nch;
    t0.q = u0 / per;
    t0.bq = (u0 - t0.q * per) / sh.nch;
    t0.ch = u0 - t0.q * per - t0.bq * sh.nch;
  }
  const int lb8 = lane >> 3, lc8 = lane & 7;
  __syncthreads();

  // rows of the stage at pb (cnt primaries) into buffer buf: the warp's
  // first kConPF units from registers (loaded by issue), the rest here
  float4 pf[kConPF];
  float wpf = 0.f;  // thread q < Q: the weight of staged primary q
  auto issue = [&](int64_t pb, int cnt) {
    if (tid < cnt) wpf = __ldg(a.wprim + pb + tid);
    const float4* src = reinterpret_cast<const float4*>(a.M + pb * rowsz);
    ConUnit t = t0;
#pragma unroll
    for (int i = 0; i < kConPF; ++i) {
      const int b = 4 * t.bq + lb8, c4 = 8 * t.ch + lc8;
      if (i < upw && t.q < cnt && b < nb && c4 < row4) pf[i] = __ldcs(src + ((int64_t)t.q * nb + b) * row4 + c4);
      con_next(sh, t);
    }
  };
  auto land = [&](float* buf, int64_t pb, int cnt) {
    if (tid < cnt) s_w[(buf == s_stage ? 0 : kConMaxQ) + tid] = wpf;
    ConUnit t = t0;
#pragma unroll
    for (int i = 0; i < kConPF; ++i) {
      const int b = 4 * t.bq + lb8, c4 = 8 * t.ch + lc8;
      if (i < upw && t.q < cnt && b < nb && c4 < row4) con_store4(buf, sh, t.q, b, c4, pf[i]);
      con_next(sh, t);
    }
    const float4* src = reinterpret_cast<const float4*>(a.M + pb * rowsz);
    for (int i = kConPF; i < upw; ++i) {
      const int b = 4 * t.bq + lb8, c4 = 8 * t.ch + lc8;
      if (t.q < cnt && b < nb && c4 < row4)
        con_store4(buf, sh, t.q, b, c4, __ldcs(src + ((int64_t)t.q * nb + b) * row4 + c4));
      con_next(sh, t);
    }
  };
  // scalar rows (a row length that is not a multiple of 4, or an unaligned base)
  auto land1 = [&](float* buf, int64_t pb, int cnt) {
    if (tid < cnt) s_w[(buf == s_stage ? 0 : kConMaxQ) + tid] = __ldg(a.wprim + pb + tid);
    const float* src = a.M + pb * rowsz;
    for (int64_t k = tid; k < (int64_t)cnt * rowsz; k += blockDim.x) {
      const int64_t pr = k / a.row;
      const int s = (int)(k - pr * a.row);
      const int q = (int)(pr / nb), b = (int)(pr - (int64_t)q * nb);
      buf[con_off(sh, q, s) + b] = __ldcs(src + k);
    }
  };

  int cur = 0;
  if (p0 < p1) {
    const int cnt = (int)min((int64_t)sh.Q, p1 - p0);
    if (vec4) {
      issue(p0, cnt);
      land(s_stage, p0, cnt);
    } else {
      land1(s_stage, p0, cnt);
    }
  }
  __syncthreads();
  for (int64_t pb = p0; pb < p1; pb += sh.Q) {
    const int cnt = (int)min((int64_t)sh.Q, p1 - pb);
    const int64_t pn = pb + sh.Q;
    const int cntn = pn < p1 ? (int)min((int64_t)sh.Q, p1 - pn) : 0;
    float* bufc = s_stage + cur * sh.Q * sh.srow;
    float* bufn = s_stage + (sh.nbuf == 2 ? cur ^ 1 : 0) * sh.Q * sh.srow;
    if (vec4 && cntn > 0) issue(pn, cntn);  // in flight during the FMAs
    if (active) {
      const float* wq = s_w + (bufc == s_stage ? 0 : kConMaxQ);
      for (int q = 0; q < cnt; ++q) {
        const float w = wq[q];
        const float* S = bufc + q * sh.srow;
        con_tile(S, sh.G, s_offc, group_start(la, a.sphere), group_size(la, a.sphere), g, B1, B2, w, acc_a);
        if (lb != la) con_tile(S, sh.G, s_offc, group_start(lb, a.sphere), group_size(lb, a.sphere), g, B1, B2, w, acc_b);
      }
    }
    if (cntn > 0) {
      if (sh.nbuf == 1) __syncthreads();  // one buffer: every thread is done reading it
      if (vec4) land(bufn, pn, cntn);
      else land1(bufn, pn, cntn);
    }
    __syncthreads();  // bufc is read no more; bufn is staged
    if (sh.nbuf == 2) cur ^= 1;
  }
  if (blockIdx.y * sh.ppb >= sh.pairs) return;  // the whole block has no pair (uniform)
  double* out = a.partial + (size_t)(a.part0 + blockIdx.x) * (L + 1) * nb * nb;
  float* s_red = s_stage;  // the stages are done
  con_flush(sh, acc_a, active && la <= L, la, g, B1, B2, nb, out, s_red);
  con_flush(sh, acc_b, active && lb != la && lb >= 0, lb, g, B1, B2, nb, out, s_red);
}

// Resident blocks per SM of the contraction for this shape (0 if it cannot run).
int contract_fp32_blocks_per_sm(int nbins, int lmax, int row, int sphere) {
  const ConShape sh = con_shape(nbins, lmax, row, sphere);
  const size_t smem = (size_t)sh.smem_floats * sizeof(float);
  if (smem > kConSmemCap) return 0;
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
  if (smem > kConSmemCap) return cudaErrorInvalidValue;
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
