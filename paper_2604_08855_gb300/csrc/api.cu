// api.cu -- the libctb C ABI (include/ctb.h): context, buffers, orchestration.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctb_internal.cuh"

using namespace ctb;

namespace ctb {
thread_local unsigned long long g_launches = 0;
}

namespace {

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

thread_local std::string g_create_err;

constexpr int kStages = 9;

}  // namespace

struct ctb_ctx {
  int dev = 0;
  int nsm = 0;
  double box = 0, rmin = 0, rmax = 0;
  int nbins = 0, lmax = 0;
  int periodic = 0;
  // options
  int precision = CTB_PREC_FP32;
  int cells_per_rmax = 0;
  int sphere = 0;            // projected multipoles on the unit sphere (lmax holds m_max)
  double tmin = 0, tmax = 0;  // sphere: angular bin range (radians)
  int autotune = 0;
  int inject = 0;     // CTB_INJECT_* test hook
  int tuned_cpr = 0;  // cells per r_max chosen by the autotuner (0: none yet)
  int wpb = 0;
  int64_t chunk = 0;
  int deterministic = 1;
  cudaStream_t st = nullptr;
  void* (*alloc_fn)(size_t, void*) = nullptr;
  void (*free_fn)(void*, void*) = nullptr;
  void* user = nullptr;
  std::string err;
  // catalogue
  int64_t n = -1;
  bool negw = true;  // the catalogue has a negative weight (from the ingest)
  bool batch_grid = false;  // c->g is the grid of the last batch (c->n < 0 then)
  Geom g{};
  double unit = 0;
  double origin[3] = {0, 0, 0};
  double hi[3] = {0, 0, 0};  // largest coordinate per axis (box for a periodic box)
  double norm2_lo = 0, norm2_hi = 0;  // open space: smallest and largest |p|^2 of the catalogue
  double bbox_volume = 0;
  Layout lay{};
  int Lk = 0;
  float beta[(kLmaxCap + 1) * (kLmaxCap + 1)];
  bool tables_ready = false;
  // device buffers
  Buf xyz_stage, w_stage, key0, val0, key1, val1, hist, scan_tmp, pts_in, pts, s2i, i2s, cell_start;
  Buf flags, bbox_part, lists, M, wprim, partial, zeta, prim, counters, norm, slot, idx64, alm, thr;
  Buf edge_in, edge_tj;  // edge correction: staged sums, 3j table
  Buf pairsum;          // FP64 partial pair sums [catalogue][part][bin] of the last compute
  int pairsum_segs = 0;  // catalogues they cover (0: none)
  int pairsum_parts = 0;
  Buf codes, code_base;  // per-candidate bin codes of a chunk; range start per (primary, row block)
  // shared neighbour lists: sort buffers, segment heads, group ids, scan scratch, representatives, weights
  Buf gk0, gv0, gk1, gv1, glo, ghi, ghead, gid, gscan, gprim, gw;
  const float* wsub = nullptr;  // primary weights replacing the points' own during a shared compute
  double shared_h = 0;          // pivot cell side of the last ctb_compute_shared
  int64_t ngroups = -1;         // its groups (-1: none since ctb_set_points)
  Buf counts, offsets, scan_tmp2;
  Buf ops[4], slot_lm, lbase_d, kp_d, partial_tc, conv;
  uint64_t list_cap = (uint64_t)1 << 32;  // neighbour-list entries per chunk (16 GB)
  const uint32_t* batch_keys = nullptr;    // sorted keys while a batch is loaded
  cudaEvent_t ev[16] = {};
  bool ev_ready = false;
  double t_ms[kStages] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  uint64_t npairs = 0;
  uint64_t nchunks = 0;  // primary chunks of the last compute
  unsigned long long launches_points = 0, launches_compute = 0;
};

namespace {

int fail(ctb_ctx* c, int code, const std::string& what) {
  c->err = what;
  return code;
}

int cuda_fail(ctb_ctx* c, cudaError_t e, const char* where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  cudaGetLastError();
  return fail(c, e == cudaErrorMemoryAllocation ? CTB_ERR_OOM : CTB_ERR_CUDA, msg);
}

#define CK(ctx, call)                                                 \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);        \
  } while (0)

void release(ctb_ctx* c, Buf& b) {
  if (!b.p) return;
  if (c->free_fn)
    c->free_fn(b.p, c->user);
  else
    cudaFreeAsync(b.p, c->st);
  b.p = nullptr;
  b.bytes = 0;
}

// grow-only device buffer
cudaError_t ensure(ctb_ctx* c, Buf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return cudaSuccess;
  if (c->inject == CTB_INJECT_ALLOC) return cudaErrorMemoryAllocation;
  release(c, b);
  size_t want = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (c->alloc_fn) {
    p = c->alloc_fn(want, c->user);
    if (!p) return cudaErrorMemoryAllocation;
  } else {
    cudaError_t e = cudaMallocAsync(&p, want, c->st);
    if (e != cudaSuccess) return e;
  }
  b.p = p;
  b.bytes = want;
  return cudaSuccess;
}

template <class T>
T* P(Buf& b) {
  return static_cast<T*>(b.p);
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void release_all(ctb_ctx* c) {
  Buf* all[] = {&c->xyz_stage, &c->w_stage, &c->key0, &c->val0, &c->key1, &c->val1, &c->hist,
                &c->scan_tmp, &c->pts_in, &c->pts, &c->s2i, &c->i2s, &c->cell_start, &c->flags,
                &c->bbox_part, &c->lists, &c->M, &c->wprim, &c->partial, &c->zeta, &c->prim,
                &c->counters, &c->norm, &c->slot, &c->idx64, &c->alm, &c->thr, &c->codes, &c->code_base, &c->pairsum, &c->edge_in, &c->edge_tj, &c->counts,
                &c->offsets, &c->scan_tmp2, &c->ops[0], &c->ops[1], &c->ops[2], &c->ops[3],
                &c->slot_lm, &c->lbase_d, &c->kp_d, &c->partial_tc, &c->conv, &c->gk0, &c->gv0, &c->gk1, &c->gv1, &c->glo, &c->ghi, &c->ghead, &c->gid, &c->gscan,
                &c->gprim, &c->gw};
  for (Buf* b : all) release(c, *b);
  c->tables_ready = false;
}

int ensure_events(ctb_ctx* c) {
  if (c->ev_ready) return CTB_OK;
  for (auto& e : c->ev) CK(c, cudaEventCreate(&e));
  c->ev_ready = true;
  return CTB_OK;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    return 0.f;
  }
  return ms;
}

// normalisation per slot and the slot table of the context's layout
int ensure_tables_sphere(ctb_ctx* c) {
  // row = [Re a_1, Im a_1, ..., Re a_K, Im a_K, a_0], padded to 32; every
  // slot its own coefficient.  Coefficient index i (0: a_0, 2m-1: Re a_m,
  // 2m: Im a_m) sits in slot i - 1, a_0 in slot 2K.
  const int nc = 2 * c->lmax + 1;
  Layout& y = c->lay;
  y = Layout{};
  y.L = c->lmax;
  y.npass = 1;
  y.row = ((nc + 31) / 32) * 32;
  for (int i = 0; i < (kLmaxCap + 1) * (kLmaxCap + 1); ++i) y.slot[i] = i < nc ? (i == 0 ? 2 * c->lmax : i - 1) : -1;
  // identity flush conversion (one entry per slot; padding slots map to 0)
  std::vector<int2> tab(y.row);
  for (int k = 0; k < y.row; ++k) {
    const float one = k < nc ? 1.f : 0.f;
    tab[k].x = k;
    std::memcpy(&tab[k].y, &one, 4);
  }
  CK(c, ensure(c, c->slot, sizeof(y.slot)));
  CK(c, cudaMemcpyAsync(c->slot.p, y.slot, sizeof(y.slot), cudaMemcpyHostToDevice, c->st));
  CK(c, ensure(c, c->conv, tab.size() * sizeof(int2)));
  CK(c, cudaMemcpyAsync(c->conv.p, tab.data(), tab.size() * sizeof(int2), cudaMemcpyHostToDevice, c->st));
  CK(c, cudaStreamSynchronize(c->st));  // host sources go out of scope
  c->tables_ready = true;
  return CTB_OK;
}

int ensure_tables(ctb_ctx* c) {
  if (c->tables_ready) return CTB_OK;
  if (c->sphere) return ensure_tables_sphere(c);
  c->Lk = lmax_kernel(c->lmax);
  make_layout(c->Lk, &c->lay);
  fill_beta(c->beta);
  std::vector<float> norm(c->lay.row, 0.f);
  for (int l = 0; l <= c->Lk; ++l)
    for (int m = -l; m <= l; ++m) norm[c->lay.slot[l * l + l + m]] = (float)norm_lm(l, m);
  CK(c, ensure(c, c->norm, norm.size() * sizeof(float)));
  CK(c, ensure(c, c->slot, sizeof(c->lay.slot)));
  CK(c, cudaMemcpyAsync(c->norm.p, norm.data(), norm.size() * sizeof(float), cudaMemcpyHostToDevice, c->st));
  CK(c, cudaMemcpyAsync(c->slot.p, c->lay.slot, sizeof(c->lay.slot), cudaMemcpyHostToDevice, c->st));
  // slot -> (l, m + l) for the tensor-core pack: l * 64 + (m + l), -1 for padding and l > ell_max
  std::vector<int> slot_lm(c->lay.row, -1);
  for (int l = 0; l <= c->lmax; ++l)
    for (int m = -l; m <= l; ++m) slot_lm[c->lay.slot[l * l + l + m]] = l * 64 + (m + l);
  std::vector<int2> tab;
  if (!make_conversion(c->lay, tab)) return fail(c, CTB_ERR_CUDA, "internal: flush conversion table overflow");
  CK(c, ensure(c, c->conv, tab.size() * sizeof(int2)));
  CK(c, cudaMemcpyAsync(c->conv.p, tab.data(), tab.size() * sizeof(int2), cudaMemcpyHostToDevice, c->st));
  CK(c, ensure(c, c->slot_lm, slot_lm.size() * sizeof(int)));
  CK(c, cudaMemcpyAsync(c->slot_lm.p, slot_lm.data(), slot_lm.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
  CK(c, cudaStreamSynchronize(c->st));  // host sources go out of scope
  c->tables_ready = true;
  return CTB_OK;
}

// ---------------------------------------------------------------------------
// exact bin-edge thresholds: fixed-width unsigned big integers (16 x 32 bits)

struct U512 {
  uint32_t w[16];
};

U512 u_from(uint64_t v) {
  U512 r{};
  r.w[0] = (uint32_t)v;
  r.w[1] = (uint32_t)(v >> 32);
  return r;
}

U512 u_mul(const U512& a, uint64_t m) {
  U512 r{};
  const uint64_t part[2] = {m & 0xffffffffull, m >> 32};
  for (int h = 0; h < 2; ++h) {
    uint64_t carry = 0;
    for (int i = 0; i + h < 16; ++i) {
      uint64_t t = (uint64_t)a.w[i] * part[h] + r.w[i + h] + carry;
      r.w[i + h] = (uint32_t)t;
      carry = t >> 32;
    }
  }
  return r;
}

U512 u_shl(const U512& a, int k) {
  U512 r{};
  const int q = k / 32, s = k % 32;
  for (int i = 15; i >= 0; --i) {
    uint64_t v = 0;
    if (i - q >= 0) v = (uint64_t)a.w[i - q] << s;
    if (s && i - q - 1 >= 0) v |= (uint64_t)a.w[i - q - 1] >> (32 - s);
    r.w[i] = (uint32_t)v;
  }
  return r;
}

int u_cmp(const U512& a, const U512& b) {
  for (int i = 15; i >= 0; --i)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
  return 0;
}

void split_double(double d, uint64_t* m, int* e) {
  int x = 0;
  double f = std::frexp(d, &x);
  *m = (uint64_t)std::ldexp(f, 53);
  *e = x - 53;
}

}  // namespace

// smallest T >= 0 with T * unit^2 >= edge^2 (edge >= 0, unit > 0), exactly
unsigned long long ctb::sq_threshold(double edge, double unit) {
  if (!(edge > 0)) return 0ull;
  uint64_t mE, mu;
  int eE, eu;
  split_double(edge, &mE, &eE);
  split_double(unit, &mu, &eu);
  const U512 mu2 = u_mul(u_from(mu), mu);
  U512 rhs = u_mul(u_from(mE), mE);
  const int k = 2 * eE - 2 * eu;
  if (k > 0) rhs = u_shl(rhs, k);
  auto ok = [&](unsigned long long T) {
    U512 lhs = u_mul(mu2, T);
    if (k < 0) lhs = u_shl(lhs, -k);
    return u_cmp(lhs, rhs) >= 0;
  };
  unsigned long long lo = 0, hi = 1ull << 62;
  if (!ok(hi)) return hi;
  while (lo < hi) {
    unsigned long long mid = lo + (hi - lo) / 2;
    if (ok(mid))
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

namespace {

// exact edges, the same FP64 values an FP64 evaluation of the bins uses:
// r_min, r_min + b (r_max - r_min)/nbins, r_max
int upload_thresholds(ctb_ctx* c) {
  std::vector<unsigned long long> thr(c->nbins + 1);
  if (c->sphere) {
    // chord edges of the linear angular bins: 2 sin(theta_b / 2)
    for (int b = 0; b <= c->nbins; ++b)
      thr[b] = sq_threshold(2.0 * std::sin(0.5 * (c->tmin + b * (c->tmax - c->tmin) / c->nbins)), c->unit);
    CK(c, ensure(c, c->thr, thr.size() * 8));
    CK(c, cudaMemcpyAsync(c->thr.p, thr.data(), thr.size() * 8, cudaMemcpyHostToDevice, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    return CTB_OK;
  }
  const double dr = (c->rmax - c->rmin) / c->nbins;
  thr[0] = sq_threshold(c->rmin, c->unit);
  for (int b = 1; b < c->nbins; ++b) {
    const double bd = b * dr;
    thr[b] = sq_threshold(c->rmin + bd, c->unit);
  }
  thr[c->nbins] = sq_threshold(c->rmax, c->unit);
  CK(c, ensure(c, c->thr, thr.size() * 8));
  CK(c, cudaMemcpyAsync(c->thr.p, thr.data(), thr.size() * 8, cudaMemcpyHostToDevice, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  return CTB_OK;
}

// float geometry of the grid and bins from c->unit, nc and g.shift
void finish_geom(ctb_ctx* c, Geom& g, uint32_t nc) {
  g.nc = nc;
  uint32_t xs = kXSub;
  while (xs > 1 && (uint64_t)nc * nc * nc * xs >= ((uint64_t)1 << 31)) xs >>= 1;
  g.ncx = nc * xs;
  g.ncells = nc * nc * g.ncx;
  const double rmin_u = c->rmin / c->unit, rmax_u = c->rmax / c->unit;
  // the float pre-filter; never 0, so that it also rejects r = 0
  g.rlo2_u = std::max((float)(rmin_u * rmin_u * (1.0 - 1e-5)), 0.25f);
  g.rhi2_u = (float)(rmax_u * rmax_u * (1.0 + 1e-5));
  g.rmin_u = (float)rmin_u;
  g.inv_dr_u = (float)(c->nbins / (rmax_u - rmin_u));
  g.cell_scale = (float)(nc / std::ldexp(1.0, g.shift));
  g.rcell = (float)(rmax_u * nc / std::ldexp(1.0, g.shift) * (1.0 + 1e-5) + 1e-3);
  g.general = c->sphere;
  if (c->sphere) {
    // the shell sqrt(norm2_lo) <= |p| <= sqrt(norm2_hi) that holds every point,
    // in cell units (centre: the origin of coordinates), padded for rounding
    const double ycell = nc / std::ldexp(1.0, g.shift) / c->unit;  // cells per coordinate unit (y, z)
    g.shell_c[0] = (float)(-c->origin[0] * ycell * (g.ncx / nc));
    g.shell_c[1] = (float)(-c->origin[1] * ycell);
    g.shell_c[2] = (float)(-c->origin[2] * ycell);
    const double rlo = std::sqrt(std::max(c->norm2_lo, 0.0)) * ycell, rhi = std::sqrt(c->norm2_hi) * ycell;
    const double pad = 1e-5 * rhi + 4e-3;
    g.shell_r2lo = (float)(rlo > pad ? (rlo - pad) * (rlo - pad) : 0.0);
    g.shell_r2hi = (float)((rhi + pad) * (rhi + pad));
  }
  g.half_unit = (float)(0.5 * c->unit);
  g.tmin = (float)c->tmin;
  g.inv_dt = c->sphere ? (float)(c->nbins / (c->tmax - c->tmin)) : 0.f;
}

int bits_for(uint32_t ncells) {
  int b = 0;
  while (b < 32 && (1ull << b) < (unsigned long long)ncells) ++b;
  return b;
}

// ---------------------------------------------------------------------------
// catalogue load: ingest -> radix sort by cell -> gather -> cell table

// Cells per r_max along an axis: the option if set, else the autotuner's
// choice, else 8.
int grid_cells_per_rmax(const ctb_ctx* c) {
  if (c->cells_per_rmax > 0) return c->cells_per_rmax;
  return c->tuned_cpr > 0 ? c->tuned_cpr : 8;
}

int load_points(ctb_ctx* c, const double* xyz, const double* w, int64_t n) {
  if (n < 0 || n >= (int64_t)1 << 31) return fail(c, CTB_ERR_ARG, "n out of range [0, 2^31)");
  if (n > 0 && !xyz) return fail(c, CTB_ERR_ARG, "xyz is NULL");
  CK(c, cudaSetDevice(c->dev));
  int r = ensure_events(c);
  if (r) return r;
  c->n = -1;
  c->batch_keys = nullptr;
  c->pairsum_segs = 0;
  c->ngroups = -1;
  c->shared_h = 0;
  const double* dxyz = xyz;
  const double* dw = w;
  if (n > 0 && !is_device_ptr(xyz)) {
    CK(c, ensure(c, c->xyz_stage, (size_t)n * 3 * sizeof(double)));
    CK(c, cudaMemcpyAsync(c->xyz_stage.p, xyz, (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice, c->st));
    dxyz = P<double>(c->xyz_stage);
  }
  if (n > 0 && w && !is_device_ptr(w)) {
    CK(c, ensure(c, c->w_stage, (size_t)n * sizeof(double)));
    CK(c, cudaMemcpyAsync(c->w_stage.p, w, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, c->st));
    dw = P<double>(c->w_stage);
  }
  CK(c, cudaEventRecord(c->ev[0], c->st));
  CK(c, ensure(c, c->flags, 64));
  CK(c, cudaMemsetAsync(c->flags.p, 0, 64, c->st));

  // units and grid
  const int cpr = grid_cells_per_rmax(c);
  Geom g{};
  g.periodic = c->periodic;
  g.nbins = c->nbins;
  g.lmax = c->lmax;
  uint32_t nc = 1;
  if (c->periodic) {
    c->unit = std::ldexp(c->box, -32);
    g.shift = 32;
    double ncd = std::floor(c->box * cpr / c->rmax);
    nc = (uint32_t)std::max(1.0, std::min(ncd, 1024.0));
    c->origin[0] = c->origin[1] = c->origin[2] = 0;
    c->hi[0] = c->hi[1] = c->hi[2] = c->box;
  } else {
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    if (n > 0) {
      int nblk = bbox_blocks(n);
      CK(c, ensure(c, c->bbox_part, (size_t)nblk * 8 * sizeof(double)));
      CK(c, launch_bbox(dxyz, n, P<double>(c->bbox_part), nblk, P<uint32_t>(c->flags), c->st));
      std::vector<double> part((size_t)nblk * 8);
      uint32_t fl = 0;
      CK(c, cudaMemcpyAsync(part.data(), c->bbox_part.p, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                            c->st));
      CK(c, cudaMemcpyAsync(&fl, c->flags.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->st));
      CK(c, cudaStreamSynchronize(c->st));
      if (fl) return fail(c, CTB_ERR_NONFINITE, "non-finite coordinate in xyz");
      for (int k = 0; k < 3; ++k) {
        lo[k] = INFINITY;
        hi[k] = -INFINITY;
      }
      c->norm2_lo = INFINITY;
      c->norm2_hi = 0.0;
      for (int b = 0; b < nblk; ++b) {
        for (int k = 0; k < 3; ++k) {
          lo[k] = std::min(lo[k], part[b * 8 + k]);
          hi[k] = std::max(hi[k], part[b * 8 + 4 + k]);
        }
        c->norm2_lo = std::min(c->norm2_lo, part[b * 8 + 3]);
        c->norm2_hi = std::max(c->norm2_hi, part[b * 8 + 7]);
      }
    }
    double ext = 0;
    c->bbox_volume = 1.0;
    for (int k = 0; k < 3; ++k) {
      ext = std::max(ext, hi[k] - lo[k]);
      c->bbox_volume *= std::max(hi[k] - lo[k], c->rmax);
    }
    if (!(ext > 0)) ext = c->rmax;
    // a power-of-two unit with the bounding cube spanning at most 2^31 - 1024
    // units: int32 differences never overflow, and a catalogue already on that
    // dyadic grid is represented exactly
    c->unit = std::ldexp(1.0, (int)std::ceil(std::log2(ext / (2147483648.0 - 1024.0))));
    while (ext / c->unit > 2147483648.0 - 1024.0) c->unit *= 2.0;
    for (int k = 0; k < 3; ++k) {
      c->origin[k] = lo[k];
      c->hi[k] = hi[k];
    }
    g.shift = 31;
    double rmax_u = c->rmax / c->unit;
    double ncd = std::ceil(2147483648.0 * cpr / rmax_u);
    nc = (uint32_t)std::max(1.0, std::min(ncd, 1024.0));
  }
  finish_geom(c, g, nc);
  c->g = g;
  r = upload_thresholds(c);
  if (r) return r;

  // buffers
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  CK(c, ensure(c, c->key0, nn * 4));
  CK(c, ensure(c, c->val0, nn * 4));
  CK(c, ensure(c, c->key1, nn * 4));
  CK(c, ensure(c, c->val1, nn * 4));
  CK(c, ensure(c, c->pts_in, nn * 16));
  CK(c, ensure(c, c->pts, nn * 16));
  CK(c, ensure(c, c->s2i, nn * 4));
  CK(c, ensure(c, c->i2s, nn * 4));
  CK(c, ensure(c, c->cell_start, ((size_t)g.ncells + 1) * 4));
  const size_t hw = sort_hist_words(n);
  CK(c, ensure(c, c->hist, hw * 4));
  CK(c, ensure(c, c->scan_tmp, std::max(scan_tmp_words(hw), scan_tmp_words((size_t)g.ncells + 1)) * 4));

  IngestOut io{P<uint32_t>(c->key0), P<uint32_t>(c->val0), P<uint4>(c->pts_in)};
  const double inv_unit = 1.0 / c->unit;
  CK(c, launch_ingest(dxyz, dw, n, c->periodic ? c->box : 0.0, c->origin, inv_unit, g, io,
                      P<uint32_t>(c->flags), c->st));
  CK(c, cudaEventRecord(c->ev[1], c->st));
  SortBufs sb{P<uint32_t>(c->key0), P<uint32_t>(c->val0), P<uint32_t>(c->key1), P<uint32_t>(c->val1),
              P<uint32_t>(c->hist), P<uint32_t>(c->scan_tmp)};
  bool in1 = false;
  CK(c, radix_sort(sb, n, bits_for(g.ncells), &in1, c->st));
  uint32_t* ks = in1 ? sb.k1 : sb.k0;
  uint32_t* vs = in1 ? sb.v1 : sb.v0;
  CK(c, launch_gather(vs, P<uint4>(c->pts_in), n, P<uint4>(c->pts), P<uint32_t>(c->s2i), P<uint32_t>(c->i2s),
                      c->st));
  CK(c, launch_cell_start(ks, n, g.ncells, P<uint32_t>(c->cell_start), P<uint32_t>(c->scan_tmp), c->st));
  CK(c, cudaEventRecord(c->ev[2], c->st));
  uint32_t fl[4] = {0, 0, 0, 0};
  CK(c, cudaMemcpyAsync(fl, c->flags.p, sizeof(fl), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  if (fl[0]) return fail(c, CTB_ERR_NONFINITE, "non-finite coordinate or weight");
  c->negw = fl[3] != 0;
  for (int k = 0; k < kStages; ++k) c->t_ms[k] = 0;
  c->t_ms[0] = elapsed(c->ev[0], c->ev[1]);
  c->t_ms[1] = elapsed(c->ev[1], c->ev[2]);
  c->n = n;
  return CTB_OK;
}

// ---------------------------------------------------------------------------
// pair multipoles + contraction over a primary list (prim == NULL: all points)
//
// Per chunk of primaries: count pairs per (primary, bin) -> read the chunk's
// total (one small device->host copy) -> exclusive scan -> fill the
// (primary, bin) neighbour lists -> accumulate a_lm per list -> contract.
// A chunk whose lists would not fit the list buffer is halved and recounted;
// the next chunk's size follows the observed pairs per primary.

struct PairPlan {
  int wpb, alm_blocks, stream_blocks, count_blocks;
  int64_t chunk_first;   // primaries in the first chunk (from the mean density)
  int64_t chunk_max;     // primaries per chunk at most
  uint64_t list_cap;     // neighbour-list entries per chunk at most
  uint64_t code_cap;     // candidate bin codes (bytes) per chunk at most
  double cand_first;     // candidates per primary assumed for the first chunk
  int nparts;            // pair-sum partial rows (blocks of k_pair_sums)
  int ncon;              // contraction partial rows (blocks of the contraction kernel in use)
};

// Bin-code buffer bound: one byte per candidate of a chunk, at most four per
// list entry of the list capacity.
constexpr uint64_t kCodeCap = 1ull << 34;

// Neighbours in range of a primary at the catalogue's mean density: the
// ball's share of the box (3-D), or the ring's share of the sphere's area.
double mean_neighbours(const ctb_ctx* c) {
  if (c->sphere) return (double)c->n * 0.5 * (std::cos(c->tmin) - std::cos(c->tmax));
  const double vol = c->periodic ? c->box * c->box * c->box : c->bbox_volume;
  const double ball = 4.0 / 3.0 * M_PI * (c->rmax * c->rmax * c->rmax - c->rmin * c->rmin * c->rmin);
  return vol > 0 ? (double)c->n * std::min(1.0, ball / vol) : 0.0;
}

int plan_pairs(ctb_ctx* c, int64_t np, PairPlan* pl) {
  int wpb = c->wpb > 0 ? c->wpb : 4;
  int bps = c->sphere ? am_blocks_per_sm(c->lmax, wpb) : alm_blocks_per_sm(c->Lk, wpb);
  int sbps = stream_blocks_per_sm(true, c->nbins, c->sphere != 0);
  int cbps = stream_blocks_per_sm(false, c->nbins, c->sphere != 0);
  if (bps < 1 || sbps < 1 || cbps < 1) return fail(c, CTB_ERR_CUDA, "pair kernels cannot be resident");
  pl->wpb = wpb;
  pl->alm_blocks = bps * c->nsm;
  pl->stream_blocks = sbps * c->nsm;
  pl->count_blocks = cbps * c->nsm;
  const size_t rowbytes = (size_t)c->nbins * c->lay.row * sizeof(float);
  int64_t chunk = c->chunk > 0 ? c->chunk : (int64_t)(((size_t)3 << 30) / rowbytes);
  pl->chunk_max = std::max<int64_t>(1, std::min<int64_t>(chunk, std::max<int64_t>(np, 1)));
  pl->list_cap = c->list_cap;
  pl->nparts = 2 * c->nsm;
  if (c->precision == CTB_PREC_FP32) {
    // one wave of the FP32 contraction's resident blocks
    const int cb = contract_fp32_blocks_per_sm(c->nbins, c->lmax, c->lay.row, c->sphere);
    if (cb < 1) return fail(c, CTB_ERR_CUDA, "the contraction kernel cannot be resident");
    pl->ncon = cb * c->nsm;
  } else {
    pl->ncon = 2 * c->nsm;
  }
  // first chunk from the mean density, with a margin for clustering; later
  // chunks follow the measured pairs per primary
  const double est = 2.0 * mean_neighbours(c) + 64.0;
  // candidates (points of the scanned cell rows) run about 1.3-1.5x the pairs
  pl->code_cap = std::min<uint64_t>(kCodeCap, 4 * pl->list_cap);
  pl->cand_first = 1.5 * est;
  const double first = std::min(0.9 * (double)pl->list_cap / est, 0.9 * (double)pl->code_cap / pl->cand_first);
  pl->chunk_first = std::max<int64_t>(1, std::min<int64_t>(pl->chunk_max, (int64_t)first));
  return CTB_OK;
}

// M rows (slot layout) -> [m][nbins][(lmax+1)^2] in the l*l+l+m order
__global__ void k_unpack_alm(const float* __restrict__ M, int64_t m, int nbins, int row, const int* __restrict__ slot,
                             int nc, float* __restrict__ out) {
  const int64_t total = m * nbins * nc;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(o % nc);
    const int64_t pb = o / nc;
    out[o] = M[pb * row + slot[c]];
  }
}

struct ChunkEv {
  cudaEvent_t e[6];
};

// Contraction of rows [off, off + cnt) of the current chunk's M into the
// partials of segment `seg` (a catalogue of a batch; 0 otherwise).
int contract_piece(ctb_ctx* c, const PairPlan& pl, int64_t off, int64_t cnt, size_t seg, cudaEvent_t* ev_pack) {
  const int nb = c->nbins;
  const size_t zsz = (size_t)(c->lmax + 1) * nb * nb;
  const size_t rowsz = (size_t)nb * c->lay.row;
  const float* M = P<float>(c->M) + (size_t)off * rowsz;
  const float* wp = P<float>(c->wprim) + off;
  // two-point pair sums from the a_00 column (every precision)
  CK(c, launch_pair_sums(M, wp, cnt, nb, c->lay.row, c->lay.slot[0],
                         P<double>(c->pairsum) + seg * pl.nparts * nb, pl.nparts, c->st));
  if (c->precision != CTB_PREC_FP32) {
    const bool tf32 = c->precision == CTB_PREC_TF32;
    std::vector<unsigned long long> lb, kp;
    size_t elems = 0;
    tc_layout(tf32, cnt, nb, c->lmax, lb, kp, &elems);
    const size_t esz = tf32 ? 4 : 2;
    // the pack kernel writes every element, the K padding of each (l, bin)
    // included: ops[2] = H (the scaled coefficients, BF16 hi or TF32), ops[3]
    // = 2 lo (BF16 only), ops[0] = sign(w) H when some weight is negative
    const bool signed_a = c->negw;
    for (int k = 0; k < 4; ++k) {
      if (k == 1 || (k == 3 && tf32) || (k == 0 && !signed_a)) continue;
      CK(c, ensure(c, c->ops[k], elems * esz));
    }
    CK(c, ensure(c, c->lbase_d, lb.size() * 8));
    CK(c, ensure(c, c->kp_d, kp.size() * 8));
    CK(c, cudaMemcpyAsync(c->lbase_d.p, lb.data(), lb.size() * 8, cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemcpyAsync(c->kp_d.p, kp.data(), kp.size() * 8, cudaMemcpyHostToDevice, c->st));
    void* opa = signed_a ? c->ops[0].p : c->ops[2].p;
    CK(c, launch_pack(tf32, M, wp, cnt, nb, c->lay.row, c->lmax, P<int>(c->slot), P<unsigned long long>(c->lbase_d),
                      P<unsigned long long>(c->kp_d), signed_a ? c->ops[0].p : nullptr, c->ops[2].p, c->ops[3].p,
                      P<unsigned int>(c->flags) + 1, c->st));
    CK(c, cudaEventRecord(*ev_pack, c->st));
    CK(c, launch_contract_tc(tf32, cnt, nb, c->lmax, lb.data(), kp.data(), opa, c->ops[2].p, c->ops[3].p,
                             P<double>(c->partial_tc) + seg * pl.ncon * zsz, pl.ncon, P<unsigned int>(c->flags) + 1,
                             c->inject == CTB_INJECT_STALL, c->st));
    // the host vectors lb / kp back the copies above: wait before releasing them
    CK(c, cudaStreamSynchronize(c->st));
  } else {
    ContractArgs ca{};
    ca.M = M;
    ca.wprim = wp;
    ca.np = cnt;
    ca.nbins = nb;
    ca.lmax = c->lmax;
    ca.row = c->lay.row;
    ca.slot = P<int>(c->slot);
    ca.partial = P<double>(c->partial) + seg * pl.ncon * zsz;
    ca.part0 = 0;
    ca.sphere = c->sphere;
    CK(c, launch_contract_fp32(ca, pl.ncon, c->st));
  }
  return CTB_OK;
}

int run_pairs(ctb_ctx* c, const uint32_t* dprim, int64_t np, bool contract, const PairPlan& pl,
              float* alm_dev_out, uint64_t* npairs_out, const std::vector<int64_t>* seg_end = nullptr) {
  const int nb = c->nbins;
  CK(c, ensure(c, c->counts, (size_t)pl.chunk_max * nb * 4));
  CK(c, ensure(c, c->offsets, (size_t)pl.chunk_max * nb * 4));
  CK(c, ensure(c, c->scan_tmp2, scan_tmp_words((size_t)pl.chunk_max * nb) * 4));
  CK(c, ensure(c, c->M, (size_t)pl.chunk_max * nb * c->lay.row * sizeof(float)));
  CK(c, ensure(c, c->wprim, (size_t)pl.chunk_max * sizeof(float)));
  CK(c, ensure(c, c->counters, 64));
  CK(c, ensure(c, c->code_base, (size_t)pl.chunk_max * row_blocks(c->g) * sizeof(unsigned long long)));
  unsigned long long* work = P<unsigned long long>(c->counters);
  unsigned long long* total = work + 1;
  unsigned long long* code_total = work + 2;
  StreamArgs sa{};
  sa.pts = P<uint4>(c->pts);
  sa.cell_start = P<uint32_t>(c->cell_start);
  sa.prim = dprim;
  sa.thr = P<unsigned long long>(c->thr);
  sa.counts = P<uint32_t>(c->counts);
  sa.offsets = P<uint32_t>(c->offsets);
  sa.wprim = P<float>(c->wprim);
  sa.wsub = c->wsub;
  sa.work = work;
  sa.total = total;
  sa.keys = c->batch_keys;
  sa.code_total = code_total;
  sa.code_base = P<unsigned long long>(c->code_base);
  sa.g = c->g;
  AlmArgs aa{};
  aa.pts = P<uint4>(c->pts);
  aa.prim = dprim;
  aa.counts = P<uint32_t>(c->counts);
  aa.offsets = P<uint32_t>(c->offsets);
  aa.M = P<float>(c->M);
  aa.conv = P<int2>(c->conv);
  aa.work = work;
  aa.nbins = nb;
  aa.row = c->lay.row;
  std::memcpy(aa.beta, c->beta, sizeof(aa.beta));
  for (int k = 0; k < 3; ++k) aa.sph_origin[k] = (float)c->origin[k];
  aa.sph_unit = (float)c->unit;
  double t_stream = 0, t_alm = 0, t_con = 0, t_pack = 0;
  uint64_t pairs = 0, chunks = 0;
  int64_t C = pl.chunk_first;
  double cand_per = pl.cand_first;  // candidates per primary (estimate, then measured)
  size_t codes_need = 0;            // bytes the last count of this chunk asked for
  int64_t c0 = 0;
  // [0] count start [1] count end [2] fill end [3] alm end [4] contraction end [5] pack end
  cudaEvent_t* ev = c->ev + 2;
  while (c0 < np) {
    const int64_t cnt = std::min(C, np - c0);
    sa.prim_begin = aa.prim_begin = c0;
    sa.prim_count = aa.prim_count = cnt;
    // bin codes of this chunk: the estimate, or what its last count asked for
    const size_t codes_want = std::max<size_t>(
        codes_need, (size_t)std::min<double>((double)pl.code_cap, 1.05 * cand_per * (double)cnt + 256.0));
    CK(c, ensure(c, c->codes, codes_want));
    sa.codes = P<uint8_t>(c->codes);
    sa.code_cap = c->codes.bytes;
    CK(c, cudaMemsetAsync(work, 0, 24, c->st));
    CK(c, cudaEventRecord(ev[0], c->st));
    sa.lists = nullptr;
    CK(c, launch_stream(sa, false, pl.count_blocks, c->st));
    CK(c, cudaEventRecord(ev[1], c->st));
    unsigned long long tc[2] = {0, 0};  // pairs, candidates
    CK(c, cudaMemcpyAsync(tc, total, sizeof(tc), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    t_stream += elapsed(ev[0], ev[1]);
    const unsigned long long tot = tc[0], ctot = tc[1];
    if (tot > pl.list_cap || ctot > pl.code_cap) {
      if (cnt > 1) {
        C = std::max<int64_t>(1, cnt / 2);
        codes_need = 0;
        continue;
      }
      return fail(c, CTB_ERR_OOM, "one primary has more neighbours than the list buffers hold");
    }
    if (ctot > c->codes.bytes) {
      // the codes did not fit: grow the buffer and count this chunk again
      codes_need = (size_t)ctot;
      continue;
    }
    codes_need = 0;
    CK(c, ensure(c, c->lists, std::max<size_t>((size_t)tot, 1) * 4 + kListSlackBytes));
    CK(c, exclusive_scan_u32(P<uint32_t>(c->counts), P<uint32_t>(c->offsets), (size_t)cnt * nb,
                             P<uint32_t>(c->scan_tmp2), c->st));
    sa.lists = P<uint32_t>(c->lists);
    aa.lists = P<uint32_t>(c->lists);
    CK(c, cudaMemsetAsync(work, 0, 8, c->st));
    CK(c, launch_stream(sa, true, pl.stream_blocks, c->st));
    CK(c, cudaEventRecord(ev[2], c->st));
    CK(c, cudaMemsetAsync(work, 0, 8, c->st));
    if (c->sphere)
      CK(c, launch_am(aa, c->lmax, pl.wpb, pl.alm_blocks, c->st));
    else
      CK(c, launch_alm(aa, c->Lk, pl.wpb, c->nsm, c->st));
    CK(c, cudaEventRecord(ev[3], c->st));
    if (contract) {
      // split the chunk at catalogue boundaries (a batch): each piece adds to its catalogue's partials
      int64_t p0 = c0;
      while (p0 < c0 + cnt) {
        size_t seg = 0;
        int64_t p1 = c0 + cnt;
        if (seg_end) {
          seg = (size_t)(std::upper_bound(seg_end->begin(), seg_end->end(), p0) - seg_end->begin());
          p1 = std::min(p1, (*seg_end)[seg]);
        }
        int r = contract_piece(c, pl, p0 - c0, p1 - p0, seg, &ev[5]);
        if (r) return r;
        p0 = p1;
      }
    }
    if (alm_dev_out) {
      const int ncf = c->sphere ? 2 * c->lmax + 1 : (c->lmax + 1) * (c->lmax + 1);
      const size_t outsz = (size_t)cnt * nb * ncf;
      int blocks = (int)std::min<size_t>((outsz + 255) / 256, 65535);
      k_unpack_alm<<<blocks, 256, 0, c->st>>>(P<float>(c->M), cnt, nb, c->lay.row, P<int>(c->slot), ncf,
                                              alm_dev_out + (size_t)c0 * nb * ncf);
      ++g_launches;
      CK(c, cudaGetLastError());
    }
    CK(c, cudaEventRecord(ev[4], c->st));
    CK(c, cudaEventSynchronize(ev[4]));
    t_stream += elapsed(ev[1], ev[2]);
    t_alm += elapsed(ev[2], ev[3]);
    if (contract && c->precision != CTB_PREC_FP32 && !seg_end) {
      t_pack += elapsed(ev[3], ev[5]);
      t_con += elapsed(ev[5], ev[4]);
    } else {
      t_con += elapsed(ev[3], ev[4]);
    }
    pairs += tot;
    ++chunks;
    c0 += cnt;
    // next chunk: fill about 90 % of the list and code buffers at the observed density
    const double per = cnt > 0 ? (double)tot / (double)cnt : 0.0;
    if (cnt > 0) cand_per = std::max(1.0, (double)ctot / (double)cnt);
    double nxt = per > 0 ? 0.9 * (double)pl.list_cap / per : (double)pl.chunk_max;
    nxt = std::min(nxt, 0.9 * (double)pl.code_cap / cand_per);
    if (seg_end && cnt > 0 && c0 < np) {
      // a batch: the catalogues differ in size, so the pairs of a primary
      // scale with its catalogue's size.  Learn pairs and candidates per
      // primary per catalogue point from this chunk, and walk the next
      // catalogues until the predicted pairs fill the buffers.
      double pts = 0.0;  // sum over this chunk's primaries of their catalogue's size
      for (size_t sg = 0; sg < seg_end->size(); ++sg) {
        const int64_t s0 = sg ? (*seg_end)[sg - 1] : 0, s1 = (*seg_end)[sg];
        const int64_t lo = std::max(s0, c0 - cnt), hi = std::min(s1, c0);
        if (hi > lo) pts += (double)(hi - lo) * (double)(s1 - s0);
      }
      if (pts > 0) {
        const double rp = (double)tot / pts, rc = (double)ctot / pts;
        double bp = 0.9 * (double)pl.list_cap, bc = 0.9 * (double)pl.code_cap;
        int64_t take = 0;
        for (size_t sg = 0; sg < seg_end->size(); ++sg) {
          const int64_t s0 = sg ? (*seg_end)[sg - 1] : 0, s1 = (*seg_end)[sg];
          if (s1 <= c0) continue;
          const int64_t avail = s1 - std::max(s0, c0);
          const double pp = std::max(rp * (double)(s1 - s0), 1e-9), pc = std::max(rc * (double)(s1 - s0), 1e-9);
          const int64_t fit = (int64_t)std::min({(double)avail, bp / pp, bc / pc});
          take += fit;
          bp -= (double)fit * pp;
          bc -= (double)fit * pc;
          if (fit < avail) break;
        }
        nxt = (double)take;
      }
    }
    C = std::max<int64_t>(1, std::min<int64_t>((int64_t)nxt, pl.chunk_max));
  }
  c->t_ms[2] = t_stream + t_alm;
  c->t_ms[3] = t_pack;
  c->t_ms[4] = t_con;
  c->t_ms[6] = t_stream;
  c->t_ms[7] = t_alm;
  c->nchunks = chunks;
  *npairs_out = pairs;
  return CTB_OK;
}

int compute_impl(ctb_ctx* c, const uint32_t* dprim, int64_t np, double* zeta_out) {
  if (c->n < 0) return fail(c, CTB_ERR_STATE, "no catalogue: call ctb_set_points first");
  if (!zeta_out) return fail(c, CTB_ERR_ARG, "zeta_out is NULL");
  CK(c, cudaSetDevice(c->dev));
  int r = ensure_tables(c);
  if (r) return r;
  PairPlan pl{};
  r = plan_pairs(c, np, &pl);
  if (r) return r;
  const size_t zsz = (size_t)(c->lmax + 1) * c->nbins * c->nbins;
  CK(c, ensure(c, c->partial, (size_t)pl.ncon * zsz * sizeof(double)));
  CK(c, ensure(c, c->zeta, zsz * sizeof(double)));
  CK(c, cudaMemsetAsync(c->partial.p, 0, (size_t)pl.ncon * zsz * sizeof(double), c->st));
  c->pairsum_segs = 0;
  CK(c, ensure(c, c->pairsum, (size_t)pl.nparts * c->nbins * sizeof(double)));
  CK(c, cudaMemsetAsync(c->pairsum.p, 0, (size_t)pl.nparts * c->nbins * sizeof(double), c->st));
  const bool tc = c->precision != CTB_PREC_FP32;
  if (tc) {
    CK(c, ensure(c, c->partial_tc, (size_t)pl.ncon * zsz * sizeof(double)));
    CK(c, cudaMemsetAsync(c->partial_tc.p, 0, (size_t)pl.ncon * zsz * sizeof(double), c->st));
    CK(c, cudaMemsetAsync(P<unsigned int>(c->flags) + 1, 0, 4, c->st));
  }
  for (int k = 2; k < kStages; ++k) c->t_ms[k] = 0;  // [0], [1]: the last ctb_set_points
  uint64_t pairs = 0;
  r = run_pairs(c, dprim, np, true, pl, nullptr, &pairs);
  if (r) return r;
  const int evs = 2 + 8;
  CK(c, cudaEventRecord(c->ev[evs], c->st));
  if (tc)
    CK(c, launch_finalize_tc(P<double>(c->partial_tc), c->lmax, pl.ncon, c->nbins, P<double>(c->zeta), c->st));
  else
    CK(c, launch_finalize(P<double>(c->partial), pl.ncon, c->lmax, c->nbins, P<double>(c->zeta), c->sphere != 0,
                          c->st));
  CK(c, cudaEventRecord(c->ev[evs + 1], c->st));
  const bool dev_out = is_device_ptr(zeta_out);
  CK(c, cudaMemcpyAsync(zeta_out, c->zeta.p, zsz * sizeof(double),
                        dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
  unsigned int tc_err = 0;
  if (tc) CK(c, cudaMemcpyAsync(&tc_err, P<unsigned int>(c->flags) + 1, 4, cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  c->npairs = pairs;
  c->t_ms[5] = elapsed(c->ev[evs], c->ev[evs + 1]);
  if (tc_err) return fail(c, CTB_ERR_TIMEOUT, "tensor-core contraction: a bounded wait timed out");
  c->pairsum_segs = 1;
  c->pairsum_parts = pl.nparts;
  return CTB_OK;
}

// ---------------------------------------------------------------------------
// batch: k catalogues in one sorted grid (cell key = catalogue * cells + cell),
// one chunked pair pipeline over all primaries, contraction pieces split at
// catalogue boundaries into per-catalogue FP64 partials

int batch_impl(ctb_ctx* c, const double* const* xyz, const double* const* w, const int64_t* n, int k,
               double* zeta_out) {
  if (k < 1 || !xyz || !n || !zeta_out) return fail(c, CTB_ERR_ARG, "batch: k < 1 or NULL argument");
  if (!c->periodic || c->sphere) return fail(c, CTB_ERR_UNSUPPORTED, "batch mode needs a periodic box");
  std::vector<int64_t> cum(k + 1, 0);
  int64_t nmax = 0;
  for (int i = 0; i < k; ++i) {
    if (n[i] < 0) return fail(c, CTB_ERR_ARG, "batch: negative catalogue size");
    if (n[i] > 0 && !xyz[i]) return fail(c, CTB_ERR_ARG, "batch: NULL xyz with n > 0");
    cum[i + 1] = cum[i] + n[i];
    nmax = std::max(nmax, n[i]);
  }
  const int64_t N = cum[k];
  if (N >= (int64_t)1 << 31) return fail(c, CTB_ERR_ARG, "batch: more than 2^31 points in total");
  CK(c, cudaSetDevice(c->dev));
  int r = ensure_events(c);
  if (r) return r;
  r = ensure_tables(c);
  if (r) return r;
  c->n = -1;
  c->batch_keys = nullptr;
  c->batch_grid = false;
  // grid of one periodic catalogue
  const int cpr = grid_cells_per_rmax(c);
  Geom g{};
  g.periodic = 1;
  g.nbins = c->nbins;
  g.lmax = c->lmax;
  g.shift = 32;
  c->unit = std::ldexp(c->box, -32);
  const uint32_t nc = (uint32_t)std::max(1.0, std::min(std::floor(c->box * cpr / c->rmax), 1024.0));
  finish_geom(c, g, nc);
  c->g = g;
  if ((uint64_t)k * g.ncells >= ((uint64_t)1 << 32) - 1)
    return fail(c, CTB_ERR_ARG, "batch: catalogues x grid cells exceed 2^32 keys");
  r = upload_thresholds(c);
  if (r) return r;
  const size_t nn = (size_t)std::max<int64_t>(N, 1);
  CK(c, ensure(c, c->xyz_stage, nn * 3 * sizeof(double)));
  CK(c, ensure(c, c->w_stage, nn * sizeof(double)));
  CK(c, ensure(c, c->key0, nn * 4));
  CK(c, ensure(c, c->val0, nn * 4));
  CK(c, ensure(c, c->key1, nn * 4));
  CK(c, ensure(c, c->val1, nn * 4));
  CK(c, ensure(c, c->pts_in, nn * 16));
  CK(c, ensure(c, c->pts, nn * 16));
  CK(c, ensure(c, c->s2i, nn * 4));
  CK(c, ensure(c, c->i2s, nn * 4));
  const uint64_t cells_all = (uint64_t)k * g.ncells;
  CK(c, ensure(c, c->cell_start, (size_t)(cells_all + 1) * 4));
  const size_t hw = sort_hist_words(N);
  CK(c, ensure(c, c->hist, hw * 4));
  CK(c, ensure(c, c->scan_tmp, std::max(scan_tmp_words(hw), scan_tmp_words((size_t)cells_all + 1)) * 4));
  CK(c, ensure(c, c->flags, 64));
  CK(c, cudaMemsetAsync(c->flags.p, 0, 64, c->st));
  CK(c, cudaEventRecord(c->ev[0], c->st));
  for (int i = 0; i < k; ++i) {
    if (n[i] == 0) continue;
    const double* dx = xyz[i];
    if (!is_device_ptr(dx)) {
      CK(c, cudaMemcpyAsync(P<double>(c->xyz_stage) + 3 * cum[i], dx, (size_t)n[i] * 3 * sizeof(double),
                            cudaMemcpyHostToDevice, c->st));
      dx = P<double>(c->xyz_stage) + 3 * cum[i];
    }
    const double* dw = (w && w[i]) ? w[i] : nullptr;
    if (dw && !is_device_ptr(dw)) {
      CK(c, cudaMemcpyAsync(P<double>(c->w_stage) + cum[i], dw, (size_t)n[i] * sizeof(double),
                            cudaMemcpyHostToDevice, c->st));
      dw = P<double>(c->w_stage) + cum[i];
    }
    IngestOut io{P<uint32_t>(c->key0) + cum[i], P<uint32_t>(c->val0) + cum[i], P<uint4>(c->pts_in) + cum[i]};
    CK(c, launch_ingest(dx, dw, n[i], c->box, nullptr, 1.0 / c->unit, g, io, P<uint32_t>(c->flags), c->st,
                        (uint32_t)(i * g.ncells), (uint32_t)cum[i]));
  }
  CK(c, cudaEventRecord(c->ev[1], c->st));
  SortBufs sb{P<uint32_t>(c->key0), P<uint32_t>(c->val0), P<uint32_t>(c->key1), P<uint32_t>(c->val1),
              P<uint32_t>(c->hist), P<uint32_t>(c->scan_tmp)};
  bool in1 = false;
  int bits = 0;
  while (bits < 32 && ((uint64_t)1 << bits) < cells_all) ++bits;
  CK(c, radix_sort(sb, N, bits, &in1, c->st));
  uint32_t* ks = in1 ? sb.k1 : sb.k0;
  uint32_t* vs = in1 ? sb.v1 : sb.v0;
  CK(c, launch_gather(vs, P<uint4>(c->pts_in), N, P<uint4>(c->pts), P<uint32_t>(c->s2i), P<uint32_t>(c->i2s), c->st));
  CK(c, launch_cell_start(ks, N, (uint32_t)cells_all, P<uint32_t>(c->cell_start), P<uint32_t>(c->scan_tmp), c->st));
  CK(c, cudaEventRecord(c->ev[2], c->st));
  uint32_t fl = 0;
  uint32_t fl3 = 0;
  CK(c, cudaMemcpyAsync(&fl, c->flags.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaMemcpyAsync(&fl3, P<uint32_t>(c->flags) + 3, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  if (fl) return fail(c, CTB_ERR_NONFINITE, "batch: non-finite coordinate or weight");
  c->negw = fl3 != 0;
  const double t_ingest = elapsed(c->ev[0], c->ev[1]), t_sort = elapsed(c->ev[1], c->ev[2]);
  // pair pipeline over all primaries; densities planned from the largest catalogue
  c->batch_keys = ks;
  c->n = nmax;
  PairPlan pl{};
  r = plan_pairs(c, N, &pl);
  c->n = -1;
  if (r) {
    c->batch_keys = nullptr;
    return r;
  }
  const size_t zsz = (size_t)(c->lmax + 1) * c->nbins * c->nbins;
  const size_t budget = (size_t)8 << 30;  // FP64 partials: k catalogues x ncon rows (one wave of the contraction)
  pl.ncon = (int)std::max<size_t>(8, std::min<size_t>((size_t)pl.ncon, budget / ((size_t)k * zsz * 8)));
  const bool tc = c->precision != CTB_PREC_FP32;
  Buf& part = tc ? c->partial_tc : c->partial;
  CK(c, ensure(c, part, (size_t)k * pl.ncon * zsz * sizeof(double)));
  CK(c, cudaMemsetAsync(part.p, 0, (size_t)k * pl.ncon * zsz * sizeof(double), c->st));
  if (tc) CK(c, cudaMemsetAsync(P<unsigned int>(c->flags) + 1, 0, 4, c->st));
  c->pairsum_segs = 0;
  CK(c, ensure(c, c->pairsum, (size_t)k * pl.nparts * c->nbins * sizeof(double)));
  CK(c, cudaMemsetAsync(c->pairsum.p, 0, (size_t)k * pl.nparts * c->nbins * sizeof(double), c->st));
  CK(c, ensure(c, c->zeta, (size_t)k * zsz * sizeof(double)));
  for (int i = 0; i < kStages; ++i) c->t_ms[i] = 0;
  std::vector<int64_t> seg_end(cum.begin() + 1, cum.end());
  uint64_t pairs = 0;
  r = run_pairs(c, nullptr, N, true, pl, nullptr, &pairs, &seg_end);
  c->batch_keys = nullptr;
  if (r) return r;
  CK(c, cudaEventRecord(c->ev[10], c->st));
  for (int i = 0; i < k; ++i) {
    const double* pi = P<double>(part) + (size_t)i * pl.ncon * zsz;
    double* zi = P<double>(c->zeta) + (size_t)i * zsz;
    if (tc)
      CK(c, launch_finalize_tc(pi, c->lmax, pl.ncon, c->nbins, zi, c->st));
    else
      CK(c, launch_finalize(pi, pl.ncon, c->lmax, c->nbins, zi, c->sphere != 0, c->st));
  }
  CK(c, cudaEventRecord(c->ev[11], c->st));
  const bool dev_out = is_device_ptr(zeta_out);
  CK(c, cudaMemcpyAsync(zeta_out, c->zeta.p, (size_t)k * zsz * sizeof(double),
                        dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
  unsigned int tc_err = 0;
  if (tc) CK(c, cudaMemcpyAsync(&tc_err, P<unsigned int>(c->flags) + 1, 4, cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  c->npairs = pairs;
  c->t_ms[0] = t_ingest;
  c->t_ms[1] = t_sort;
  c->t_ms[5] = elapsed(c->ev[10], c->ev[11]);
  if (tc_err) return fail(c, CTB_ERR_TIMEOUT, "tensor-core contraction: a bounded wait timed out");
  c->pairsum_segs = k;
  c->pairsum_parts = pl.nparts;
  c->batch_grid = true;
  return CTB_OK;
}

// catalogue indices (int64, host or device) -> sorted positions (uint32, device)
__global__ void k_map_prim(const int64_t* __restrict__ idx, int64_t m, int64_t n, const uint32_t* __restrict__ i2s,
                           uint32_t* __restrict__ out, uint32_t* flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t v = idx[i];
    if (v < 0 || v >= n) {
      atomicOr(flags, 2u);
      out[i] = 0;
    } else {
      out[i] = i2s[v];
    }
  }
}

int map_primaries(ctb_ctx* c, const int64_t* idx, int64_t m) {
  if (m < 0) return fail(c, CTB_ERR_ARG, "negative primary count");
  if (m > 0 && !idx) return fail(c, CTB_ERR_ARG, "primary_idx is NULL");
  if (m == 0) return CTB_OK;
  const int64_t* didx = idx;
  if (!is_device_ptr(idx)) {
    for (int64_t i = 0; i < m; ++i)
      if (idx[i] < 0 || idx[i] >= c->n) return fail(c, CTB_ERR_ARG, "primary index out of range");
    CK(c, ensure(c, c->idx64, (size_t)m * 8));
    CK(c, cudaMemcpyAsync(c->idx64.p, idx, (size_t)m * 8, cudaMemcpyHostToDevice, c->st));
    didx = P<int64_t>(c->idx64);
  }
  CK(c, ensure(c, c->prim, (size_t)m * 4));
  CK(c, cudaMemsetAsync(c->flags.p, 0, 4, c->st));
  int blocks = (int)std::min<int64_t>((m + 255) / 256, 65535);
  k_map_prim<<<blocks, 256, 0, c->st>>>(didx, m, c->n, P<uint32_t>(c->i2s), P<uint32_t>(c->prim),
                                        P<uint32_t>(c->flags));
  ++g_launches;
  CK(c, cudaGetLastError());
  uint32_t fl = 0;
  CK(c, cudaMemcpyAsync(&fl, c->flags.p, 4, cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  if (fl & 2u) return fail(c, CTB_ERR_ARG, "primary index out of range");
  return CTB_OK;
}

// ---------------------------------------------------------------------------
// shared neighbour lists: group the points by pivot cell, then run the pair
// pipeline over the groups' representatives with the group weights

// key bits a radix sort needs for keys below ncells (<= 2^64, as a double)
int key_bits(double ncells) {
  int b = 0;
  while (b < 64 && std::ldexp(1.0, b) < ncells) ++b;
  return b;
}

int shared_impl(ctb_ctx* c, double h, double* zeta_out) {
  if (c->n < 0) return fail(c, CTB_ERR_STATE, "no catalogue: call ctb_set_points first");
  if (!zeta_out) return fail(c, CTB_ERR_ARG, "zeta_out is NULL");
  if (!std::isfinite(h) || h < 0) return fail(c, CTB_ERR_ARG, "pivot cell side must be >= 0 and finite");
  const int64_t n = c->n;
  if (h == 0 && n > 0) {
    // the mean separation of the catalogue
    if (c->sphere) {
      h = std::sqrt(4.0 * M_PI / (double)n);
    } else {
      const double vol = c->periodic ? c->box * c->box * c->box : c->bbox_volume;
      h = std::cbrt(vol / (double)n);
    }
  }
  CK(c, cudaSetDevice(c->dev));
  int64_t ng = 0;
  double t_group = 0;
  if (n > 0) {
    PivotGrid pg{};
    pg.unit = c->unit;
    pg.h = h;
    double ncell = 1.0;
    for (int k = 0; k < 3; ++k) {
      pg.origin[k] = c->origin[k];
      const double k0 = std::floor(c->origin[k] / h), k1 = std::floor(c->hi[k] / h);
      ncell *= k1 - k0 + 1.0;
      // cell indices stay well inside int64, each axis inside uint32, the product inside uint64
      if (!(std::fabs(k0) < 0x1p62 && std::fabs(k1) < 0x1p62 && k1 - k0 + 1.0 < 4294967296.0 &&
            ncell <= 18446744073709551616.0))
        return fail(c, CTB_ERR_ARG, "pivot cells: more than 2^64 over the catalogue's extent");
      pg.k0[k] = (long long)k0;
      pg.n[k] = (uint32_t)(k1 - k0 + 1.0);
    }
    const size_t nn = (size_t)n;
    CK(c, ensure(c, c->gk0, nn * 4));
    CK(c, ensure(c, c->gv0, nn * 4));
    CK(c, ensure(c, c->gk1, nn * 4));
    CK(c, ensure(c, c->gv1, nn * 4));
    CK(c, ensure(c, c->glo, nn * 4));
    CK(c, ensure(c, c->ghi, nn * 4));
    CK(c, ensure(c, c->ghead, nn * 4));
    CK(c, ensure(c, c->gid, nn * 4));
    CK(c, ensure(c, c->gscan, scan_tmp_words(nn) * 4));
    CK(c, ensure(c, c->gprim, nn * 4));
    CK(c, ensure(c, c->gw, nn * 4));
    CK(c, cudaEventRecord(c->ev[12], c->st));
    CK(c, launch_pivot_key(P<uint4>(c->pts), P<uint32_t>(c->i2s), n, pg, P<uint32_t>(c->glo), P<uint32_t>(c->ghi),
                           P<uint32_t>(c->gk0), P<uint32_t>(c->gv0), c->st));
    // stable LSD sort: low 32 key bits, then the high ones
    const int bits = key_bits(ncell);
    SortBufs sb{P<uint32_t>(c->gk0), P<uint32_t>(c->gv0), P<uint32_t>(c->gk1), P<uint32_t>(c->gv1),
                P<uint32_t>(c->hist), P<uint32_t>(c->scan_tmp)};
    bool in1 = false;
    CK(c, radix_sort(sb, n, std::min(bits, 32), &in1, c->st));
    const uint32_t* vs = in1 ? sb.v1 : sb.v0;
    if (bits > 32) {
      SortBufs hb{in1 ? sb.k0 : sb.k1, in1 ? sb.v1 : sb.v0, in1 ? sb.k1 : sb.k0, in1 ? sb.v0 : sb.v1, sb.hist,
                  sb.scan_tmp};
      CK(c, launch_gather_hi(hb.v0, P<uint32_t>(c->ghi), n, hb.k0, c->st));
      bool hin1 = false;
      CK(c, radix_sort(hb, n, bits - 32, &hin1, c->st));
      vs = hin1 ? hb.v1 : hb.v0;
    }
    CK(c, launch_group_heads(vs, P<uint32_t>(c->glo), P<uint32_t>(c->ghi), n, P<uint32_t>(c->ghead), c->st));
    CK(c, exclusive_scan_u32(P<uint32_t>(c->ghead), P<uint32_t>(c->gid), nn, P<uint32_t>(c->gscan), c->st));
    CK(c, launch_group_reduce(vs, P<uint32_t>(c->ghead), P<uint32_t>(c->gid), n, P<uint4>(c->pts),
                              P<uint32_t>(c->i2s), P<uint32_t>(c->gprim), P<float>(c->gw), c->st));
    CK(c, cudaEventRecord(c->ev[13], c->st));
    uint32_t last[2] = {0, 0};
    CK(c, cudaMemcpyAsync(&last[0], P<uint32_t>(c->gid) + (n - 1), 4, cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaMemcpyAsync(&last[1], P<uint32_t>(c->ghead) + (n - 1), 4, cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    ng = (int64_t)last[0] + (int64_t)last[1];
    t_group = elapsed(c->ev[12], c->ev[13]);
  }
  c->wsub = P<float>(c->gw);
  const int r = compute_impl(c, P<uint32_t>(c->gprim), ng, zeta_out);
  c->wsub = nullptr;
  if (r) return r;
  c->t_ms[8] = t_group;
  c->shared_h = h;
  c->ngroups = ng;
  return CTB_OK;
}

}  // namespace

// ===========================================================================
// C ABI

// ---------------------------------------------------------------------------
// Autotuner: the grid's cells per r_max (the cell size h = r_max / k).  Each
// candidate grids the catalogue, then the pair kernels (enumeration and
// accumulation, no contraction) run twice on the same sample of primaries:
// eight runs of consecutive primaries in cell order, spread over the
// catalogue, so their neighbourhoods are as local as in a full pass.  The
// second run is timed; the fastest candidate is kept for this context.

int autotune_grid(ctb_ctx* c, const double* xyz, const double* w, int64_t n) {
  static const int kCand[] = {3, 4, 6, 8, 12, 16};
  int best = 8;
  float best_ms = INFINITY;
  uint32_t prev_nc = 0;
  for (int cpr : kCand) {
    c->tuned_cpr = cpr;
    int r = load_points(c, xyz, w, n);
    if (r) return r;
    if (c->g.nc == prev_nc) continue;  // clamped to the same grid
    prev_nc = c->g.nc;
    r = ensure_tables(c);
    if (r) return r;
    // sample size: about 5e8 pairs at the mean density, 256..8192 primaries
    const double per = mean_neighbours(c) + 1.0;
    const int64_t S = std::min<int64_t>(n, std::max<int64_t>(256, std::min<int64_t>(8192, (int64_t)(5e8 / per))));
    std::vector<uint32_t> sample;
    sample.reserve((size_t)S);
    const int64_t runs = 8, len = std::max<int64_t>(1, S / runs);
    for (int64_t k = 0; k < runs && (int64_t)sample.size() < S; ++k) {
      const int64_t s0 = std::min<int64_t>(n - len, k * n / runs);
      for (int64_t q = 0; q < len && (int64_t)sample.size() < S; ++q) sample.push_back((uint32_t)(s0 + q));
    }
    const int64_t m = (int64_t)sample.size();
    CK(c, ensure(c, c->prim, (size_t)m * 4));
    CK(c, cudaMemcpyAsync(c->prim.p, sample.data(), (size_t)m * 4, cudaMemcpyHostToDevice, c->st));
    PairPlan pl{};
    r = plan_pairs(c, m, &pl);
    if (r) return r;
    uint64_t pairs = 0;
    for (int rep = 0; rep < 2; ++rep) {
      r = run_pairs(c, P<uint32_t>(c->prim), m, false, pl, nullptr, &pairs);
      if (r) return r;
    }
    const float ms = (float)(c->t_ms[6] + c->t_ms[7]);
    if (ms < best_ms) {
      best_ms = ms;
      best = cpr;
    }
  }
  c->tuned_cpr = best;
  return CTB_OK;
}

extern "C" {

const char* ctb_version(void) { return "ctb 0.1 (sm_103a)"; }

ctb_ctx* ctb_create_sphere(double theta_min, double theta_max, int nbins, int m_max) {
  if (!std::isfinite(theta_min) || !std::isfinite(theta_max) || !(theta_min >= 0.0) || !(theta_max > theta_min) ||
      theta_max > M_PI) {
    g_create_err = "need 0 <= theta_min < theta_max <= pi";
    return nullptr;
  }
  if (m_max < 0 || m_max > CTB_MMAX_CAP) {
    g_create_err = "m_max out of range [0, 16]";
    return nullptr;
  }
  // open space with the chord limits; bins and the estimator follow the sphere
  ctb_ctx* c = ctb_create(0.0, 2.0 * std::sin(0.5 * theta_min), 2.0 * std::sin(0.5 * theta_max), nbins, 0);
  if (!c) return nullptr;
  c->sphere = 1;
  c->lmax = m_max;
  c->tmin = theta_min;
  c->tmax = theta_max;
  return c;
}

ctb_ctx* ctb_create(double box, double r_min, double r_max, int nbins, int ell_max) {
  if (!std::isfinite(box) || !std::isfinite(r_min) || !std::isfinite(r_max)) {
    g_create_err = "non-finite argument";
    return nullptr;
  }
  if (!(r_min >= 0) || !(r_max > r_min)) {
    g_create_err = "need 0 <= r_min < r_max";
    return nullptr;
  }
  if (nbins < 1 || nbins > CTB_NBINS_CAP) {
    g_create_err = "nbins out of range [1, 64]";
    return nullptr;
  }
  if (ell_max < 0 || ell_max > CTB_LMAX_CAP) {
    g_create_err = "ell_max out of range [0, 20]";
    return nullptr;
  }
  if (box > 0 && r_max > 0.5 * box) {
    g_create_err = "periodic box needs r_max <= box/2";
    return nullptr;
  }
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    g_create_err = std::string("no usable CUDA device: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return nullptr;
  }
  ctb_ctx* c = new ctb_ctx();
  c->dev = dev;
  c->nsm = nsm;
  c->box = box;
  c->rmin = r_min;
  c->rmax = r_max;
  c->nbins = nbins;
  c->lmax = ell_max;
  c->periodic = box > 0 ? 1 : 0;
  return c;
}

void ctb_destroy(ctb_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->dev);
  release_all(c);
  cudaStreamSynchronize(c->st);
  if (c->ev_ready)
    for (auto& e : c->ev) cudaEventDestroy(e);
  cudaGetLastError();
  delete c;
}

const char* ctb_last_error(const ctb_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

int ctb_set_points(ctb_ctx* c, const double* xyz, const double* w, int64_t n) {
  if (!c) return CTB_ERR_ARG;
  if (c->autotune && c->cells_per_rmax == 0 && c->tuned_cpr == 0 && n > 1) {
    int r = autotune_grid(c, xyz, w, n);
    if (r) {
      c->tuned_cpr = 0;
      return r;
    }
  }
  const unsigned long long l0 = g_launches;
  int r = load_points(c, xyz, w, n);
  c->launches_points = g_launches - l0;
  return r;
}

int ctb_compute(ctb_ctx* c, double* zeta_out) {
  if (!c) return CTB_ERR_ARG;
  if (c->n < 0) return fail(c, CTB_ERR_STATE, "no catalogue: call ctb_set_points first");
  const unsigned long long l0 = g_launches;
  int r = compute_impl(c, nullptr, c->n, zeta_out);
  c->launches_compute = g_launches - l0;
  return r;
}

int ctb_compute_subset(ctb_ctx* c, const int64_t* primary_idx, int64_t m, double* zeta_out) {
  if (!c) return CTB_ERR_ARG;
  if (c->n < 0) return fail(c, CTB_ERR_STATE, "no catalogue: call ctb_set_points first");
  int r = map_primaries(c, primary_idx, m);
  if (r) return r;
  return compute_impl(c, m > 0 ? P<uint32_t>(c->prim) : nullptr, m, zeta_out);
}

int ctb_compute_shared(ctb_ctx* c, double pivot_cell, double* zeta_out) {
  if (!c) return CTB_ERR_ARG;
  const unsigned long long l0 = g_launches;
  int r = shared_impl(c, pivot_cell, zeta_out);
  c->launches_compute = g_launches - l0;
  return r;
}

int ctb_get_pivot_groups(ctb_ctx* c, double* pivot_cell, int64_t* groups) {
  if (!c || !pivot_cell || !groups) return CTB_ERR_ARG;
  if (c->ngroups < 0) return fail(c, CTB_ERR_STATE, "no ctb_compute_shared since the last ctb_set_points");
  *pivot_cell = c->shared_h;
  *groups = c->ngroups;
  return CTB_OK;
}

int ctb_get_alm(ctb_ctx* c, const int64_t* primary_idx, int64_t m, float* alm_out) {
  if (!c) return CTB_ERR_ARG;
  if (c->n < 0) return fail(c, CTB_ERR_STATE, "no catalogue: call ctb_set_points first");
  if (m > 0 && !alm_out) return fail(c, CTB_ERR_ARG, "alm_out is NULL");
  int r = map_primaries(c, primary_idx, m);
  if (r) return r;
  if (m == 0) return CTB_OK;
  r = ensure_tables(c);
  if (r) return r;
  PairPlan pl{};
  r = plan_pairs(c, m, &pl);
  if (r) return r;
  const int nc = c->sphere ? 2 * c->lmax + 1 : (c->lmax + 1) * (c->lmax + 1);
  const size_t outsz = (size_t)m * c->nbins * nc;
  const bool dev_out = is_device_ptr(alm_out);
  float* dst = alm_out;
  if (!dev_out) {
    CK(c, ensure(c, c->alm, outsz * 4));
    dst = P<float>(c->alm);
  }
  uint64_t pairs = 0;
  r = run_pairs(c, P<uint32_t>(c->prim), m, false, pl, dst, &pairs);
  if (r) return r;
  if (!dev_out) CK(c, cudaMemcpyAsync(alm_out, dst, outsz * 4, cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  c->npairs = pairs;
  return CTB_OK;
}

int ctb_compute_batch(ctb_ctx* c, const double* const* xyz, const double* const* w, const int64_t* n, int k,
                      double* zeta_out) {
  if (!c) return CTB_ERR_ARG;
  // the autotuner's grid: tuned once, on the batch's largest catalogue (the
  // one with the most work), and kept for the context
  if (c->autotune && c->cells_per_rmax == 0 && c->tuned_cpr == 0 && k >= 1 && xyz && n && c->periodic &&
      !c->sphere) {
    int imax = 0;
    for (int i = 1; i < k; ++i)
      if (n[i] > n[imax]) imax = i;
    if (n[imax] > 1 && xyz[imax]) {
      int r = autotune_grid(c, xyz[imax], (w && w[imax]) ? w[imax] : nullptr, n[imax]);
      if (r) {
        c->tuned_cpr = 0;
        return r;
      }
    }
  }
  const unsigned long long l0 = g_launches;
  int r = batch_impl(c, xyz, w, n, k, zeta_out);
  c->launches_points = 0;
  c->launches_compute = g_launches - l0;
  return r;
}

int ctb_set_option(ctb_ctx* c, int key, int64_t v) {
  if (!c) return CTB_ERR_ARG;
  switch (key) {
    case CTB_OPT_PRECISION:
      if (v != CTB_PREC_FP32 && v != CTB_PREC_BF16X3 && v != CTB_PREC_TF32)
        return fail(c, CTB_ERR_ARG, "unknown precision");
      if (c->sphere && v != CTB_PREC_FP32)
        return fail(c, CTB_ERR_UNSUPPORTED, "the sphere contraction runs in FP32 only");
      c->precision = (int)v;
      return CTB_OK;
    case CTB_OPT_CELLS_PER_RMAX:
      if (v < 0 || v > 64) return fail(c, CTB_ERR_ARG, "cells per r_max out of range [0, 64]");
      c->cells_per_rmax = (int)v;
      c->n = -1;  // grid changes: the catalogue must be reloaded
      return CTB_OK;
    case CTB_OPT_LIST_CAPACITY:
      if (v != 0 && (v < 4096 || v > ((int64_t)1 << 32)))
        return fail(c, CTB_ERR_ARG, "list capacity must be 0 or in [4096, 2^32]");
      c->list_cap = v == 0 ? (uint64_t)1 << 32 : (uint64_t)v;
      return CTB_OK;
    case CTB_OPT_WARPS_PER_BLOCK:
      // the pair kernels are compiled for blocks of at most 128 threads
      if (v < 0 || v > 4) return fail(c, CTB_ERR_ARG, "warps per block out of range [0, 4]");
      c->wpb = (int)v;
      return CTB_OK;
    case CTB_OPT_CHUNK_PRIMARIES:
      if (v != 0 && v < 1024) return fail(c, CTB_ERR_ARG, "chunk must be 0 or >= 1024");
      c->chunk = v;
      return CTB_OK;
    case CTB_OPT_FAULT_INJECT:
      if (v != 0 && v != CTB_INJECT_STALL && v != CTB_INJECT_ALLOC) return fail(c, CTB_ERR_ARG, "unknown fault");
      c->inject = (int)v;
      return CTB_OK;
    case CTB_OPT_AUTOTUNE:
      if (v != 0 && v != 1) return fail(c, CTB_ERR_ARG, "autotune must be 0 or 1");
      c->autotune = (int)v;
      c->tuned_cpr = 0;  // (re)tune on the next ctb_set_points
      return CTB_OK;
    case CTB_OPT_DETERMINISTIC:
      if (v != 0 && v != 1) return fail(c, CTB_ERR_ARG, "deterministic must be 0 or 1");
      c->deterministic = (int)v;
      return CTB_OK;
    default:
      return fail(c, CTB_ERR_ARG, "unknown option key");
  }
}

int ctb_set_stream(ctb_ctx* c, void* stream) {
  if (!c) return CTB_ERR_ARG;
  c->st = static_cast<cudaStream_t>(stream);
  return CTB_OK;
}

int ctb_set_allocator(ctb_ctx* c, void* (*alloc)(size_t, void*), void (*free_fn)(void*, void*), void* user) {
  if (!c) return CTB_ERR_ARG;
  if ((alloc == nullptr) != (free_fn == nullptr)) return fail(c, CTB_ERR_ARG, "alloc and free must both be set");
  cudaSetDevice(c->dev);
  release_all(c);
  cudaStreamSynchronize(c->st);
  c->alloc_fn = alloc;
  c->free_fn = free_fn;
  c->user = user;
  c->n = -1;
  return CTB_OK;
}

int ctb_get_timings(ctb_ctx* c, double* ms, int cap) {
  if (!c || (cap > 0 && !ms)) return CTB_ERR_ARG;
  int k = std::min(cap, kStages);
  for (int i = 0; i < k; ++i) ms[i] = c->t_ms[i];
  return k;
}

int ctb_get_launch_count(ctb_ctx* c, uint64_t* kernels) {
  if (!c || !kernels) return CTB_ERR_ARG;
  *kernels = c->launches_points + c->launches_compute;
  return CTB_OK;
}

int ctb_get_pair_count(ctb_ctx* c, uint64_t* pairs) {
  if (!c || !pairs) return CTB_ERR_ARG;
  *pairs = c->npairs;
  return CTB_OK;
}

int ctb_edge_correct(ctb_ctx* c, const double* zeta_nnn, const double* zeta_rrr, double* zeta_out) {
  if (!c) return CTB_ERR_ARG;
  if (!zeta_nnn || !zeta_rrr || !zeta_out) return fail(c, CTB_ERR_ARG, "NULL argument");
  if (c->sphere) return fail(c, CTB_ERR_UNSUPPORTED, "edge correction of the 3-D multipoles only");
  CK(c, cudaSetDevice(c->dev));
  const int n = c->lmax + 1, nb = c->nbins;
  const size_t zsz = (size_t)n * nb * nb;
  // the 3j table, then both inputs and the output in device memory (staged when on the host)
  std::vector<double> tj;
  make_threej_table(c->lmax, tj);
  CK(c, ensure(c, c->edge_tj, tj.size() * sizeof(double)));
  CK(c, ensure(c, c->edge_in, 3 * zsz * sizeof(double)));
  double* dn = P<double>(c->edge_in);
  double* dr = dn + zsz;
  double* dout = dr + zsz;
  CK(c, cudaMemcpyAsync(c->edge_tj.p, tj.data(), tj.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CK(c, cudaMemcpyAsync(dn, zeta_nnn, zsz * sizeof(double), cudaMemcpyDefault, c->st));
  CK(c, cudaMemcpyAsync(dr, zeta_rrr, zsz * sizeof(double), cudaMemcpyDefault, c->st));
  CK(c, launch_edge_correct(dn, dr, P<double>(c->edge_tj), c->lmax, nb, dout, c->st));
  CK(c, cudaMemcpyAsync(zeta_out, dout, zsz * sizeof(double), cudaMemcpyDefault, c->st));
  CK(c, cudaStreamSynchronize(c->st));  // the host table and host outputs are done with
  return CTB_OK;
}

int ctb_get_2pcf(ctb_ctx* c, double* out, int cap) {
  if (!c || !out) return CTB_ERR_ARG;
  if (c->pairsum_segs <= 0) return fail(c, CTB_ERR_STATE, "no zeta computed on this catalogue yet");
  const int nb = c->nbins, nseg = c->pairsum_segs, np = c->pairsum_parts;
  if ((int64_t)cap < (int64_t)nseg * nb) return fail(c, CTB_ERR_ARG, "out holds fewer than catalogues * nbins values");
  CK(c, cudaSetDevice(c->dev));
  std::vector<double> part((size_t)nseg * np * nb);
  CK(c, cudaMemcpyAsync(part.data(), c->pairsum.p, part.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  // a_00 = sum_j w_j / sqrt(4 pi); on the sphere a_0 = sum_j w_j
  const double s4pi = c->sphere ? 1.0 : std::sqrt(4.0 * M_PI);
  for (int k = 0; k < nseg; ++k)
    for (int b = 0; b < nb; ++b) {
      double s = 0.0;
      for (int p = 0; p < np; ++p) s += part[((size_t)k * np + p) * nb + b];
      out[(size_t)k * nb + b] = s4pi * s;
    }
  return nseg * nb;
}

int ctb_get_grid(ctb_ctx* c, int* cells_per_rmax, int* cells_per_axis) {
  if (!c || !cells_per_rmax || !cells_per_axis) return CTB_ERR_ARG;
  if (c->n < 0 && !c->batch_grid) return fail(c, CTB_ERR_STATE, "no catalogue: call ctb_set_points first");
  *cells_per_rmax = grid_cells_per_rmax(c);
  *cells_per_axis = (int)c->g.nc;
  return CTB_OK;
}

int ctb_get_chunk_count(ctb_ctx* c, uint64_t* chunks) {
  if (!c || !chunks) return CTB_ERR_ARG;
  *chunks = c->nchunks;
  return CTB_OK;
}

}  // extern "C"
