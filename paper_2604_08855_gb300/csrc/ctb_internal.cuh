// ctb_internal.cuh -- shared declarations of the libctb CUDA implementation.
//
// Point representation on the device (one uint4 per point, 16 B):
//   x, y, z : unsigned 32-bit fixed-point coordinates.  Periodic cube: the
//             side L maps onto 2^32 units, so the wrapped difference of two
//             coordinates read as int32 IS the minimum-image separation.
//             Open space: the bounding cube maps onto [0, 2^31) units, so a
//             difference never overflows int32.
//   w       : float32 weight bits.
// One unit is L / 2^32 (about 2.3e-7 for L = 1000), so quantisation moves a
// point by far less than float32 rounding of a separation does.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ctb.h"

namespace ctb {

constexpr int kLmaxCap = CTB_LMAX_CAP;
// bytes allocated past the last neighbour-list entry (read by L2 prefetches only)
constexpr size_t kListSlackBytes = 1024;
constexpr int kNbinsCap = CTB_NBINS_CAP;
constexpr int kWarp = 32;
// coefficients accumulated per pass of the pair kernel (register budget: a
// pass of more than 136 runs at 255 registers and 8 warps per SM, which
// measured faster at l_max 20 than one more pass at 168 registers and 12)
constexpr int kPassCap = 184;

// ---------------------------------------------------------------------------
// grid / estimator geometry shared by the kernels

// A row of cells (fixed y, z) is split this many times finer along x than
// across: a primary's scan of a row then starts and ends closer to its ball
// (at 6 cells per r_max, about 9 % fewer candidates) at no extra rows.
constexpr uint32_t kXSub = 8;

struct Geom {
  int periodic;        // 1: periodic cube, 0: open space
  int shift;           // 32 (periodic) or 31 (open): unit coordinates < 2^shift
  uint32_t nc;         // cells per axis across the rows (y, z)
  uint32_t ncx;        // cells along a row (x): nc times kXSub, or less for very fine grids
  uint32_t ncells;     // nc * nc * ncx
  int nbins;
  int lmax;            // requested ell_max
  float rlo2_u;        // r_min^2 in units^2, widened by 1e-5 (float pre-filter)
  float rhi2_u;        // r_max^2 in units^2, widened by 1e-5 (float pre-filter)
  float rmin_u;        // r_min in units
  float inv_dr_u;      // nbins / (r_max - r_min) in 1/units
  float rcell;         // r_max in cell units, padded by a small slack
  float cell_scale;    // nc / 2^shift : units -> cell units
  int general;         // 1: bin edges not linear in r (sphere: chords of linear angles)
  float half_unit;     // sphere: unit / 2, so that chord / 2 = r_units * half_unit
  float tmin;          // sphere: theta_min (radians)
  float inv_dt;        // sphere: nbins / (theta_max - theta_min)
  float shell_c[3];    // sphere: the origin of coordinates in cell units (x in x-cells)
  float shell_r2lo;    // sphere: (smallest |p|)^2 and (largest |p|)^2 of the catalogue in
  float shell_r2hi;    //   (y, z) cell units squared, padded: every point lies in that shell
};

// Rows of the neighbour scan: W x W x-rows of cells at (dy, dz) offsets
// off0 .. off0 + W - 1 around the primary's cell, or the whole periodic cube
// when that window would wrap onto itself.  The scan takes the rows in blocks
// of 32 (one per lane).
struct RowWindow {
  int W, off0;
  bool fullwin;
};
__host__ __device__ inline RowWindow row_window(const Geom& g) {
  const int K = (int)floorf(g.rcell) + 1;
  RowWindow w{2 * K + 1, -K, false};
  if (g.periodic && w.W >= (int)g.nc) {
    w.W = (int)g.nc;
    w.off0 = -(((int)g.nc - 1) / 2);
    w.fullwin = true;
  }
  return w;
}
__host__ __device__ inline int row_blocks(const Geom& g) {
  const RowWindow w = row_window(g);
  return (w.W * w.W + 31) / 32;
}

// ---------------------------------------------------------------------------
// real-harmonic coefficient layout of one pair-kernel configuration
//
// The pair kernel accumulates the (l, m) coefficients in passes over m ranges
// [m0, m1] (one pass when ell_max <= 10).  Each pass accumulates moments of
// its columns in one polynomial basis q_k(z), k = 0..L - m0: the Chebyshev
// T_k for the pass that starts at m = 0, and the monic recurrence
// polynomials of its first column, p^{m0}_{m0+k}, for the others.  Moment k
// of column m, sum_j w_j (x+iy)^m q_k(z_j), sits in the slot of (m + k, +-m);
// the flush turns moments into normalised a_lm by a fixed linear map.
//
// Slots of a pass: first the (+m, -m) pairs, for l = max(m0,1)..L and
// m = max(m0,1)..min(l, m1), each pair on an even slot (+m) and the odd slot
// after it (-m), so one paired FP32 instruction updates both; then, in the
// pass that holds m = 0, the singles (l, 0) for l = 0..L.  Pass p occupies
// slots [base_p, base_p + ncp_p) of a row, ncp_p the pass's coefficient
// count rounded up to a multiple of 32.

__host__ __device__ constexpr int coef_count(int L, int m0, int m1) {
  int s = 0;
  for (int m = m0; m <= m1 && m <= L; ++m) s += (L - m + 1) * (m == 0 ? 1 : 2);
  return s;
}

// Largest l_max whose whole coefficient set is one pass (Chebyshev basis).
constexpr int kSinglePassLmax = 10;
// Columns of the first pass when l_max > kSinglePassLmax: the Chebyshev
// moments lose float32 accuracy as m grows, so this pass stops at m = 2.
constexpr int kFirstPassM1 = 2;

// end column of the pass starting at m0 when every further pass holds at
// most `cap` coefficients
__host__ __device__ constexpr int pass_end(int L, int m0, int cap) {
  if (L <= kSinglePassLmax) return L;
  if (m0 == 0) return kFirstPassM1;
  int s = 0, m = m0;
  while (m <= L) {
    int c = (L - m + 1) * (m == 0 ? 1 : 2);
    if (s + c > cap && m > m0) break;
    s += c;
    ++m;
  }
  return m - 1;
}

__host__ __device__ constexpr int passes_with_cap(int L, int cap) {
  int n = 0;
  for (int m0 = 0; m0 <= L; m0 = pass_end(L, m0, cap) + 1) ++n;
  return n;
}

// The passes after the first are balanced: the smallest cap that keeps the
// pass count of filling each to kPassCap coefficients.
__host__ __device__ constexpr int pass_cap_all(int L) {
  const int target = passes_with_cap(L, kPassCap);
  int lo = 1, hi = kPassCap;
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (passes_with_cap(L, mid) <= target) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// accumulator slots of the m-range pass of the pair kernel for ell_max L that
// starts at column m0 (pass_end with this cap ends the pass where the
// balanced split does)
__host__ __device__ constexpr int pass_cap(int L, int m0) {
  return coef_count(L, m0, pass_end(L, m0, pass_cap_all(L)));
}

__host__ __device__ constexpr int round32(int v) { return (v + 31) / 32 * 32; }

// Flush conversion entries per slot of the pass starting at m0: a_lm of
// column m takes the moments of degrees l - m, l - m - 2, ... (p^m_l has
// the parity of its degree, and so does each basis polynomial).
__host__ __device__ constexpr int conv_entries(int L, int m0) { return (L - m0) / 2 + 1; }

// (+m, -m) pairs of the pass [m0, m1] with degree below l
__host__ __device__ constexpr int pairs_below(int l, int m0, int m1) {
  const int ms = m0 < 1 ? 1 : m0;
  int s = 0;
  for (int q = ms; q < l; ++q) {
    const int hi = q < m1 ? q : m1;
    if (hi >= ms) s += hi - ms + 1;
  }
  return s;
}

// slot of (l, m) inside the pass [m0, m1] of kernel L (requires
// m0 <= |m| <= min(l, m1) and l <= L)
__host__ __device__ constexpr int local_slot(int L, int l, int m, int m0, int m1) {
  const int ms = m0 < 1 ? 1 : m0;
  if (m == 0) return 2 * pairs_below(L + 1, m0, m1) + l;
  const int am = m < 0 ? -m : m;
  return 2 * (pairs_below(l, m0, m1) + (am - ms)) + (m < 0 ? 1 : 0);
}

// pair-kernel instantiation that serves a requested ell_max
__host__ __device__ constexpr int lmax_kernel(int lmax) {
  return lmax <= 10 ? lmax : (lmax + 1) / 2 * 2;
}

// Host-side description of the row layout for a kernel L.
struct Layout {
  int L;                         // kernel ell_max
  int npass;
  int m0[kLmaxCap + 1], m1[kLmaxCap + 1], base[kLmaxCap + 1], ncp[kLmaxCap + 1];
  int row;                       // floats per (primary, bin) row
  // slot of coefficient index l*l + l + m for l <= L
  int slot[(kLmaxCap + 1) * (kLmaxCap + 1)];
};
void make_layout(int L, Layout* out);

// kernels launched by this host thread (every launcher adds its launches)
extern thread_local unsigned long long g_launches;

// smallest integer T >= 0 with T * unit^2 >= edge^2, in exact arithmetic
// (api.cu); a pair whose squared separation in units^2 is T lies at or
// beyond `edge` exactly when T >= threshold.
unsigned long long sq_threshold(double edge, double unit);

// recurrence constants (pair_dispatch.cu)
void fill_beta(float* beta);   // beta_lm at [l*(kLmaxCap+1)+m]
double norm_lm(int l, int m);  // C_lm of the real orthonormal Y_l,m
// flush conversion table of kernel L: accumulator totals -> normalised a_lm
// (entries padded per pass to conv_entries(L, m0_p), entry-major; see AlmArgs::conv)
bool make_conversion(const Layout& lay, std::vector<int2>& tab);

// ---------------------------------------------------------------------------
// kernels and launchers (all asynchronous on `st`)

// grid.cu
struct IngestOut {
  uint32_t* key;    // cell key per point (input order)
  uint32_t* val;    // input index
  uint4* pts;       // fixed-point point per input index
};
// box > 0: periodic; else origin/inv_unit map into [0, 2^31).  key_base is
// added to every cell key (catalogue index * cells per catalogue in a batch),
// val_base to every input index.
cudaError_t launch_ingest(const double* xyz, const double* w, int64_t n, double box,
                          const double* origin3, double inv_unit, const Geom& g,
                          IngestOut out, uint32_t* d_flags, cudaStream_t st,
                          uint32_t key_base = 0, uint32_t val_base = 0);
cudaError_t launch_bbox(const double* xyz, int64_t n, double* d_part, int nblk,
                        uint32_t* d_flags, cudaStream_t st);
int bbox_blocks(int64_t n);

// radix sort of (key, val), key < 2^bits; returns the buffers holding the result
struct SortBufs {
  uint32_t *k0, *v0, *k1, *v1;
  uint32_t* hist;       // [256 * nblk]
  uint32_t* scan_tmp;   // scan workspace
};
int sort_blocks(int64_t n);
size_t sort_hist_words(int64_t n);
size_t scan_tmp_words(size_t len);
cudaError_t radix_sort(SortBufs& b, int64_t n, int bits, bool* result_in_1, cudaStream_t st);
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, size_t len,
                               uint32_t* tmp, cudaStream_t st);

cudaError_t launch_gather(const uint32_t* val_sorted, const uint4* pts_in, int64_t n,
                          uint4* pts_sorted, uint32_t* sorted_to_input,
                          uint32_t* input_to_sorted, cudaStream_t st);
// cell_start[c] = first sorted position with key >= c, c in [0, ncells];
// scan_tmp holds scan_tmp_words(ncells + 1) words
cudaError_t launch_cell_start(const uint32_t* key_sorted, int64_t n, uint32_t ncells, uint32_t* cell_start,
                              uint32_t* scan_tmp, cudaStream_t st);

// shared.cu -- pivot groups for shared neighbour lists
struct PivotGrid {
  double origin[3];  // stored coordinate = origin + u * unit
  double unit;
  double h;          // pivot cell side
  long long k0[3];   // floor(lo / h) per axis: the first cell
  uint32_t n[3];     // cells per axis (product <= 2^64)
};
// key_lo / key_hi: the 64-bit cell key of each point (catalogue order);
// sort_key: a copy of key_lo for the sort; val: the catalogue index
cudaError_t launch_pivot_key(const uint4* pts, const uint32_t* i2s, int64_t n, const PivotGrid& pg,
                             uint32_t* key_lo, uint32_t* key_hi, uint32_t* sort_key, uint32_t* val,
                             cudaStream_t st);
cudaError_t launch_gather_hi(const uint32_t* val, const uint32_t* key_hi, int64_t n, uint32_t* out,
                             cudaStream_t st);
cudaError_t launch_group_heads(const uint32_t* val_sorted, const uint32_t* key_lo, const uint32_t* key_hi,
                               int64_t n, uint32_t* head, cudaStream_t st);
cudaError_t launch_group_reduce(const uint32_t* val_sorted, const uint32_t* head, const uint32_t* gid, int64_t n,
                                const uint4* pts, const uint32_t* i2s, uint32_t* prim_out, float* w_out,
                                cudaStream_t st);

// stream.cu -- neighbour enumeration (count pass, then fill pass)
struct StreamArgs {
  const uint4* pts;               // sorted points
  const uint32_t* cell_start;     // [ncells + 1]
  const uint32_t* prim;           // sorted positions of the primaries (NULL: identity)
  int64_t prim_begin;             // first primary of this launch
  int64_t prim_count;             // primaries in this launch
  const unsigned long long* thr;  // [nbins+1] exact edges in units^2
  uint32_t* counts;               // [prim_count][nbins] pairs per (primary, bin)   (count pass)
  const uint32_t* offsets;        // [prim_count][nbins] list start per (primary, bin) (fill pass)
  uint32_t* lists;                // neighbour indices grouped by (primary, bin)      (fill pass)
  float* wprim;                   // [prim_count] primary weights                      (count pass)
  const float* wsub;              // weights replacing the primaries' own, indexed like prim (NULL: none)
  unsigned long long* work;       // work counter (zeroed before launch)
  unsigned long long* total;      // binned pairs of this launch (count pass, accumulated)
  const uint32_t* keys;           // sorted cell keys of a batch (catalogue = key / ncells), or NULL
  uint8_t* codes;                 // bin code per candidate (written: count, read: fill)
  unsigned long long code_cap;    // bytes of codes
  unsigned long long* code_total; // code bytes of this launch (count pass; the range allocator)
  unsigned long long* code_base;  // [prim_count][row_blocks] start of each row block's codes
  Geom g;
};
int stream_blocks_per_sm(bool fill, int nbins, bool general);
cudaError_t launch_stream(const StreamArgs& a, bool fill, int nblocks, cudaStream_t st);
constexpr int kStreamThreads = 256;

// pair.cuh -- harmonic accumulation over the (primary, bin) lists
struct AlmArgs {
  const uint4* pts;               // sorted points
  const uint32_t* prim;           // sorted positions of the primaries (NULL: identity)
  int64_t prim_begin;
  int64_t prim_count;
  const uint32_t* counts;         // [prim_count][nbins]
  const uint32_t* offsets;        // [prim_count][nbins]
  const uint32_t* lists;
  float* M;                       // [prim_count][nbins][row]
  const int2* conv;               // flush conversion, per pass p (at conv_pass_offset(L, p)): entry e of local
                                  //   slot s at [e * ncp_p + s] = (source local slot, coefficient bits)
  unsigned long long* work;
  int nbins;
  int row;
  float sph_origin[3];            // sphere mode: the points' position = origin + unit * (x, y, z)
  float sph_unit;
  float beta[(kLmaxCap + 1) * (kLmaxCap + 1)];  // recurrence beta_lm at [l*(kLmaxCap+1)+m]
};
int alm_blocks_per_sm(int lmax_kernel, int warps_per_block);
// sphere.cu: projected multipoles m = 0..mmax (mmax <= CTB_MMAX_CAP)
int am_blocks_per_sm(int mmax, int warps_per_block);
cudaError_t launch_am(const AlmArgs& a, int mmax, int warps_per_block, int nblocks, cudaStream_t st);
// one launch per m-pass, each sized from its own occupancy on nsm SMs
cudaError_t launch_alm(const AlmArgs& a, int lmax_kernel, int warps_per_block, int nsm, cudaStream_t st);

// contract.cu
struct ContractArgs {
  const float* M;          // [np][nbins][row]
  const float* wprim;      // [np]
  int64_t np;
  int nbins;
  int lmax;
  int row;
  const int* slot;         // device copy of Layout::slot
  double* partial;         // [nparts][(lmax+1)][nbins][nbins] (upper triangle used)
  int part0;               // first partial row this launch writes
  int sphere;              // 0: group l = components l^2 .. l^2+2l; 1: group m = {0} or {2m-1, 2m}
};
cudaError_t launch_contract_fp32(const ContractArgs& a, int nparts, cudaStream_t st);
int contract_fp32_blocks_per_sm(int nbins, int lmax, int row, int sphere);

// edge.cu
void make_threej_table(int lmax, std::vector<double>& t);  // (a b c; 0 0 0)^2, [a][b][c], a,b,c <= lmax
cudaError_t launch_edge_correct(const double* zn, const double* zr, const double* tj, int lmax, int nbins,
                                double* out, cudaStream_t st);
// partial[part][b] += sum over a fixed slice of the primaries of w_p * M[p][b][col]
cudaError_t launch_pair_sums(const float* M, const float* w, int64_t np, int nbins, int row, int col,
                             double* partial, int nparts, cudaStream_t st);
cudaError_t launch_finalize(const double* partial, int nparts, int lmax, int nbins, double* zeta, bool sphere,
                            cudaStream_t st);

// contract_tc.cu -- tcgen05 contraction (BF16 hi/lo split or TF32)
int tc_npad(int nbins);
void tc_layout(bool tf32, int64_t np, int nbins, int lmax, std::vector<unsigned long long>& lbase,
               std::vector<unsigned long long>& kp, size_t* elems);
// slot: the layout's slot of coefficient l*l+l+m (l <= lmax)
// outS (sign(w) times the scaled coefficients) may be NULL: no negative weights
cudaError_t launch_pack(bool tf32, const float* M, const float* wprim, int64_t np, int nbins, int row, int lmax,
                        const int* slot, const unsigned long long* lbase, const unsigned long long* kp, void* outS,
                        void* outH, void* outL, unsigned int* err, cudaStream_t st);
// opA = outS, or outH when there is no negative weight
cudaError_t launch_contract_tc(bool tf32, int64_t np, int nbins, int lmax, const unsigned long long* h_lbase,
                               const unsigned long long* h_kp, void* opA, void* opH, void* opL, double* partial,
                               int nsplit, unsigned int* err, bool inject_stall, cudaStream_t st);
cudaError_t launch_finalize_tc(const double* partial, int lmax, int nsplit, int nbins, double* zeta,
                               cudaStream_t st);

}  // namespace ctb
