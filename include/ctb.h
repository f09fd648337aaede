/*
 * ctb.h -- C ABI of libctb: Legendre-multipole three-point correlation
 * function (3PCF) on one GB300 GPU.
 *
 * The method (cTreeBalls paper, "Implementation" section): every catalogue
 * point in turn is the pivot (here "primary") of the triangles it closes; all
 * its neighbours inside the search range are found, and the multipole bins
 * are filled with the harmonic coefficients of the neighbours' directions
 * ("Statement of need": the 3PCF mapped onto an orthogonal basis whose
 * coefficients cost pair-count time, after Szapudi 2004 and Slepian &
 * Eisenstein).  The paper writes no formula; this library computes
 *
 *   a_lm(p,b)      = sum_{j != p, r_pj in bin b} w_j Y_lm(rhat_pj)
 *   zeta_l(b1,b2)  = 4 pi/(2l+1) * sum_p w_p sum_{m=-l..l} a_lm(p,b1) a_lm(p,b2)
 *
 * with real orthonormal Y_lm, linear half-open bins
 * [r_min + b D, r_min + (b+1) D), D = (r_max - r_min)/nbins, minimum-image
 * separations in a periodic cube of side `box` (box > 0) or plain separations
 * in open space (box <= 0).  j = k terms are included; pairs at zero
 * separation are never binned.  By the addition theorem
 *   zeta_l(b1,b2) = sum_p w_p sum_{j,k} w_j w_k P_l(rhat_pj . rhat_pk)
 *                   [b_j = b1][b_k = b2].
 *
 * Conventions for every entry point:
 *  - All functions return CTB_OK (0) or a negative CTB_ERR_* code, except
 *    ctb_create (NULL on failure), ctb_destroy and ctb_last_error.  No
 *    exception, abort or device trap crosses this boundary.  After a failure
 *    ctb_last_error() describes it.
 *  - Pointers marked "host or device" may point to host memory or to device
 *    memory of the current CUDA device; the library tells them apart with
 *    cudaPointerGetAttributes.  Inputs are copied; the caller keeps its
 *    buffers and may reuse them as soon as the call returns.
 *  - Work is issued on the context's stream (ctb_set_stream; default: the
 *    legacy default stream); calls that return results to the host
 *    synchronise that stream before returning.
 *  - A context is not thread-safe: use one context per host thread.
 */
#ifndef CTB_H
#define CTB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ctb_ctx ctb_ctx;

/* status codes */
#define CTB_OK 0
#define CTB_ERR_ARG (-1)        /* invalid argument (see each call)              */
#define CTB_ERR_NONFINITE (-2)  /* a coordinate or weight is NaN or infinite      */
#define CTB_ERR_OOM (-3)        /* device allocation failed                       */
#define CTB_ERR_CUDA (-4)       /* a CUDA call or kernel launch failed            */
#define CTB_ERR_TIMEOUT (-5)    /* a bounded device-side wait gave up             */
#define CTB_ERR_STATE (-6)      /* call out of order (e.g. compute before points) */
#define CTB_ERR_UNSUPPORTED (-7)/* option value or mode the library does not offer */

/* largest ell_max a context accepts */
#define CTB_LMAX_CAP 20
/* largest number of radial bins a context accepts */
#define CTB_NBINS_CAP 64
/* largest m_max of a sphere context (ctb_create_sphere) */
#define CTB_MMAX_CAP 16

/* option keys for ctb_set_option */
#define CTB_OPT_PRECISION 1      /* contraction precision, CTB_PREC_* (default FP32)        */
#define CTB_OPT_CELLS_PER_RMAX 2 /* grid cells per r_max along an axis, 1..64 (0 = auto)    */
#define CTB_OPT_LIST_CAPACITY 3  /* neighbour-list entries per chunk, 4096..2^32 (0 = 2^32) */
#define CTB_OPT_WARPS_PER_BLOCK 4/* pair-kernel warps per block, 1..4 (0 = auto: 4)         */
#define CTB_OPT_CHUNK_PRIMARIES 5/* primaries per pair-kernel launch, >= 1024 (0 = auto)    */
#define CTB_OPT_DETERMINISTIC 6  /* 1: fixed reduction order (default 1)                    */
#define CTB_OPT_AUTOTUNE 7       /* 1: time the grid cell sizes on the next set_points    */
#define CTB_OPT_FAULT_INJECT 8   /* test hook: 0 none, CTB_INJECT_STALL, CTB_INJECT_ALLOC   */

/* injected faults (CTB_OPT_FAULT_INJECT); nothing faults, traps or hangs the GPU */
#define CTB_INJECT_STALL 1 /* the tensor-core contraction's MMA thread first waits on a
                              barrier nothing signals; the wait gives up after ~10 ms, the
                              kernel takes its abort path, compute returns CTB_ERR_TIMEOUT
                              and the context stays usable */
#define CTB_INJECT_ALLOC 2 /* every device allocation the context attempts fails:
                              CTB_ERR_OOM */

/* contraction precisions (zeta = M^T W M per ell on the tensor cores or not) */
#define CTB_PREC_FP32 0   /* plain FP32 on the CUDA cores                       */
#define CTB_PREC_BF16X3 1 /* tcgen05 kind::f16, hi/lo BF16 split, 3 products     */
#define CTB_PREC_TF32 2   /* tcgen05 kind::tf32, one product                     */

/*
 * Create a context for one estimator configuration.
 *   box      side of the periodic cube; box <= 0 selects open (non-periodic)
 *            space
 *   r_min    inner edge of bin 0, >= 0
 *   r_max    outer edge of the last bin, > r_min; periodic: r_max <= box/2
 *   nbins    number of linear radial bins, 1..CTB_NBINS_CAP
 *   ell_max  largest multipole, 0..CTB_LMAX_CAP
 * Returns a new context, or NULL if an argument is invalid or no CUDA device
 * is usable (ctb_last_error(NULL) then says why).  The context binds to the
 * CUDA device current at this call.
 */
ctb_ctx* ctb_create(double box, double r_min, double r_max, int nbins, int ell_max);

/*
 * Projected (angular) multipoles of a scalar field on the unit sphere -- the
 * paper's own workload ("Statement of need": 3PCF multipoles for projected
 * fields such as the weak-lensing convergence; "Implementation": a harmonic
 * decomposition of one angle of the triangle, sin and cos by a Chebyshev
 * recurrence).  Points passed to ctb_set_points are directions (unit
 * vectors, float64 xyz, not re-normalised), weights the field values.
 *   separation  theta = 2 asin(|n_j - n_p| / 2), bins linear in theta on
 *               [theta_min, theta_max) (radians; theta_max <= pi), decided
 *               exactly on the chord against 2 sin(theta_b / 2) in FP64
 *   angle       phi_pj = atan2(u, v): u, v the components of n_j - n_p on the
 *               east and north unit vectors of p's tangent plane (at a pole
 *               east = +y); phi = 0 when both vanish
 *   a_m(p,b)    = sum_{j != p in b} w_j exp(i m phi_pj), m = 0..m_max
 *   zeta_m(b1,b2) = sum_p w_p Re[a_m(p,b1) conj(a_m(p,b2))]   (no 4 pi factor)
 * ctb_compute writes zeta_m as [(m_max+1)][nbins][nbins]; ctb_get_alm writes
 * [primary][bin][2 m_max + 1] as (a_0, Re a_1, Im a_1, ..., Re a_mmax, Im a_mmax)
 * in the library's tangent frame; ctb_get_2pcf gives sum_p w_p sum_{j in b} w_j.
 * zeta_m does not depend on the tangent frame.  The contraction runs in FP32
 * (CTB_OPT_PRECISION other than FP32, ctb_compute_batch and ctb_edge_correct
 * return CTB_ERR_UNSUPPORTED).  m_max in [0, CTB_MMAX_CAP]; NULL on bad
 * arguments (message from ctb_last_error(NULL)).
 */
ctb_ctx* ctb_create_sphere(double theta_min, double theta_max, int nbins, int m_max);

/*
 * Load a catalogue (paper, "Implementation": the points that act as pivots
 * and as neighbours).  Ingests, builds the uniform cell grid and sorts the
 * points into cell order on the device.
 *   xyz  [n][3] float64, row-major, host or device.  Periodic: any finite
 *        value, wrapped into [0, box).
 *   w    [n] float64 weights (may be negative), host or device; NULL means
 *        unit weights.
 *   n    number of points, 0 <= n < 2^31.
 * Errors: CTB_ERR_ARG (n out of range, xyz NULL with n > 0),
 * CTB_ERR_NONFINITE (any coordinate or weight not finite; the context then
 * holds no points), CTB_ERR_OOM, CTB_ERR_CUDA.
 */
int ctb_set_points(ctb_ctx* ctx, const double* xyz, const double* w, int64_t n);

/*
 * Compute zeta_l(b1,b2) over all points as primaries.
 *   zeta_out  [(ell_max+1)][nbins][nbins] float64, host or device, written
 *             in full (the matrix is symmetric in b1, b2).
 * Errors: CTB_ERR_STATE (no ctb_set_points yet), CTB_ERR_ARG (zeta_out
 * NULL), CTB_ERR_OOM, CTB_ERR_CUDA, CTB_ERR_TIMEOUT.
 */
int ctb_compute(ctb_ctx* ctx, double* zeta_out);

/*
 * As ctb_compute, with the primaries restricted to the listed points (all
 * points stay secondaries).  Summing the results of a partition of the
 * primaries reproduces ctb_compute up to rounding.
 *   primary_idx  [m] int64 indices into the catalogue of ctb_set_points,
 *                host or device, each in [0, n); duplicates count twice.
 *   m            number of primaries, >= 0.
 * Errors: as ctb_compute, plus CTB_ERR_ARG for an index out of range.
 */
int ctb_compute_subset(ctb_ctx* ctx, const int64_t* primary_idx, int64_t m, double* zeta_out);

/*
 * Shared neighbour lists for close pivots (paper, "Implementation": pivots
 * close to one another share one neighbour list; the pivot radius is set
 * from the mean separation unless the user gives one).  An approximation of
 * ctb_compute that runs the pair pipeline once per group of pivots.
 *   groups      a point belongs to the pivot cell (floor(x/h), floor(y/h),
 *               floor(z/h)) of side h, cells aligned at the origin of
 *               coordinates, taken on the coordinates as stored (periodic:
 *               wrapped into [0, box) on the box / 2^32 grid; open: on a
 *               power-of-two grid over the bounding box)
 *   estimate    each group g is represented by its member of smallest
 *               catalogue index c_g and carries W_g = sum of its members'
 *               weights:
 *                 zeta_l(b1,b2) ~= 4 pi/(2l+1) sum_g W_g sum_m a_lm(c_g,b1) a_lm(c_g,b2)
 *               (on the sphere, zeta_m with the projected a_m), i.e. every
 *               member takes its representative's neighbour list.
 *   bound       per entry, |shared - ctb_compute| <= sum_p |w_p| [min(l (A1 S2
 *               + S1 A2), 2 S1 S2) + D1 U2 + U1 D2], summed over non-
 *               representatives p with representative c.  S_b and A_b are
 *               the |w_j| sums, plain and times the angle between x_j - x_p
 *               and x_j - x_c, over neighbours j in bin b from both p and c.
 *               D_b and U_b are the |w_j| sums over j in b from exactly one
 *               of them and from either.  The angular term follows from
 *               Bernstein's inequality, |d/dgamma P_l(cos gamma)| <= l.  This
 *               is a statement about the estimate, up to FP32 rounding of the
 *               computation.  Sphere mode: the same sum with m for l and,
 *               for the angle, the angle between p's tangent direction to j
 *               and c's carried to p's tangent plane by the rotation taking
 *               c's normal to p's (|d/dpsi cos(m psi)| <= m).
 *   pivot_cell  h > 0, or 0 for the mean separation: (V / n)^(1/3) with
 *               V = box^3 (periodic) or the product of the bounding box's
 *               sides, each at least r_max (open); sqrt(4 pi / n) on the
 *               sphere.
 *   zeta_out    as ctb_compute.  ctb_get_2pcf then gives the same shared
 *               estimate of the pair sums.
 * Errors: as ctb_compute, plus CTB_ERR_ARG for h negative or not finite, or
 * more than 2^64 pivot cells over the catalogue's extent.
 */
int ctb_compute_shared(ctb_ctx* ctx, double pivot_cell, double* zeta_out);

/* The pivot cell side h and the number of groups of the last
 * ctb_compute_shared.  CTB_ERR_STATE if there was none since the last
 * ctb_set_points. */
int ctb_get_pivot_groups(ctb_ctx* ctx, double* pivot_cell, int64_t* groups);

/*
 * Export a_lm(p, b) of the listed primaries (debug / parity; the same
 * coefficients the contraction consumes, rounded to float32).
 *   primary_idx  [m] int64 catalogue indices, host or device
 *   alm_out      [m][nbins][(ell_max+1)^2] float32, host or device;
 *                coefficient (l, m) of the real basis at index l*l + l + m,
 *                Y_l,+m ~ cos(m phi), Y_l,-m ~ sin(m phi), Condon-Shortley
 *                phase included.
 */
int ctb_get_alm(ctb_ctx* ctx, const int64_t* primary_idx, int64_t m, float* alm_out);

/*
 * Compute zeta for k independent catalogues in one pass (mock batches for
 * covariance estimates).  All catalogues share the context's box, bins and
 * ell_max; catalogue i has n[i] points at xyz[i] (host or device, [n_i][3])
 * and weights w[i] (NULL pointer or NULL array: unit weights).
 *   zeta_out  [k][(ell_max+1)][nbins][nbins] float64, host or device.
 * All catalogues go into one sorted grid (cell key = catalogue * cells +
 * cell), one pair pipeline runs over every primary with each neighbour search
 * kept inside its own catalogue, and the contraction keeps one set of FP64
 * partial sums per catalogue.  With CTB_OPT_AUTOTUNE set (and no fixed
 * CTB_OPT_CELLS_PER_RMAX) the first batch tunes the grid on its largest
 * catalogue and the context keeps it.  The batch replaces the context's catalogue:
 * call ctb_set_points again before the next ctb_compute.  Periodic boxes only.
 * Errors: CTB_ERR_ARG (k < 1, a NULL xyz[i] with n[i] > 0, a negative n[i],
 * more than 2^31 points in total or k * grid cells >= 2^32),
 * CTB_ERR_UNSUPPORTED (open boundary), CTB_ERR_NONFINITE, CTB_ERR_OOM,
 * CTB_ERR_CUDA, CTB_ERR_TIMEOUT.
 */
int ctb_compute_batch(ctb_ctx* ctx, const double* const* xyz, const double* const* w,
                      const int64_t* n, int k, double* zeta_out);

/* Set an option (CTB_OPT_*).  Returns CTB_ERR_ARG for an unknown key or a value
 * out of range, CTB_ERR_UNSUPPORTED for a precision the library cannot run.
 * CTB_OPT_LIST_CAPACITY bounds the neighbour lists of one chunk of primaries
 * (4 bytes per entry) and the candidates' bin codes of that chunk (1 byte per
 * candidate, at most 4 per list entry of the capacity); chunks are sized to
 * fit, and a compute in which one primary alone has more pairs (or candidates)
 * than that fails with CTB_ERR_OOM.
 * CTB_OPT_AUTOTUNE = 1 (with CTB_OPT_CELLS_PER_RMAX left at 0) makes the next
 * ctb_set_points grid the catalogue at 3, 4, 6, 8, 12 and 16 cells per r_max,
 * time the pair kernels on a sample of at most 8192 primaries for each, and
 * keep the fastest grid for this context (setting the option again re-tunes).
 * The result does not depend on the grid beyond FP32 summation order. */
int ctb_set_option(ctb_ctx* ctx, int key, int64_t value);

/* Issue all further work on `stream` (a cudaStream_t of the context's device,
 * e.g. torch.cuda.current_stream().cuda_stream); NULL = legacy default. */
int ctb_set_stream(ctb_ctx* ctx, void* stream);

/*
 * Route the library's device allocations through a caller's allocator (e.g.
 * the PyTorch caching allocator).  alloc(bytes, user) returns device memory
 * or NULL; free(ptr, user) releases it.  Pass alloc = NULL to go back to
 * cudaMallocAsync on the context's stream.  Buffers already held are
 * released first, so call this before ctb_set_points.
 */
int ctb_set_allocator(ctb_ctx* ctx, void* (*alloc)(size_t bytes, void* user),
                      void (*free_fn)(void* ptr, void* user), void* user);

/*
 * Per-stage device times in milliseconds, measured with CUDA events on the
 * context's stream: [0], [1] from the last ctb_set_points (or batch), the
 * others from the last ctb_compute* call:
 *   [0] ingest  [1] sort + grid  [2] pair multipoles (= [6] + [7])  [3] pack
 *   [4] contraction  [5] reduce + normalise
 *   [6] neighbour enumeration (count + scan + fill)  [7] harmonic accumulation
 *   [8] pivot grouping (ctb_compute_shared; 0 otherwise)
 * Writes min(cap, 9) values; returns the number written.
 */
int ctb_get_timings(ctb_ctx* ctx, double* ms_per_stage, int cap);

/* Number of CUDA kernels the library launched during the last ctb_set_points
 * plus the last ctb_compute (observability: what one full pass costs in
 * launches). */
int ctb_get_launch_count(ctb_ctx* ctx, uint64_t* kernels);

/* Number of ordered (primary, secondary) pairs binned by the last compute. */
int ctb_get_pair_count(ctb_ctx* ctx, uint64_t* pairs);

/* Number of primary chunks the last compute ran.  Each chunk is one launch of
 * each pair kernel (count, fill, accumulate) over its own neighbour lists, so
 * pairs / chunks is the mean work of one launch.  A chunk that overflowed the
 * list buffer and was split is not counted.  0 before the first compute. */
int ctb_get_chunk_count(ctb_ctx* ctx, uint64_t* chunks);

/*
 * Two-point function from the same pass (paper, "Statement of need": the
 * 2PCF alongside the 3PCF).  out[k * nbins + b] = sum_p w_p sum_{j != p,
 * r_pj in bin b} w_j, the weighted pair sums of the last ctb_compute /
 * ctb_compute_subset (k = 0; over the given primaries) or of each catalogue k
 * of the last ctb_compute_batch.  They come from the a_00 column of the
 * accumulation (a_00 = sum_j w_j / sqrt(4 pi)), FP32 per (primary, bin) and
 * FP64 over primaries.  `cap` is the capacity of the host array `out`.
 * Returns the number of values written (catalogues * nbins), CTB_ERR_STATE if
 * no zeta was computed since the last ctb_set_points, CTB_ERR_ARG if cap is
 * too small.
 */
int ctb_get_2pcf(ctb_ctx* ctx, double* out, int cap);

/*
 * Edge-corrected multipoles (Slepian & Eisenstein 2015; paper, "Implementation":
 * edge corrections).  Inputs are two results of ctb_compute with this
 * context's ell_max and nbins, [(ell_max+1)][nbins][nbins] FP64:
 *   zeta_nnn  the data-minus-randoms catalogue (randoms with negative weights)
 *   zeta_rrr  the randoms alone, with the same weights taken positive
 * Per bin pair the coefficients zeta_l of zeta(mu) = N(mu) / R(mu) =
 * sum_l zeta_l P_l(mu) solve  n_l / r_0 = sum_l' M_ll' zeta_l'  with
 *   n_l = (2l+1)/2 zeta_nnn_l,  r_l = (2l+1)/2 zeta_rrr_l,  f_l = r_l / r_0,
 *   M_ll' = (2l+1) sum_l'' (l l' l''; 0 0 0)^2 f_l''   (all l <= ell_max),
 * in FP64 on the device (one thread per bin pair, partial pivoting).
 * zeta_out receives zeta_l [(ell_max+1)][nbins][nbins]; bin pairs without
 * random triplets or with a singular system are NaN.  Pointers may be host
 * or device memory; the caller keeps them.  Returns CTB_OK, CTB_ERR_ARG,
 * CTB_ERR_OOM or CTB_ERR_CUDA.
 */
int ctb_edge_correct(ctb_ctx* ctx, const double* zeta_nnn, const double* zeta_rrr, double* zeta_out);

/* The cell grid of the current catalogue (or of the last ctb_compute_batch):
 * cells per r_max along an axis (the option, else the autotuner's choice,
 * else 8) and cells per axis of the (per-catalogue) cube.  CTB_ERR_STATE
 * before ctb_set_points or a batch. */
int ctb_get_grid(ctb_ctx* ctx, int* cells_per_rmax, int* cells_per_axis);

/*
 * zeta_l(b1,b2) from a_lm rows and primary weights already on the device,
 * without allocating any device memory.  The paper has no counterpart: this
 * exists for callers that must not allocate device memory when they call in
 * -- services that reserve the whole device in their own pool up front and
 * hand out only fixed buffers, or loops with a latency budget in which an
 * allocation, or its failure, is not acceptable.  It runs the same FP32
 * contraction and FP64 normalisation as ctb_compute, with its per-block
 * partial sums in a fixed, file-scope device array of the library: 8 MB on
 * every GPU that loads the library, held until the process exits.
 *   alm       [np][nbins][(ell_max+1)^2] float32, device; coefficient (l, m)
 *             at index l*l + l + m (the layout of ctb_get_alm)
 *   w         [np] float32 primary weights, device
 *   np        number of primaries, >= 0 (0 gives zeta = 0)
 *   zeta_out  [(ell_max+1)][nbins][nbins] float64, device, written in full
 *   stream    cudaStream_t to run on (NULL = legacy default); the call returns
 *             once the work is queued
 * Limits: nbins 1..CTB_NBINS_CAP, ell_max 0..CTB_LMAX_CAP and
 * (ell_max+1) * nbins^2 <= 16384 (the array then holds at least 64 partial
 * blocks); otherwise CTB_ERR_ARG.  A failed CUDA call gives CTB_ERR_CUDA.
 * ctb_last_error() does not describe failures of this call.
 * The first call on a device looks up the array's device address and the SM
 * count with that device current (no device work); make that first call
 * before any stream capture.  The partials use one wave of the contraction's
 * resident blocks, as far as the array holds them.  All calls share the
 * array: calls whose work overlaps on the GPU race and must be serialised by
 * the caller (e.g. one stream).  Each call first clears the partial blocks it
 * uses (nparts * (ell_max+1) * nbins^2 values), and its finalisation reads
 * exactly those, so what an earlier call with another shape left beyond them
 * is never read.
 */
int ctb_contract_noalloc(const float* alm, const float* w, int64_t np, int nbins, int ell_max,
                         double* zeta_out, void* stream);

/* Release the context and all device memory it holds.  NULL is a no-op. */
void ctb_destroy(ctb_ctx* ctx);

/* Text of the last error on ctx (or of the last failed ctb_create on this
 * thread when ctx is NULL).  Valid until the next call on the same context. */
const char* ctb_last_error(const ctb_ctx* ctx);

/* Library version string. */
const char* ctb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CTB_H */
