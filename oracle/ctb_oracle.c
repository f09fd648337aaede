/*
 * ctb_oracle.c -- plain FP64 CPU oracle for the 3-D Legendre-multipole
 * three-point correlation function (3PCF).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py use it.  It shares no code, header, table or
 * constant with the CUDA library; the two meet only through the seeded input
 * generators.
 *
 * What it computes (paper: "Implementation" section -- pick each catalogue
 * point as the pivot / vertex of a triangle, find all its neighbours within
 * the search range, fill the multipole bins; "Statement of need" -- map the
 * 3PCF onto an orthogonal harmonic basis whose coefficients cost pair-count
 * time, after Szapudi 2004 and Slepian & Eisenstein).  The paper writes no
 * formula, so this file takes the reading recorded in the design notes:
 *
 *   a_lm(p,b)   = sum_{j != p, r_pj in bin b} w_j Y_lm(rhat_pj)
 *   zeta_l(b1,b2) = 4 pi / (2l+1) * sum_p w_p sum_m a_lm(p,b1) a_lm(p,b2)
 *
 * with real orthonormal Y_lm (m = -l..l), bins [rmin + b D, rmin + (b+1) D),
 * D = (rmax - rmin)/nbins, r_pj the minimum-image separation when the box is
 * periodic (box > 0) and the plain separation otherwise (box <= 0).  By the
 * addition theorem this equals
 *   sum_p w_p sum_{j,k} w_j w_k P_l(rhat_pj . rhat_pk) [b_j = b1][b_k = b2]
 * including the j = k terms.
 *
 * Algorithm: brute force, O(N x N_primaries), no spatial index, every
 * quantity in double precision, the direction's azimuth from atan2 and
 * cos(m phi), sin(m phi) from libm, the polar part from the textbook
 * normalised associated-Legendre recurrence.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#ifndef M_SQRT2
#define M_SQRT2 1.41421356237309504880
#endif

#define ORACLE_LMAX_CAP 40

/* Index of the real coefficient (l, m), m = -l..l, in a flat array. */
static inline int lm_index(int l, int m) { return l * l + l + m; }

/*
 * Real orthonormal spherical harmonics at the unit direction (x, y, z) for
 * all l <= lmax, written to out[l*l + l + m].  Convention:
 *   Y_l0      = S(l, 0)
 *   Y_l,+m    = sqrt(2) S(l, m) cos(m phi)      m > 0
 *   Y_l,-m    = sqrt(2) S(l, m) sin(m phi)      m > 0
 * where S(l, m) = (-1)^m sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_l^m(cos theta)
 * (P_l^m without the Condon-Shortley phase, so S carries it), i.e. S is the
 * C++17 std::sph_legendre(l, m, theta).
 * Polar recurrence (normalised, Numerical-Recipes form):
 *   Pbar_0^0 = 1/sqrt(4 pi)
 *   Pbar_m^m = -sqrt((2m+1)/(2m)) sin(theta) Pbar_{m-1}^{m-1}
 *   Pbar_{m+1}^m = sqrt(2m+3) cos(theta) Pbar_m^m
 *   Pbar_l^m = sqrt((4l^2-1)/(l^2-m^2)) (cos(theta) Pbar_{l-1}^m
 *              - sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)) Pbar_{l-2}^m)
 */
void oracle_ylm(int lmax, double x, double y, double z, double* out)
{
    double ct = z;
    double st = hypot(x, y);
    double phi = atan2(y, x);
    double pmm = 1.0 / sqrt(4.0 * M_PI);
    for (int m = 0; m <= lmax; ++m) {
        if (m > 0) pmm = -sqrt((2.0 * m + 1.0) / (2.0 * m)) * st * pmm;
        double cm = cos(m * phi), sm = sin(m * phi);
        double p_lm2 = 0.0, p_lm1 = pmm;
        for (int l = m; l <= lmax; ++l) {
            double p;
            if (l == m) {
                p = pmm;
            } else if (l == m + 1) {
                p = sqrt(2.0 * m + 3.0) * ct * pmm;
            } else {
                double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
                double b = sqrt((((double)(l - 1) * (l - 1)) - (double)m * m) /
                                (4.0 * (l - 1) * (l - 1) - 1.0));
                p = a * (ct * p_lm1 - b * p_lm2);
            }
            if (l > m) { p_lm2 = p_lm1; p_lm1 = p; }
            if (m == 0) {
                out[lm_index(l, 0)] = p;
            } else {
                out[lm_index(l, m)] = M_SQRT2 * p * cm;
                out[lm_index(l, -m)] = M_SQRT2 * p * sm;
            }
        }
    }
}

/* Check the arguments the way the library's contract states them. */
static int check_args(int64_t n, double box, double rmin, double rmax, int nbins, int lmax)
{
    if (n < 0 || nbins < 1 || lmax < 0 || lmax > ORACLE_LMAX_CAP) return -1;
    if (!(rmin >= 0.0) || !(rmax > rmin)) return -1;
    if (box > 0.0 && rmax > 0.5 * box) return -1;
    return 0;
}

/* Separation vector from point p to point j (minimum image if periodic). */
static inline void separation(const double* xyz, int64_t p, int64_t j, double box, double d[3])
{
    for (int k = 0; k < 3; ++k) {
        double v = xyz[3 * j + k] - xyz[3 * p + k];
        if (box > 0.0) v -= box * nearbyint(v / box);
        d[k] = v;
    }
}

/*
 * Bin of a separation r: the b with rmin + b D <= r < rmin + (b+1) D, or -1.
 * Pairs with r == 0 (coincident points) are never binned.
 */
static inline int bin_of(double r, double rmin, double rmax, double dr, int nbins)
{
    if (!(r >= rmin) || !(r < rmax) || r == 0.0) return -1;
    int b = (int)floor((r - rmin) / dr);
    if (b < 0) b = 0;
    if (b >= nbins) b = nbins - 1;
    /* settle rounding at an edge against the edge values themselves */
    while (b > 0 && r < rmin + b * dr) --b;
    while (b + 1 < nbins && r >= rmin + (b + 1) * dr) ++b;
    return b;
}

/*
 * a_lm(p, b) for the listed primaries (prim[i], i < np; prim == NULL means
 * primaries 0..np-1).  a_out is [np][nbins][(lmax+1)^2], row-major.
 * Returns 0, or -1 on bad arguments.  npairs_out (may be NULL) receives the
 * number of (primary, secondary) pairs that fell in a bin.
 */
int oracle_alm(const double* xyz, const double* w, int64_t n, double box, double rmin,
               double rmax, int nbins, int lmax, const int64_t* prim, int64_t np,
               double* a_out, int64_t* npairs_out, int nthreads)
{
    if (check_args(n, box, rmin, rmax, nbins, lmax)) return -1;
    const int nc = (lmax + 1) * (lmax + 1);
    const double dr = (rmax - rmin) / nbins;
    int64_t npairs = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : npairs)
    for (int64_t i = 0; i < np; ++i) {
        int64_t p = prim ? prim[i] : i;
        double* a = a_out + (size_t)i * nbins * nc;
        double y[(ORACLE_LMAX_CAP + 1) * (ORACLE_LMAX_CAP + 1)];
        memset(a, 0, sizeof(double) * (size_t)nbins * nc);
        for (int64_t j = 0; j < n; ++j) {
            if (j == p) continue;
            double d[3];
            separation(xyz, p, j, box, d);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            int b = bin_of(r, rmin, rmax, dr, nbins);
            if (b < 0) continue;
            ++npairs;
            oracle_ylm(lmax, d[0] / r, d[1] / r, d[2] / r, y);
            double wj = w ? w[j] : 1.0;
            double* ab = a + (size_t)b * nc;
            for (int c = 0; c < nc; ++c) ab[c] += wj * y[c];
        }
    }
    if (npairs_out) *npairs_out = npairs;
    return 0;
}

/*
 * zeta_l(b1, b2) summed over the listed primaries (prim == NULL: all n).
 *   zeta   [(lmax+1)][nbins][nbins]  the estimator above
 *   gram   [(lmax+1)][nbins][nbins]  the same with |w_p| (NULL to skip);
 *          sqrt(gram(b1,b1) gram(b2,b2)) >= |zeta(b1,b2)| bounds every entry
 *   wpairs [nbins]   sum_p w_p sum_{j in b} w_j      (NULL to skip)
 *   selfw  [nbins]   sum_p w_p sum_{j in b} w_j^2    (NULL to skip): the j = k
 *          part of each diagonal entry (P_l(1) = 1, times 4 pi/(2l+1) Y-sum)
 *   wprim  [np] or NULL: the weight each listed primary carries in the sums
 *          over p in place of w_p (its neighbours keep their own weights);
 *          used for primaries that stand for a group of pivots
 *   npairs_out   number of binned (p, j) pairs
 *   namb_out     pairs whose separation lies within amb_tol (relative) of a
 *                bin edge, rmin or rmax: the ones a lower-precision binning
 *                may legitimately place in the neighbouring bin
 * Sums run per thread over a static primary partition and are combined in
 * thread order, so the result is fixed for a fixed thread count.
 */
int oracle_zeta(const double* xyz, const double* w, int64_t n, double box, double rmin,
                double rmax, int nbins, int lmax, const int64_t* prim, int64_t np,
                double* zeta, double* gram, double* wpairs, double* selfw,
                int64_t* npairs_out, int64_t* namb_out, double amb_tol, int nthreads,
                const double* wprim)
{
    if (check_args(n, box, rmin, rmax, nbins, lmax)) return -1;
    if (!prim) np = n;
    const int nc = (lmax + 1) * (lmax + 1);
    const int L1 = lmax + 1;
    const double dr = (rmax - rmin) / nbins;
    const size_t zsz = (size_t)L1 * nbins * nbins;
    int nt = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        nt = omp_get_num_threads();
    }
#endif
    double* zpart = (double*)calloc((size_t)nt * zsz, sizeof(double));
    double* gpart = (double*)calloc((size_t)nt * zsz, sizeof(double));
    double* ppart = (double*)calloc((size_t)nt * nbins, sizeof(double));
    double* spart = (double*)calloc((size_t)nt * nbins, sizeof(double));
    int64_t* cnt = (int64_t*)calloc((size_t)nt * 2, sizeof(int64_t));
    if (!zpart || !gpart || !ppart || !spart || !cnt) {
        free(zpart); free(gpart); free(ppart); free(spart); free(cnt);
        return -2;
    }
#pragma omp parallel
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double* zt = zpart + (size_t)t * zsz;
        double* gt = gpart + (size_t)t * zsz;
        double* pt = ppart + (size_t)t * nbins;
        double* st = spart + (size_t)t * nbins;
        double* a = (double*)malloc(sizeof(double) * (size_t)nbins * nc);
        double* nb = (double*)malloc(sizeof(double) * (size_t)nbins);
        double* sb = (double*)malloc(sizeof(double) * (size_t)nbins);
        double y[(ORACLE_LMAX_CAP + 1) * (ORACLE_LMAX_CAP + 1)];
#pragma omp for schedule(static)
        for (int64_t i = 0; i < np; ++i) {
            int64_t p = prim ? prim[i] : i;
            memset(a, 0, sizeof(double) * (size_t)nbins * nc);
            memset(nb, 0, sizeof(double) * (size_t)nbins);
            memset(sb, 0, sizeof(double) * (size_t)nbins);
            for (int64_t j = 0; j < n; ++j) {
                if (j == p) continue;
                double d[3];
                separation(xyz, p, j, box, d);
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                if (amb_tol > 0.0 && r > 0.0) {
                    double tol = amb_tol * r;
                    for (int k = 0; k <= nbins; ++k) {
                        if (fabs(r - (rmin + k * dr)) < tol) { cnt[2 * t + 1]++; break; }
                    }
                }
                int b = bin_of(r, rmin, rmax, dr, nbins);
                if (b < 0) continue;
                cnt[2 * t]++;
                oracle_ylm(lmax, d[0] / r, d[1] / r, d[2] / r, y);
                double wj = w ? w[j] : 1.0;
                double* ab = a + (size_t)b * nc;
                for (int c = 0; c < nc; ++c) ab[c] += wj * y[c];
                nb[b] += wj;
                sb[b] += wj * wj;
            }
            double wp = wprim ? wprim[i] : (w ? w[p] : 1.0);
            for (int b = 0; b < nbins; ++b) { pt[b] += wp * nb[b]; st[b] += wp * sb[b]; }
            for (int l = 0; l <= lmax; ++l) {
                for (int b1 = 0; b1 < nbins; ++b1) {
                    for (int b2 = 0; b2 < nbins; ++b2) {
                        double s = 0.0;
                        for (int m = -l; m <= l; ++m)
                            s += a[(size_t)b1 * nc + lm_index(l, m)] * a[(size_t)b2 * nc + lm_index(l, m)];
                        size_t o = ((size_t)l * nbins + b1) * nbins + b2;
                        zt[o] += wp * s;
                        gt[o] += fabs(wp) * s;
                    }
                }
            }
        }
        free(a); free(nb); free(sb);
    }
    int64_t npairs = 0, namb = 0;
    for (size_t o = 0; o < zsz; ++o) {
        double s = 0.0, g = 0.0;
        for (int t = 0; t < nt; ++t) { s += zpart[(size_t)t * zsz + o]; g += gpart[(size_t)t * zsz + o]; }
        int l = (int)(o / ((size_t)nbins * nbins));
        double f = 4.0 * M_PI / (2.0 * l + 1.0);
        zeta[o] = f * s;
        if (gram) gram[o] = f * g;
    }
    for (int b = 0; b < nbins; ++b) {
        double s = 0.0, q = 0.0;
        for (int t = 0; t < nt; ++t) { s += ppart[(size_t)t * nbins + b]; q += spart[(size_t)t * nbins + b]; }
        if (wpairs) wpairs[b] = s;
        if (selfw) selfw[b] = q;
    }
    for (int t = 0; t < nt; ++t) { npairs += cnt[2 * t]; namb += cnt[2 * t + 1]; }
    if (npairs_out) *npairs_out = npairs;
    if (namb_out) *namb_out = namb;
    free(zpart); free(gpart); free(ppart); free(spart); free(cnt);
    return 0;
}

/*
 * Edge-ambiguous pairs of the listed primaries: every (p, j) whose separation
 * r lies within amb_tol * r of an edge rmin + k D, k = 0..nbins (so within the
 * rounding of any binning that is not exact in FP64 -- e.g. one that first
 * rounds the coordinates onto a fixed-point grid -- it may land on the other
 * side of that edge).  Up to `cap` records are written, in primary order:
 *   rec_i[2 t]     index of the primary in the list (i, not p)
 *   rec_i[2 t + 1] j
 *   rec_d[5 t..]   separation vector d (3), r, and the edge index k
 * Returns the number of such pairs (which may exceed cap), or -1 on bad
 * arguments.  Serial: the record order is fixed.
 */
int64_t oracle_ambiguous(const double* xyz, int64_t n, double box, double rmin, double rmax, int nbins,
                         const int64_t* prim, int64_t np, double amb_tol, int64_t* rec_i, double* rec_d,
                         int64_t cap)
{
    if (check_args(n, box, rmin, rmax, nbins, 0) || !(amb_tol > 0.0)) return -1;
    if (!prim) np = n;
    const double dr = (rmax - rmin) / nbins;
    int64_t cnt = 0;
    for (int64_t i = 0; i < np; ++i) {
        int64_t p = prim ? prim[i] : i;
        for (int64_t j = 0; j < n; ++j) {
            if (j == p) continue;
            double d[3];
            separation(xyz, p, j, box, d);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (r == 0.0) continue;
            for (int k = 0; k <= nbins; ++k) {
                if (fabs(r - (rmin + k * dr)) < amb_tol * r) {
                    if (cnt < cap) {
                        rec_i[2 * cnt] = i;
                        rec_i[2 * cnt + 1] = j;
                        rec_d[5 * cnt] = d[0];
                        rec_d[5 * cnt + 1] = d[1];
                        rec_d[5 * cnt + 2] = d[2];
                        rec_d[5 * cnt + 3] = r;
                        rec_d[5 * cnt + 4] = (double)k;
                    }
                    ++cnt;
                    break;
                }
            }
        }
    }
    return cnt;
}

/* Number of OpenMP threads a parallel region gets (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
