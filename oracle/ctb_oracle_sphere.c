/*
 * ctb_oracle_sphere.c -- plain FP64 CPU oracle for the projected
 * (angular) 3PCF multipoles on the unit sphere.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py use it.  It shares no code with the CUDA library.
 *
 * What it computes (paper, "Statement of need": 3PCF multipoles of scalar
 * fields on the sphere, such as the weak-lensing convergence, by a harmonic
 * decomposition of one angle of the triangle; "Implementation": for each
 * pivot, its neighbours in the search range fill the multipole bins, the
 * sin/cos of the angle coming from a Chebyshev recurrence).  The paper
 * writes no formula; the reading taken here:
 *
 *   points     directions n_j (the given xyz; not re-normalised), weight w_j
 *              (the field value)
 *   separation theta_pj = 2 asin(|n_j - n_p| / 2); bin b when the chord
 *              |n_j - n_p| lies in [c_b, c_{b+1}), c_b = 2 sin(theta_b / 2),
 *              theta_b = theta_min + b (theta_max - theta_min) / nbins
 *   angle      phi_pj = atan2(u, v), u and v the components of n_j - n_p on
 *              the east and north unit vectors of the tangent plane at p
 *              (e_E = z x n_p / |z x n_p|, e_N = n_p x e_E with n_p
 *              normalised; at a pole e_E = y); phi = 0 when u = v = 0
 *   a_m(p,b)   = sum_{j != p in bin b} w_j exp(i m phi_pj),  m = 0..m_max
 *   zeta_m(b1,b2) = sum_p w_p Re[a_m(p,b1) conj(a_m(p,b2))]
 *              = sum_p w_p sum_{j in b1, k in b2} w_j w_k cos(m (phi_pj - phi_pk))
 *
 * zeta_m does not depend on the choice of tangent frame at each pivot (a
 * rotation of the frame multiplies every a_m(p, .) by one phase).
 *
 * Algorithm: brute force, O(N x N_primaries), no spatial index, double
 * precision, cos(m phi) and sin(m phi) from libm.  OpenMP over the primaries,
 * per-thread partial sums added in thread order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

#define SPHERE_MMAX_CAP 64

static void tangent_frame(const double* n, double eE[3], double eN[3])
{
    double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double u[3] = {n[0] / len, n[1] / len, n[2] / len};
    double rho = sqrt(u[0] * u[0] + u[1] * u[1]);
    if (rho > 0.0) {
        eE[0] = -u[1] / rho;
        eE[1] = u[0] / rho;
        eE[2] = 0.0;
    } else {
        eE[0] = 0.0;
        eE[1] = 1.0;
        eE[2] = 0.0;
    }
    eN[0] = u[1] * eE[2] - u[2] * eE[1];
    eN[1] = u[2] * eE[0] - u[0] * eE[2];
    eN[2] = u[0] * eE[1] - u[1] * eE[0];
}

/*
 * zeta [mmax+1][nbins][nbins], gram (same with |w_p|) and wpairs [nbins]
 * (sum_p w_p sum_{j in b} w_j) may be NULL except zeta.  prim: primaries (NULL
 * = all).  wprim [np] or NULL: the weight each listed primary carries in place
 * of w_p (its neighbours keep their own).  Returns 0, -1 on bad arguments, -2 on allocation failure.
 */
int oracle_zeta_sphere(const double* xyz, const double* w, int64_t n, double tmin, double tmax, int nbins,
                       int mmax, const int64_t* prim, int64_t np, double* zeta, double* gram, double* wpairs,
                       int64_t* npairs_out, int nthreads, const double* wprim)
{
    if (n < 0 || nbins < 1 || mmax < 0 || mmax > SPHERE_MMAX_CAP || !(tmin >= 0.0) || !(tmax > tmin) ||
        tmax > 3.14159265358979323846)
        return -1;
    if (!prim) np = n;
    double* edge = (double*)malloc(sizeof(double) * (size_t)(nbins + 1));
    if (!edge) return -2;
    for (int b = 0; b <= nbins; ++b) edge[b] = 2.0 * sin(0.5 * (tmin + b * (tmax - tmin) / nbins));
    const int M1 = mmax + 1;
    const size_t zsz = (size_t)M1 * nbins * nbins;
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
    int64_t* cnt = (int64_t*)calloc((size_t)nt, sizeof(int64_t));
    if (!zpart || !gpart || !ppart || !cnt) {
        free(edge); free(zpart); free(gpart); free(ppart); free(cnt);
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
        /* a[b][m][re, im] */
        double* a = (double*)malloc(sizeof(double) * (size_t)nbins * M1 * 2);
        double* nb = (double*)malloc(sizeof(double) * (size_t)nbins);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < np; ++i) {
            int64_t p = prim ? prim[i] : i;
            const double* xp = xyz + 3 * p;
            double eE[3], eN[3];
            tangent_frame(xp, eE, eN);
            memset(a, 0, sizeof(double) * (size_t)nbins * M1 * 2);
            memset(nb, 0, sizeof(double) * (size_t)nbins);
            for (int64_t j = 0; j < n; ++j) {
                if (j == p) continue;
                const double* xj = xyz + 3 * j;
                double d[3] = {xj[0] - xp[0], xj[1] - xp[1], xj[2] - xp[2]};
                double c = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                if (!(c > 0.0) || c < edge[0] || c >= edge[nbins]) continue;
                int b = 0;
                while (b + 1 < nbins && c >= edge[b + 1]) ++b;
                cnt[t]++;
                double u = d[0] * eE[0] + d[1] * eE[1] + d[2] * eE[2];
                double v = d[0] * eN[0] + d[1] * eN[1] + d[2] * eN[2];
                double phi = (u == 0.0 && v == 0.0) ? 0.0 : atan2(u, v);
                double wj = w ? w[j] : 1.0;
                double* ab = a + (size_t)b * M1 * 2;
                for (int m = 0; m <= mmax; ++m) {
                    ab[2 * m] += wj * cos(m * phi);
                    ab[2 * m + 1] += wj * sin(m * phi);
                }
                nb[b] += wj;
            }
            double wp = wprim ? wprim[i] : (w ? w[p] : 1.0);
            for (int b = 0; b < nbins; ++b) pt[b] += wp * nb[b];
            for (int m = 0; m <= mmax; ++m)
                for (int b1 = 0; b1 < nbins; ++b1)
                    for (int b2 = 0; b2 < nbins; ++b2) {
                        const double* x = a + ((size_t)b1 * M1 + m) * 2;
                        const double* y = a + ((size_t)b2 * M1 + m) * 2;
                        double s = x[0] * y[0] + x[1] * y[1];
                        size_t o = ((size_t)m * nbins + b1) * nbins + b2;
                        zt[o] += wp * s;
                        gt[o] += fabs(wp) * s;
                    }
        }
        free(a);
        free(nb);
    }
    for (size_t o = 0; o < zsz; ++o) {
        double s = 0.0, g = 0.0;
        for (int t = 0; t < nt; ++t) { s += zpart[(size_t)t * zsz + o]; g += gpart[(size_t)t * zsz + o]; }
        zeta[o] = s;
        if (gram) gram[o] = g;
    }
    if (wpairs)
        for (int b = 0; b < nbins; ++b) {
            double s = 0.0;
            for (int t = 0; t < nt; ++t) s += ppart[(size_t)t * nbins + b];
            wpairs[b] = s;
        }
    int64_t npairs = 0;
    for (int t = 0; t < nt; ++t) npairs += cnt[t];
    if (npairs_out) *npairs_out = npairs;
    free(edge); free(zpart); free(gpart); free(ppart); free(cnt);
    return 0;
}
