// edge.cu -- edge-corrected multipoles (Slepian & Eisenstein 2015).
//
// Paper, "Implementation": the estimator includes edge corrections; "Statement
// of need": the harmonic 3PCF after Slepian & Eisenstein.  With the sums
// S_l(b1,b2) = sum over triplets of P_l(mu) of a data-minus-randoms catalogue
// (N) and of its randoms alone (R, weights taken positive), the corrected
// 3PCF zeta(mu) = N(mu) / R(mu) has Legendre coefficients zeta_l that solve,
// per bin pair,
//     n_l / r_0 = sum_l' M_ll' zeta_l',   M_ll' = (2l+1) sum_l'' (l l' l''; 0 0 0)^2 f_l'',
// where n_l = (2l+1)/2 S_l(N), r_l = (2l+1)/2 S_l(R), f_l = r_l / r_0, all
// sums truncated at l_max.  One thread solves one bin pair's system in FP64
// by Gaussian elimination with partial pivoting.
#include <cmath>
#include <vector>

#include "ctb_internal.cuh"

namespace ctb {

// (a b c; 0 0 0)^2 from the closed form in log-gamma:
// zero unless a+b+c = 2g is even and (a, b, c) a triangle, else
// (2g-2a)!(2g-2b)!(2g-2c)!/(2g+1)! * [g!/((g-a)!(g-b)!(g-c)!)]^2.
static double threej000_sq(int a, int b, int c) {
  if ((a + b + c) & 1) return 0.0;
  if (c < std::abs(a - b) || c > a + b) return 0.0;
  const int g = (a + b + c) / 2;
  auto lf = [](int n) { return std::lgamma((double)n + 1.0); };
  const double lg = lf(2 * g - 2 * a) + lf(2 * g - 2 * b) + lf(2 * g - 2 * c) - lf(2 * g + 1) +
                    2.0 * (lf(g) - lf(g - a) - lf(g - b) - lf(g - c));
  return std::exp(lg);
}

void make_threej_table(int lmax, std::vector<double>& t) {
  const int n = lmax + 1;
  t.assign((size_t)n * n * n, 0.0);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c) t[((size_t)a * n + b) * n + c] = threej000_sq(a, b, c);
}

constexpr int kEdgeN = kLmaxCap + 1;

__global__ void k_edge_correct(const double* __restrict__ zn, const double* __restrict__ zr,
                               const double* __restrict__ tj, int lmax, int nb, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb * nb) return;
  const int n = lmax + 1;
  const size_t plane = (size_t)nb * nb;
  double f[kEdgeN], rhs[kEdgeN], m[kEdgeN][kEdgeN];
  const double r0 = 0.5 * zr[t];  // (2*0+1)/2 S_0
  bool ok = r0 != 0.0 && isfinite(r0);
  for (int l = 0; l < n; ++l) {
    const double c = 0.5 * (2.0 * l + 1.0);
    f[l] = ok ? c * zr[l * plane + t] / r0 : 0.0;
    rhs[l] = ok ? c * zn[l * plane + t] / r0 : 0.0;
  }
  for (int l = 0; l < n; ++l)
    for (int lp = 0; lp < n; ++lp) {
      double s = 0.0;
      for (int lpp = 0; lpp < n; ++lpp) s += tj[((size_t)l * n + lp) * n + lpp] * f[lpp];
      m[l][lp] = (2.0 * l + 1.0) * s;
    }
  // Gaussian elimination with partial pivoting
  for (int k = 0; k < n && ok; ++k) {
    int piv = k;
    double best = fabs(m[k][k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(m[i][k]) > best) {
        best = fabs(m[i][k]);
        piv = i;
      }
    if (!(best > 0.0)) {
      ok = false;
      break;
    }
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        const double tmp = m[k][j];
        m[k][j] = m[piv][j];
        m[piv][j] = tmp;
      }
      const double tmp = rhs[k];
      rhs[k] = rhs[piv];
      rhs[piv] = tmp;
    }
    for (int i = k + 1; i < n; ++i) {
      const double q = m[i][k] / m[k][k];
      for (int j = k; j < n; ++j) m[i][j] -= q * m[k][j];
      rhs[i] -= q * rhs[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = rhs[k];
    for (int j = k + 1; j < n; ++j) s -= m[k][j] * rhs[j];
    rhs[k] = ok ? s / m[k][k] : NAN;
  }
  for (int l = 0; l < n; ++l) out[l * plane + t] = ok ? rhs[l] : NAN;
}

cudaError_t launch_edge_correct(const double* zn, const double* zr, const double* tj, int lmax, int nbins,
                                double* out, cudaStream_t st) {
  const int total = nbins * nbins;
  k_edge_correct<<<(total + 63) / 64, 64, 0, st>>>(zn, zr, tj, lmax, nbins, out);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ctb
