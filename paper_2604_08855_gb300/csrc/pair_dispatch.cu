// pair_dispatch.cu -- coefficient layout, recurrence constants, and the
// ell_max dispatch of the pair-multipole kernel.
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "ctb_internal.cuh"

namespace ctb {

// explicit instantiations live in pair_[a-f].cu
template <int L>
cudaError_t launch_alm_L(const AlmArgs&, int, int, cudaStream_t);
template <int L>
int alm_occupancy_L(int);

void make_layout(int L, Layout* out) {
  Layout& y = *out;
  y.L = L;
  y.npass = 0;
  int base = 0;
  for (int i = 0; i < (kLmaxCap + 1) * (kLmaxCap + 1); ++i) y.slot[i] = -1;
  for (int m0 = 0; m0 <= L;) {
    int m1 = pass_end(L, m0, pass_cap(L, m0));
    int ncp = round32(coef_count(L, m0, m1));
    y.m0[y.npass] = m0;
    y.m1[y.npass] = m1;
    y.base[y.npass] = base;
    y.ncp[y.npass] = ncp;
    for (int l = m0; l <= L; ++l) {
      int hi = l < m1 ? l : m1;
      for (int m = -hi; m <= hi; ++m) {
        int am = m < 0 ? -m : m;
        if (am < m0) continue;
        y.slot[l * l + l + m] = base + local_slot(L, l, m, m0, m1);
      }
    }
    base += ncp;
    ++y.npass;
    m0 = m1 + 1;
  }
  y.row = base;
}

// a_lm = sqrt((4l^2-1)/(l^2-m^2)),  b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)):
// the normalised associated-Legendre recurrence  Pbar_l = a (z Pbar_{l-1} - b Pbar_{l-2}).
static double rec_a(int l, int m) { return std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m)); }
static double rec_b(int l, int m) {
  return std::sqrt((((double)(l - 1) * (l - 1)) - (double)m * m) / (4.0 * (l - 1) * (l - 1) - 1.0));
}

// Monic form p_l = z p_{l-1} - beta p_{l-2}:  beta_lm = b_lm / a_{l-1,m}.
void fill_beta(float* beta) {
  for (int i = 0; i < (kLmaxCap + 1) * (kLmaxCap + 1); ++i) beta[i] = 0.f;
  for (int m = 0; m <= kLmaxCap; ++m)
    for (int l = m + 2; l <= kLmaxCap; ++l) beta[l * (kLmaxCap + 1) + m] = (float)(rec_b(l, m) / rec_a(l - 1, m));
}

// Normalisation C_lm turning the monic p_l^m times Re/Im (x+iy)^m into the
// real orthonormal Y_l,+-m (Condon-Shortley phase and sqrt 2 for m != 0):
//   C_mm = (-1)^m / sqrt(4 pi) prod_{k=1..m} sqrt((2k+1)/(2k)),
//   C_lm = C_mm prod_{k=m+1..l} a_km.
double norm_lm(int l, int m) {
  int am = m < 0 ? -m : m;
  double c = 1.0 / std::sqrt(4.0 * M_PI);
  for (int k = 1; k <= am; ++k) c *= -std::sqrt((2.0 * k + 1.0) / (2.0 * k));
  for (int k = am + 1; k <= l; ++k) c *= rec_a(k, am);
  if (am != 0) c *= M_SQRT2;
  return c;
}

// T-basis coefficients of the monic recurrence polynomial p_l^m(z) (degree
// l - m): p_m = 1, p_{m+1} = z, p_l = z p_{l-1} - beta_lm p_{l-2}, with
// z T_0 = T_1 and z T_k = (T_{k+1} + T_{k-1}) / 2.
static std::vector<double> monic_in_T(int l, int m) {
  const int n = l - m;
  std::vector<double> p2(n + 2, 0.0), p1(n + 2, 0.0);
  p2[0] = 1.0;  // p_m
  if (n == 0) return std::vector<double>(p2.begin(), p2.begin() + 1);
  p1[1] = 1.0;  // p_{m+1} = z = T_1
  for (int ll = m + 2; ll <= l; ++ll) {
    std::vector<double> zp(n + 2, 0.0);
    for (int k = 0; k <= n; ++k) {
      if (p1[k] == 0.0) continue;
      if (k == 0) {
        zp[1] += p1[0];
      } else {
        zp[k + 1] += 0.5 * p1[k];
        zp[k - 1] += 0.5 * p1[k];
      }
    }
    const double beta = rec_b(ll, m) / rec_a(ll - 1, m);
    for (int k = 0; k <= n; ++k) zp[k] -= beta * p2[k];
    p2 = p1;
    p1 = zp;
  }
  return std::vector<double>(p1.begin(), p1.begin() + n + 1);
}

// Coefficients D of p^m_l in the basis q_k = p^{m0}_{m0+k} (k <= l - m):
// p^m_l = sum_k D_k q_k, by back substitution on the T-basis coefficients
// (q_k has degree k with a nonzero T_k coefficient).
static std::vector<double> monic_in_basis(int l, int m, int m0) {
  const int n = l - m;
  const std::vector<double> target = monic_in_T(l, m);
  std::vector<std::vector<double>> q(n + 1);
  for (int k = 0; k <= n; ++k) q[k] = monic_in_T(m0 + k, m0);
  std::vector<double> r(target), d(n + 1, 0.0);
  for (int k = n; k >= 0; --k) {
    d[k] = r[k] / q[k][k];
    for (int j = 0; j <= k; ++j) r[j] -= d[k] * q[k][j];
  }
  return d;
}

// Each pass accumulates moments S_{m,k} = sum w c_m q_k(z) of its columns in
// slot (m + k, +-m), q_k its basis: the Chebyshev T_k for the pass that
// starts at m = 0, else p^{m0}_{m0+k}.  Normalised a_lm = C_lm sum_k D_k S_{m,k},
// D the coefficients of p^m_l in that basis.
bool make_conversion(const Layout& lay, std::vector<int2>& tab) {
  const int L = lay.L;
  std::vector<std::vector<std::pair<int, float>>> ent(lay.row);
  for (int p = 0; p < lay.npass; ++p) {
    const int m0 = lay.m0[p];
    for (int am = m0; am <= lay.m1[p] && am <= L; ++am) {
      for (int l = am; l <= L; ++l) {
        const std::vector<double> d = m0 == 0 ? monic_in_T(l, am) : monic_in_basis(l, am, m0);
        double dmax = 0.0;
        for (double v : d) dmax = std::fmax(dmax, std::fabs(v));
        for (int sg = (am == 0 ? 1 : -1); sg <= 1; sg += 2) {
          const int m = sg * am;
          const int s = lay.slot[l * l + l + m];
          const double nrm = norm_lm(l, m);
          for (int k = 0; k <= l - am; ++k) {
            if (std::fabs(d[k]) <= 1e-13 * dmax) continue;  // the other parity: exactly zero
            const int sl = am + k;
            ent[s].push_back({lay.slot[sl * sl + sl + m], (float)(nrm * d[k])});
          }
        }
      }
    }
  }
  // padded, entry-major per pass; local slot numbers
  tab.clear();
  for (int p = 0; p < lay.npass; ++p) {
    const int E = conv_entries(L, lay.m0[p]), ncp = lay.ncp[p], base = lay.base[p];
    const size_t t0 = tab.size();
    tab.resize(t0 + (size_t)E * ncp);
    for (int sl = 0; sl < ncp; ++sl) {
      const auto& v = ent[base + sl];
      if ((int)v.size() > E) return false;
      for (int e = 0; e < E; ++e) {
        int2 t;
        if (e < (int)v.size()) {
          t.x = v[e].first - base;
          float cf = v[e].second;
          std::memcpy(&t.y, &cf, 4);
        } else {
          t.x = sl;
          t.y = 0;  // +0.0f
        }
        tab[t0 + (size_t)e * ncp + sl] = t;
      }
    }
  }
  return true;
}

int alm_blocks_per_sm(int L, int wpb) {
  switch (L) {
#define CASE(X) \
  case X:       \
    return alm_occupancy_L<X>(wpb);
    CASE(0) CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
    CASE(12) CASE(14) CASE(16) CASE(18) CASE(20)
#undef CASE
    default:
      return 0;
  }
}

cudaError_t launch_alm(const AlmArgs& a, int L, int wpb, int nsm, cudaStream_t st) {
  switch (L) {
#define CASE(X) \
  case X:       \
    return launch_alm_L<X>(a, wpb, nsm, st);
    CASE(0) CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
    CASE(12) CASE(14) CASE(16) CASE(18) CASE(20)
#undef CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace ctb
