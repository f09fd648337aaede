// pair_dispatch.cu -- coefficient layout, recurrence constants, and the
// ell_max dispatch of the pair-multipole kernel.
#include <cmath>
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
        y.slot[l * l + l + m] = base + local_slot(l, m, m0, m1);
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

// Columns m <= cheb_max_m(L) hold Chebyshev moments S_{m,k} = sum w c_m T_k(z)
// in slot (m + k, +-m); the others hold Legendre sums in slot (l, +-m).
void make_conversion(const Layout& lay, std::vector<int>& off, std::vector<int>& src, std::vector<float>& coef) {
  const int L = lay.L;
  const int MC = L <= 10 ? L : 3;
  std::vector<std::vector<std::pair<int, float>>> ent(lay.row);
  for (int l = 0; l <= L; ++l) {
    for (int m = -l; m <= l; ++m) {
      const int am = m < 0 ? -m : m;
      const int s = lay.slot[l * l + l + m];
      const double nrm = norm_lm(l, m);
      if (am <= MC) {
        const std::vector<double> c = monic_in_T(l, am);
        for (int k = 0; k <= l - am; ++k) {
          const int sl = am + k, srcm = m;
          ent[s].push_back({lay.slot[sl * sl + sl + srcm], (float)(nrm * c[k])});
        }
      } else {
        ent[s].push_back({s, (float)nrm});
      }
    }
  }
  off.assign(lay.row + 1, 0);
  src.clear();
  coef.clear();
  for (int s = 0; s < lay.row; ++s) {
    off[s] = (int)src.size();
    for (auto& e : ent[s]) {
      src.push_back(e.first);
      coef.push_back(e.second);
    }
  }
  off[lay.row] = (int)src.size();
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
