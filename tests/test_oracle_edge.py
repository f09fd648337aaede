"""Pins of the oracle's edge correction (CPU only).

- the 3j symbols against sympy's Wigner 3j (exact rationals);
- an exact case: zeta(mu) and R(mu) Legendre series of low degree, N = zeta R
  formed with numpy's Legendre product; the solve must return zeta;
- no edges (R flat in mu): the correction is the plain ratio n_l / r_0;
- the normalisation against a direct quadrature of N / R.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import edge


def sums_from_coeffs(c, L):
    """Our sums S_l = 2/(2l+1) c_l of a Legendre series, padded to l <= L."""
    c = np.pad(np.asarray(c, float), (0, max(0, L + 1 - len(c))))[: L + 1]
    ell = np.arange(L + 1)
    return 2.0 / (2 * ell + 1) * c


def test_threej_matches_sympy():
    sympy = pytest.importorskip("sympy")
    from sympy.physics.wigner import wigner_3j
    for a in range(0, 9):
        for b in range(0, 9):
            for c in range(0, 17):
                want = float(wigner_3j(a, b, c, 0, 0, 0))
                assert edge.threej_000(a, b, c) == pytest.approx(want, rel=1e-13, abs=1e-15), (a, b, c)


def test_threej_selection_rules_and_orthogonality():
    # odd sum or broken triangle: zero
    assert edge.threej_000(1, 1, 1) == 0.0
    assert edge.threej_000(1, 2, 4) == 0.0
    # sum_c (2c+1) (a b c; 000)^2 = 1 (completeness)
    for a in range(6):
        for b in range(6):
            s = sum((2 * c + 1) * edge.threej_000(a, b, c) ** 2 for c in range(a + b + 1))
            assert s == pytest.approx(1.0, rel=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_legendre_quotient_is_recovered(seed):
    rng = np.random.default_rng(seed)
    L = 6
    zc = rng.normal(size=3)                        # zeta(mu), degree 2
    rc = np.array([1.0, 0.3, -0.2, 0.1])           # R(mu) > 0 on [-1, 1], degree 3
    rc[1:] *= rng.uniform(0.5, 1.0, size=3)
    nc = npleg.legmul(zc, rc)                      # N = zeta R, degree 5 <= L
    zn = sums_from_coeffs(nc, L)[:, None, None] * np.ones((1, 2, 2))
    zr = sums_from_coeffs(rc, L)[:, None, None] * np.ones((1, 2, 2))
    got = edge.edge_correct(zn, zr)
    want = np.pad(zc, (0, L + 1 - len(zc)))
    for b1 in range(2):
        for b2 in range(2):
            np.testing.assert_allclose(got[:, b1, b2], want, rtol=0, atol=1e-12)


def test_flat_randoms_give_the_plain_ratio():
    L = 4
    rng = np.random.default_rng(5)
    zn = rng.normal(size=(L + 1, 3, 3))
    zr = np.zeros((L + 1, 3, 3))
    zr[0] = 2.0 * 7.0  # R(mu) = 7 flat: S_0 = 14, S_l>0 = 0
    got = edge.edge_correct(zn, zr)
    ell = np.arange(L + 1)[:, None, None]
    np.testing.assert_allclose(got, (2 * ell + 1) / 2.0 * zn / 7.0, rtol=1e-14, atol=1e-14)


def test_against_quadrature_of_the_ratio():
    # N(mu) = zeta(mu) R(mu) with zeta degree 1 and R degree 2: the corrected
    # coefficients are the Legendre projections of N/R
    L = 4
    zc = np.array([0.5, -1.25])
    rc = np.array([2.0, 0.5, 0.25])
    nc = npleg.legmul(zc, rc)
    zn = sums_from_coeffs(nc, L)[:, None, None]
    zr = sums_from_coeffs(rc, L)[:, None, None]
    got = edge.edge_correct(zn, zr)[:, 0, 0]
    x, wq = npleg.leggauss(40)
    ratio = npleg.legval(x, nc) / npleg.legval(x, rc)
    proj = [(2 * l + 1) / 2.0 * np.sum(wq * ratio * npleg.legval(x, np.eye(L + 1)[l])) for l in range(L + 1)]
    np.testing.assert_allclose(got, proj, atol=1e-12)


def test_empty_random_bin_is_nan():
    zn = np.ones((3, 1, 1))
    zr = np.zeros((3, 1, 1))
    assert np.isnan(edge.edge_correct(zn, zr)).all()
