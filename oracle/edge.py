"""Edge-corrected multipoles (Slepian & Eisenstein 2015) in FP64 numpy.

TEST INFRASTRUCTURE ONLY: only tests/ may call this module.  It shares no code
or table with the CUDA library.

The paper names the edge correction among its estimator's steps
("Implementation": edge corrections; "Statement of need": Slepian &
Eisenstein).  The reading taken here:

For one radial bin pair (b1, b2) let N(mu) be the triplet density of the
data-minus-randoms catalogue in mu = cos(angle between the two sides) and
R(mu) that of the randoms alone (same random weights, taken positive).  The
corrected 3PCF is zeta(mu) = N(mu) / R(mu).  Our sums are
S_l = sum_triplets P_l(mu) = int N(mu) P_l(mu) dmu, so the Legendre
coefficients of N (N(mu) = sum_l n_l P_l(mu)) are n_l = (2l+1)/2 S_l, and
likewise r_l for R.  Multiplying the expansions of zeta and R and projecting
with int P_a P_b P_c dmu = 2 (a b c; 0 0 0)^2 gives

    n_l / r_0 = sum_l' M_ll' zeta_l',   M_ll' = (2l+1) sum_l'' (l l' l''; 0 0 0)^2 f_l'',

with f_l = r_l / r_0, all sums truncated at l_max.  Solving this
(l_max+1) x (l_max+1) system per bin pair gives the Legendre coefficients
zeta_l of the corrected 3PCF (zeta(mu) = sum_l zeta_l P_l(mu)).

Parity status: pinned (tests/test_oracle_edge.py) by sympy's Wigner 3j
symbols and by exact Legendre products (numpy legmul) whose quotient the
solve must return.
"""
from __future__ import annotations

from math import factorial, sqrt

import numpy as np


def threej_000(a: int, b: int, c: int) -> float:
    """Wigner 3j symbol (a b c; 0 0 0) from its closed form with integer
    factorials: zero unless a+b+c is even and (a, b, c) is a triangle, else
    (-1)^g sqrt[(2g-2a)!(2g-2b)!(2g-2c)!/(2g+1)!] g!/((g-a)!(g-b)!(g-c)!)
    with 2g = a+b+c."""
    if (a + b + c) % 2 or c < abs(a - b) or c > a + b:
        return 0.0
    g = (a + b + c) // 2
    num = factorial(2 * g - 2 * a) * factorial(2 * g - 2 * b) * factorial(2 * g - 2 * c)
    den = factorial(2 * g + 1)
    pre = factorial(g) // (factorial(g - a) * factorial(g - b) * factorial(g - c))
    return (-1) ** g * sqrt(num / den) * pre


def coupling(f: np.ndarray) -> np.ndarray:
    """M_ll' = (2l+1) sum_l'' (l l' l''; 0 0 0)^2 f_l'' for l, l', l'' <= len(f)-1."""
    L = len(f) - 1
    m = np.zeros((L + 1, L + 1))
    for l in range(L + 1):
        for lp in range(L + 1):
            m[l, lp] = (2 * l + 1) * sum(threej_000(l, lp, lpp) ** 2 * f[lpp] for lpp in range(L + 1))
    return m


def edge_correct(zeta_n: np.ndarray, zeta_r: np.ndarray) -> np.ndarray:
    """Corrected Legendre coefficients [l][b1][b2] from the sums S_l of the
    data-minus-randoms catalogue (zeta_n) and of the randoms (zeta_r), both
    [l_max+1][nbins][nbins].  Bin pairs without random triplets (S_0 = 0) are
    NaN."""
    zn = np.asarray(zeta_n, dtype=np.float64)
    zr = np.asarray(zeta_r, dtype=np.float64)
    L = zn.shape[0] - 1
    ell = np.arange(L + 1)[:, None, None]
    n = (2 * ell + 1) / 2.0 * zn
    r = (2 * ell + 1) / 2.0 * zr
    out = np.full_like(zn, np.nan)
    for b1 in range(zn.shape[1]):
        for b2 in range(zn.shape[2]):
            r0 = r[0, b1, b2]
            if r0 == 0.0:
                continue
            m = coupling(r[:, b1, b2] / r0)
            out[:, b1, b2] = np.linalg.solve(m, n[:, b1, b2] / r0)
    return out
