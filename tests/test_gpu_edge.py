"""Edge correction on the GPU (ctb_edge_correct) against the oracle's.

1. The device solve on the same inputs as the oracle: an exact Legendre
   quotient (the solve must return zeta) and generic inputs (FP64 both sides).
2. End to end on a small sector catalogue with an open boundary: zeta of
   data-minus-randoms and of the randoms from the CUDA path, corrected on the
   GPU, against the same chain in the oracle.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle
from oracle import edge as oedge
from paper_2604_08855_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctbmod():
    from paper_2604_08855_gb300 import build
    build.build()
    from paper_2604_08855_gb300 import ctb
    return ctb


def sums(c, L):
    c = np.pad(np.asarray(c, float), (0, max(0, L + 1 - len(c))))[: L + 1]
    return 2.0 / (2 * np.arange(L + 1) + 1) * c


def test_device_solve_recovers_an_exact_quotient(ctbmod):
    L, nb = 6, 3
    est = ctbmod.CTB(100.0, 1.0, 10.0, nb, L)
    rng = np.random.default_rng(11)
    zn = np.zeros((L + 1, nb, nb))
    zr = np.zeros((L + 1, nb, nb))
    want = np.zeros((L + 1, nb, nb))
    for b1 in range(nb):
        for b2 in range(nb):
            zc = rng.normal(size=3)
            rc = np.array([1.0, 0.3, -0.2, 0.1]) * np.r_[1.0, rng.uniform(0.5, 1.0, 3)]
            zn[:, b1, b2] = sums(npleg.legmul(zc, rc), L)
            zr[:, b1, b2] = sums(rc, L)
            want[:3, b1, b2] = zc
    got = est.edge_correct(zn, zr)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-11)
    np.testing.assert_allclose(got, oedge.edge_correct(zn, zr), rtol=0, atol=1e-11)


def test_device_solve_matches_oracle_and_flags_empty_bins(ctbmod):
    import torch
    L, nb = 10, 4
    est = ctbmod.CTB(100.0, 1.0, 10.0, nb, L)
    rng = np.random.default_rng(12)
    zr = np.zeros((L + 1, nb, nb))
    for b1 in range(nb):
        for b2 in range(nb):
            rc = np.r_[1.0, 0.4 * rng.uniform(-1, 1, 4)] * rng.uniform(1e3, 1e5)
            zr[:, b1, b2] = sums(rc, L)
    zn = rng.normal(size=(L + 1, nb, nb)) * 1e3
    zr[:, 0, 3] = 0.0  # no random triplets in this bin pair
    ref = oedge.edge_correct(zn, zr)
    got = est.edge_correct(zn, zr)
    assert np.isnan(got[:, 0, 3]).all() and np.isnan(ref[:, 0, 3]).all()
    ok = ~np.isnan(ref)
    np.testing.assert_allclose(got[ok], ref[ok], rtol=1e-9, atol=1e-9 * np.abs(ref[ok]).max())
    # device pointers in and out
    d = torch.device("cuda")
    out = torch.zeros(est.zeta_shape, dtype=torch.float64, device=d)
    est.edge_correct(torch.from_numpy(zn).to(d), torch.from_numpy(zr).to(d), out=out)
    np.testing.assert_array_equal(out.cpu().numpy(), got)


def test_edge_corrected_sector_end_to_end(ctbmod):
    n_d, n_r = 3000, 9000
    d = synth.sector_data(n_d, seed=71)
    r = synth.sector_randoms(n_r, seed=72)
    alpha = n_d / n_r
    xyz = np.concatenate([d, r])
    w_nnn = np.concatenate([np.ones(n_d), np.full(n_r, -alpha)])
    w_rrr = np.full(n_r, alpha)
    kw = dict(box=0.0, rmin=20.0, rmax=200.0, nbins=4, lmax=4)
    est = ctbmod.CTB(**kw)
    est.set_points(xyz, w_nnn)
    zn = est.compute()
    est.set_points(r, w_rrr)
    zr = est.compute()
    got = est.edge_correct(zn, zr)
    ref = oedge.edge_correct(oracle.zeta(xyz, w_nnn, **kw)["zeta"], oracle.zeta(r, w_rrr, **kw)["zeta"])
    ok = ~np.isnan(ref)
    assert ok.any() and np.array_equal(ok, ~np.isnan(got))
    scale = np.abs(ref[ok]).max()
    assert np.max(np.abs(got[ok] - ref[ok])) < 1e-3 * scale
