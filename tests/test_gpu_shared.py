"""Shared neighbour lists for close pivots: CUDA path vs the FP64 oracle.

- parity with oracle.shared.zeta_shared: the Gram-normalised metric of
  tests/parity.py at 1e-5 (FP32 accumulation), same group count;
- the stated bound: |shared - exact oracle| <= shared_bound + 1e-5 x scale;
- one-point groups reproduce the exact oracle; the automatic cell side is
  the mean separation;
- the sphere mode (parity with the oracle's shared estimate, and the sphere
  bound against the exact oracle), the shared 2PCF, and the argument errors.
"""
import numpy as np
import pytest

import oracle
from oracle import shared
from paper_2604_08855_gb300 import synth
from tests.parity import zeta_err

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def ctbmod():
    from paper_2604_08855_gb300 import build
    build.build()
    from paper_2604_08855_gb300 import ctb
    return ctb


def gram_scale(ref):
    g = ref["gram"]
    return np.sqrt(np.einsum("lii,ljj->lij", g, g))


@pytest.mark.parametrize("box", [150.0, 0.0])
@pytest.mark.parametrize("hfac", [0.5, 1.0, 2.5])
def test_shared_vs_oracle(ctbmod, box, hfac):
    xyz, w = synth.thomas(6000, 150.0, 60, 4.0, seed=601, weights="u0.5-1.5")
    if box == 0.0:
        xyz = synth.snap_dyadic(xyz)
    kw = dict(box=box, rmin=2.0, rmax=30.0, nbins=6, lmax=8)
    h = hfac * shared.mean_separation(xyz, box, kw["rmax"])
    est = ctbmod.CTB(box, kw["rmin"], kw["rmax"], kw["nbins"], kw["lmax"])
    est.set_option(ctbmod.OPT_CELLS_PER_RMAX, 4)
    est.set_points(xyz, w)
    z = est.compute_shared(h)
    ref = shared.zeta_shared(xyz, w, h=h, **kw)
    assert est.pivot_groups() == (h, ref["rep"].shape[0])
    assert ref["rep"].shape[0] < xyz.shape[0]
    assert est.pair_count() == ref["npairs"]
    assert zeta_err(z, ref) < TOL
    np.testing.assert_allclose(est.pair_sums(), ref["wpairs"], rtol=1e-5, atol=1e-6 * np.abs(ref["wpairs"]).max())
    if hfac == 1.0:
        # the stated error bound against the exact estimate
        exact = oracle.zeta(xyz, w, **kw)
        B = shared.shared_bound(xyz, w, h=h, **kw)
        dev = np.abs(z - exact["zeta"])
        assert np.all(dev <= B + TOL * gram_scale(exact))
        assert np.any(dev > 10 * TOL * gram_scale(exact))  # the approximation does change zeta


def test_singleton_groups_match_exact(ctbmod):
    xyz, w = synth.uniform(3000, 120.0, seed=602, weights="u0.5-1.5")
    kw = dict(box=120.0, rmin=3.0, rmax=25.0, nbins=5, lmax=6)
    h = 0.25
    _, rep, _ = shared.pivot_groups(xyz, h, 120.0)
    assert rep.shape[0] == 3000
    est = ctbmod.CTB(120.0, kw["rmin"], kw["rmax"], kw["nbins"], kw["lmax"])
    est.set_points(xyz, w)
    z = est.compute_shared(h)
    assert est.pivot_groups() == (h, 3000)
    ref = oracle.zeta(xyz, w, **kw)
    assert est.pair_count() == ref["npairs"]
    assert zeta_err(z, ref) < TOL


@pytest.mark.parametrize("h", [0.1, 0.02])  # 10^9 cells; 1.25e11 cells: 64-bit keys, two sort passes
def test_coincident_groups_match_exact(ctbmod, h):
    xyz, w1 = synth.thomas(2000, 100.0, 20, 3.0, seed=603, weights="u0.5-1.5")
    w2 = np.random.default_rng(604).uniform(-1.0, 1.0, 2000)
    xyz2 = np.concatenate([xyz, xyz])
    w = np.concatenate([w1, w2])
    kw = dict(box=100.0, rmin=1.0, rmax=20.0, nbins=5, lmax=6)
    est = ctbmod.CTB(100.0, kw["rmin"], kw["rmax"], kw["nbins"], kw["lmax"])
    est.set_points(xyz2, w)
    _, rep, W = shared.pivot_groups(xyz2, h, 100.0, w=w)
    assert np.array_equal(rep, np.arange(2000))   # each group is a point and its copy
    z = est.compute_shared(h)
    assert est.pivot_groups() == (h, 2000)
    ref = oracle.zeta(xyz2, w, **kw)
    assert zeta_err(z, ref) < TOL


@pytest.mark.parametrize("box", [200.0, 0.0])
def test_automatic_cell_is_mean_separation(ctbmod, box):
    xyz, w = synth.thomas(5000, 200.0, 50, 5.0, seed=605, weights="u0.5-1.5")
    if box == 0.0:
        xyz = synth.snap_dyadic(xyz)
    kw = dict(box=box, rmin=2.0, rmax=30.0, nbins=4, lmax=4)
    est = ctbmod.CTB(box, kw["rmin"], kw["rmax"], kw["nbins"], kw["lmax"])
    est.set_points(xyz, w)
    z = est.compute_shared(0.0)
    h, g = est.pivot_groups()
    assert h == pytest.approx(shared.mean_separation(xyz, box, kw["rmax"]), rel=1e-14)
    ref = shared.zeta_shared(xyz, w, h=h, **kw)
    assert g == ref["rep"].shape[0]
    assert zeta_err(z, ref) < TOL
    # the timing of the grouping stage is reported, and a plain compute clears it
    assert est.timings()[8] > 0
    est.compute()
    assert est.timings()[8] == 0


def test_shared_precision_modes(ctbmod):
    xyz, w = synth.thomas(5000, 150.0, 50, 4.0, seed=606, weights="u0.5-1.5")
    kw = dict(box=150.0, rmin=2.0, rmax=30.0, nbins=6, lmax=8)
    h = shared.mean_separation(xyz, 150.0)
    ref = shared.zeta_shared(xyz, w, h=h, **kw)
    for prec in ("BF16X3", "TF32"):
        est = ctbmod.CTB(150.0, kw["rmin"], kw["rmax"], kw["nbins"], kw["lmax"])
        est.set_option(ctbmod.OPT_PRECISION, getattr(ctbmod, "PREC_" + prec))
        est.set_points(xyz, w)
        assert zeta_err(est.compute_shared(h), ref) < 1e-3


def test_shared_sphere_vs_oracle(ctbmod):
    xyz = synth.snap_dyadic(synth.fibonacci_sphere(40_000))
    w = synth.sphere_field(xyz, seed=607)
    kw = dict(theta_min=0.005, theta_max=0.12, nbins=5, mmax=8)
    est = ctbmod.CTB.sphere(kw["theta_min"], kw["theta_max"], kw["nbins"], kw["mmax"])
    est.set_points(xyz, w)
    z = est.compute_shared(0.0)
    h, g = est.pivot_groups()
    assert h == pytest.approx(np.sqrt(4 * np.pi / xyz.shape[0]), rel=1e-14)
    ref = shared.zeta_shared_sphere(xyz, w, h=h, **kw)
    assert g == ref["rep"].shape[0]
    assert g < xyz.shape[0]
    assert est.pair_count() == ref["npairs"]
    assert zeta_err(z, ref) < TOL


def test_shared_sphere_within_stated_bound(ctbmod):
    """The projected multipoles: GPU shared estimate vs the exact oracle,
    within the sphere bound of oracle/shared.py."""
    xyz = synth.snap_dyadic(synth.sphere_cap(3000, seed=609, theta_cap=0.25, centre=(0.2, 0.4, 0.89)))
    w = synth.sphere_field(xyz / np.linalg.norm(xyz, axis=1, keepdims=True), seed=610, width=0.04)
    kw = dict(theta_min=0.005, theta_max=0.15, nbins=5, mmax=8)
    h = 0.02
    est = ctbmod.CTB.sphere(kw["theta_min"], kw["theta_max"], kw["nbins"], kw["mmax"])
    est.set_points(xyz, w)
    z = est.compute_shared(h)
    assert est.pivot_groups()[1] < xyz.shape[0]
    exact = oracle.zeta_sphere(xyz, w, **kw)
    B = shared.shared_bound_sphere(xyz, w, h=h, **kw)
    dev = np.abs(z - exact["zeta"])
    assert np.all(dev <= B + TOL * gram_scale(exact))
    assert np.any(dev > 10 * TOL * gram_scale(exact))


def test_shared_errors(ctbmod):
    est = ctbmod.CTB(100.0, 1.0, 20.0, 4, 4)
    z = np.zeros(est.zeta_shape)
    with pytest.raises(ctbmod.CTBError) as e:
        est.compute_shared(1.0, out=z)
    assert e.value.code == ctbmod.ERR_STATE
    xyz, w = synth.uniform(1000, 100.0, seed=608)
    est.set_points(xyz, w)
    with pytest.raises(ctbmod.CTBError) as e:
        est.pivot_groups()
    assert e.value.code == ctbmod.ERR_STATE
    for bad in (-1.0, float("nan"), float("inf"), 1e-5):  # 1e-5: (10^7)^3 cells > 2^64
        with pytest.raises(ctbmod.CTBError) as e:
            est.compute_shared(bad)
        assert e.value.code == ctbmod.ERR_ARG
    est.compute_shared(5.0)
    assert est.pivot_groups()[0] == 5.0
    est.set_points(xyz[:10], w[:10])
    with pytest.raises(ctbmod.CTBError):
        est.pivot_groups()
    est.set_points(xyz[:0], w[:0])
    assert not np.any(est.compute_shared(0.0))
    assert est.pivot_groups()[1] == 0
