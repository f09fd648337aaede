"""Projected (angular) multipoles on the sphere: CUDA path vs the FP64 oracle.

Tolerance: the Gram-normalised metric of tests/parity.py at 1e-5 (FP32
accumulation; the Chebyshev recurrence's error grows like m^2 and stays
below it for m <= 16).
"""
import numpy as np
import pytest

import oracle
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


def run(ctbmod, xyz, w, kw, prim=None, **opts):
    est = ctbmod.CTB.sphere(kw["theta_min"], kw["theta_max"], kw["nbins"], kw["mmax"])
    for k, v in opts.items():
        est.set_option(getattr(ctbmod, "OPT_" + k.upper()), v)
    est.set_points(xyz, w)
    z = est.compute() if prim is None else est.compute_subset(prim)
    return z, est


@pytest.mark.parametrize("centre", [(0.2, -0.3, 0.93), (0.0, 0.0, 1.0), (1.0, 0.0, 0.0)])
def test_cap_vs_oracle(ctbmod, centre):
    xyz = synth.sphere_cap(6000, seed=81, theta_cap=0.25, centre=centre)
    w = synth.sphere_field(xyz, seed=82, width=0.03)
    kw = dict(theta_min=0.004, theta_max=0.15, nbins=6, mmax=8)
    z, est = run(ctbmod, xyz, w, kw)
    ref = oracle.zeta_sphere(xyz, w, **kw)
    assert est.pair_count() == ref["npairs"]
    assert zeta_err(z, ref) < TOL
    np.testing.assert_allclose(est.pair_sums(), ref["wpairs"], rtol=1e-5, atol=1e-6 * np.abs(ref["wpairs"]).max())


@pytest.mark.parametrize("mmax,nbins", [(0, 1), (3, 4), (16, 5)])
def test_full_sky_subset_vs_oracle(ctbmod, mmax, nbins):
    xyz = synth.fibonacci_sphere(40_000)
    w = synth.sphere_field(xyz, seed=83)
    kw = dict(theta_min=0.0, theta_max=0.2, nbins=nbins, mmax=mmax)
    prim = synth.sample_primaries(xyz.shape[0], 300, seed=5)
    z, est = run(ctbmod, xyz, w, kw, prim=prim)
    ref = oracle.zeta_sphere(xyz, w, prim=prim, **kw)
    assert est.pair_count() == ref["npairs"]
    assert zeta_err(z, ref) < TOL


def test_grid_and_chunks_do_not_change_result(ctbmod):
    xyz = synth.sphere_cap(5000, seed=84, theta_cap=0.3, centre=(0.0, 0.01, 1.0))
    w = synth.sphere_field(xyz, seed=85, width=0.04)
    kw = dict(theta_min=0.01, theta_max=0.12, nbins=5, mmax=6)
    ref = oracle.zeta_sphere(xyz, w, **kw)
    for opts in (dict(cells_per_rmax=2), dict(cells_per_rmax=12, list_capacity=4096), dict(autotune=1)):
        z, est = run(ctbmod, xyz, w, kw, **opts)
        assert est.pair_count() == ref["npairs"]
        assert zeta_err(z, ref) < TOL


def frame(n):
    n = n / np.linalg.norm(n)
    rho = np.hypot(n[0], n[1])
    e = np.array([-n[1] / rho, n[0] / rho, 0.0]) if rho > 0 else np.array([0.0, 1.0, 0.0])
    return e, np.cross(n, e)


def test_get_alm_matches_the_documented_frame(ctbmod):
    xyz = synth.sphere_cap(3000, seed=86, theta_cap=0.2)
    w = synth.sphere_field(xyz, seed=87, width=0.03)
    kw = dict(theta_min=0.005, theta_max=0.1, nbins=3, mmax=5)
    est = ctbmod.CTB.sphere(kw["theta_min"], kw["theta_max"], kw["nbins"], kw["mmax"])
    est.set_points(xyz, w)
    prim = synth.sample_primaries(xyz.shape[0], 12, seed=6)
    a = est.get_alm(prim)
    assert a.shape == (12, 3, 11)
    edges = 2 * np.sin(0.5 * np.linspace(kw["theta_min"], kw["theta_max"], kw["nbins"] + 1))
    for i, p in enumerate(prim):
        d = xyz - xyz[p]
        c = np.linalg.norm(d, axis=1)
        ok = (c > 0) & (c >= edges[0]) & (c < edges[-1])
        b = np.searchsorted(edges, c, side="right") - 1
        e, nn = frame(xyz[p])
        phi = np.arctan2(d @ e, d @ nn)
        for bb in range(kw["nbins"]):
            s = ok & (b == bb)
            scale = np.abs(w[s]).sum() + 1e-30
            want = [w[s].sum()]
            for m in range(1, kw["mmax"] + 1):
                want += [np.sum(w[s] * np.cos(m * phi[s])), np.sum(w[s] * np.sin(m * phi[s]))]
            assert np.max(np.abs(a[i, bb] - np.array(want))) < 1e-5 * scale


def test_rotation_leaves_zeta_unchanged(ctbmod):
    xyz = synth.fibonacci_sphere(30_000)
    w = synth.sphere_field(xyz, seed=88)
    kw = dict(theta_min=0.01, theta_max=0.15, nbins=4, mmax=6)
    z0, _ = run(ctbmod, xyz, w, kw)
    q, _ = np.linalg.qr(np.random.default_rng(10).normal(size=(3, 3)))
    z1, _ = run(ctbmod, synth.snap_dyadic(xyz @ q.T), w, kw)
    ref = oracle.zeta_sphere(xyz, w, **kw)
    assert zeta_err(z0, ref) < TOL
    assert zeta_err(z1, ref) < 1e-3  # snapping the rotated points moves a few pairs across edges


def test_sphere_mode_errors(ctbmod):
    with pytest.raises(ctbmod.CTBError):
        ctbmod.CTB.sphere(0.1, 0.05, 3, 4)
    with pytest.raises(ctbmod.CTBError):
        ctbmod.CTB.sphere(0.0, 0.1, 3, ctbmod.MMAX_CAP + 1)
    est = ctbmod.CTB.sphere(0.0, 0.1, 3, 4)
    with pytest.raises(ctbmod.CTBError) as e:
        est.set_option(ctbmod.OPT_PRECISION, ctbmod.PREC_BF16X3)
    assert e.value.code == ctbmod.ERR_UNSUPPORTED
    xyz = synth.fibonacci_sphere(1000)
    with pytest.raises(ctbmod.CTBError) as e:
        est.compute_batch([(xyz, None)])
    assert e.value.code == ctbmod.ERR_UNSUPPORTED
    z = np.zeros(est.zeta_shape)
    with pytest.raises(ctbmod.CTBError) as e:
        est.edge_correct(z, z)
    assert e.value.code == ctbmod.ERR_UNSUPPORTED


@pytest.mark.parametrize("cpr", [2, 6, 16])
def test_points_off_the_unit_sphere(ctbmod, cpr):
    """Directions scaled by 0.8-1.2: the rows are cut to the shell the points
    occupy, and no pair may be lost at any grid size."""
    xyz = synth.sphere_cap(5000, seed=89, theta_cap=0.3, centre=(0.3, 0.5, 0.81))
    xyz = synth.snap_dyadic(xyz * np.random.default_rng(90).uniform(0.8, 1.2, (xyz.shape[0], 1)))
    w = synth.sphere_field(xyz / np.linalg.norm(xyz, axis=1, keepdims=True), seed=91, width=0.04)
    kw = dict(theta_min=0.002, theta_max=0.2, nbins=6, mmax=6)
    z, est = run(ctbmod, xyz, w, kw, cells_per_rmax=cpr)
    ref = oracle.zeta_sphere(xyz, w, **kw)
    assert est.pair_count() == ref["npairs"]
    assert zeta_err(z, ref) < TOL
