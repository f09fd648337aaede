"""CUDA path vs the FP64 oracle on inputs OFF the library's fixed-point grid.

ctb_set_points takes any float64 coordinates and rounds them onto its
fixed-point grid (box / 2^32 in a periodic cube; a power-of-two unit of at
most twice extent / 2^31 in open space).  A pair whose separation lies
within that rounding of a bin edge may then be binned on the other side of
the edge from the oracle, which bins the exact float64 separation.  The
oracle lists those edge-ambiguous pairs (oracle.ambiguous), and each test
grants exactly their worst-case effect (tests/parity.py bin_flip_bound):

  pair counts   |n_gpu - n_oracle| <= ambiguous pairs at r_min or r_max
  zeta          |dzeta| <= 1e-5 s + flip bound   (s the Gram scale)
  pair sums     |dDD| <= 1e-5 |DD| + flip bound

Every other difference (the rounded directions, FP32 arithmetic) is inside
the FP32 tolerance.  The two secondary metrics (plain relative error over
the entries above 1e-3 of the largest, and the per-l normwise error) are
reported beside the Gram metric and held to the bounds stated below.
"""
import numpy as np
import pytest

import oracle
from paper_2604_08855_gb300 import synth
from tests.parity import (bin_flip_bound, zeta_err, zeta_err_elementwise, zeta_err_normwise,
                          zeta_err_with_flips)

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_MIXED = 1e-3
# Secondary metrics: the per-l normwise error shares the Gram metric's scale
# on these catalogues (positive weights: the diagonal's self terms set
# max |zeta_l|), so it is held to the same tolerance; the plain relative
# error over entries above 1e-3 of the largest may exceed it by the ratio of
# the Gram scale to the entry (at most 1e3), and is held to 1e-3.
TOL_NORMWISE = 1e-5
TOL_ELEMENTWISE = 1e-3


@pytest.fixture(scope="module")
def ctbmod():
    from paper_2604_08855_gb300 import build
    build.build()
    from paper_2604_08855_gb300 import ctb
    return ctb


def unit_bound(xyz, box):
    """Largest grid unit the library may round these coordinates onto."""
    if box > 0:
        return box / 2.0 ** 32
    ext = float(np.max(xyz.max(axis=0) - xyz.min(axis=0)))
    return 2.0 * max(ext, 1e-300) / (2.0 ** 31 - 1024)


def check(ctbmod, xyz, w, kw, prim=None, precision=None, tol=TOL_FP32, label=""):
    est = ctbmod.CTB(kw["box"], kw["rmin"], kw["rmax"], kw["nbins"], kw["lmax"])
    if precision is not None:
        est.set_option(ctbmod.OPT_PRECISION, precision)
    est.set_points(xyz, w)
    z = est.compute() if prim is None else est.compute_subset(prim)
    # edge-ambiguous pairs: within 4 grid units of an edge (the separation's
    # rounding is below sqrt(3) units)
    amb_tol = 4.0 * unit_bound(xyz, kw["box"]) / kw["rmin"]
    ref = oracle.zeta(xyz, w, prim=prim, amb_tol=amb_tol, **kw)
    amb = oracle.ambiguous(xyz, kw["box"], kw["rmin"], kw["rmax"], kw["nbins"], amb_tol, prim=prim)
    assert len(amb[0]) == ref["namb"]
    bz, bp, outer = bin_flip_bound(xyz, w, kw, prim, amb)
    gram = zeta_err(z, ref)
    err = zeta_err_with_flips(z, ref, bz)
    elem = zeta_err_elementwise(z, ref)
    normw = zeta_err_normwise(z, ref)
    print(f"\n[{label}] pairs {ref['npairs']} ambiguous {ref['namb']} (outer {outer}): "
          f"gram {gram:.2e}  gram after flip bound {err:.2e}  elementwise {elem:.2e}  normwise {normw:.2e}")
    assert abs(est.pair_count() - ref["npairs"]) <= outer
    assert err < tol
    wp = ref["wpairs"]
    assert np.all(np.abs(est.pair_sums() - wp) <= 1e-5 * np.abs(wp) + bp + 1e-12)
    if ref["namb"] == 0:
        assert est.pair_count() == ref["npairs"]
        assert gram < tol
        if tol == TOL_FP32:
            assert normw < TOL_NORMWISE
            assert elem < TOL_ELEMENTWISE
    est.close()
    return ref


def test_offgrid_uniform_20k_periodic(ctbmod):
    """C1's workload with raw float64 draws: 20,000 uniform points, L = 1000."""
    xyz, w = synth.uniform(20_000, 1000.0, seed=0, snap=False)
    kw = synth.config_params(1)
    check(ctbmod, xyz, w, kw, label="uniform 20k L=1000")


@pytest.mark.parametrize("box", [250.0, 333.3])
def test_offgrid_thomas_periodic_odd_box(ctbmod, box):
    """A box side that is not a short binary mantissa: no float64 value is on
    the box / 2^32 grid except by chance."""
    xyz, w = synth.thomas(8000, box, 80, 5.0, seed=61, weights="u0.5-1.5", snap=False)
    kw = dict(box=box, rmin=2.0, rmax=40.0, nbins=8, lmax=10)
    check(ctbmod, xyz, w, kw, label=f"thomas periodic L={box}")


def test_offgrid_thomas_open(ctbmod):
    """Open space: the same kind of catalogue without wrap, shifted off zero."""
    xyz, w = synth.thomas(6000, 400.0, 60, 5.0, seed=62, weights="u0.5-1.5", snap=False)
    xyz = xyz + np.array([-123.456789, 17.1, 1000.0 / 3.0])
    kw = dict(box=0.0, rmin=2.0, rmax=60.0, nbins=7, lmax=10)
    check(ctbmod, xyz, w, kw, label="thomas open")


def test_offgrid_cut_sky_subset(ctbmod):
    """The cut-sky sector (data w = +1, randoms w = -1/3) without snapping,
    on seeded primaries with all points as secondaries."""
    d = synth.sector_data(60_000, seed=63, snap=False)
    r = synth.sector_randoms(180_000, seed=64, snap=False)
    xyz = np.vstack([d, r])
    w = np.concatenate([np.ones(d.shape[0]), -np.full(r.shape[0], 1.0 / 3.0)])
    kw = dict(box=0.0, rmin=20.0, rmax=120.0, nbins=10, lmax=10)
    prim = synth.sample_primaries(xyz.shape[0], 256, seed=65)
    check(ctbmod, xyz, w, kw, prim=prim, label="cut sky 240k, 256 primaries")


def test_offgrid_lmax20_multipass(ctbmod):
    xyz, w = synth.thomas(3000, 300.0, 30, 5.0, seed=66, weights="u0.5-1.5", snap=False)
    kw = dict(box=300.0, rmin=3.0, rmax=50.0, nbins=5, lmax=20)
    check(ctbmod, xyz, w, kw, label="thomas l_max 20")


def test_offgrid_mixed_precision(ctbmod):
    xyz, w = synth.thomas(8000, 250.0, 80, 5.0, seed=67, weights="u0.5-1.5", snap=False)
    kw = dict(box=250.0, rmin=2.0, rmax=40.0, nbins=8, lmax=10)
    check(ctbmod, xyz, w, kw, precision=ctbmod.PREC_BF16X3, tol=TOL_MIXED, label="thomas BF16x3")


def test_offgrid_sphere_cap(ctbmod):
    """Exact unit vectors (not on the dyadic grid) in a cap.  The angle bins
    are decided on the chord, so a pair whose chord lies within 4 grid units
    of an edge chord may be binned on either side.  Those pairs are found
    here by brute force, and each is granted its worst case: moving w_j
    between two bins changes a_m(p, b) by |w_j| in those bins only, so
    |dzeta_m(b1, b2)| <= |w_p| |w_j| ([b1 moved] (A_p(b2) + |w_j|) +
    [b2 moved] (A_p(b1) + |w_j|)), with A_p(b) the primary's |w| sum in bin b
    (the oracle's pair sums with |w| and a unit primary weight)."""
    xyz = synth.sphere_cap(6000, seed=84, theta_cap=0.25, snap=False)
    w = synth.sphere_field(xyz, seed=85, width=0.03)
    kw = dict(theta_min=0.004, theta_max=0.15, nbins=6, mmax=8)
    nb = kw["nbins"]
    edges = kw["theta_min"] + np.arange(nb + 1) * (kw["theta_max"] - kw["theta_min"]) / nb
    chords = 2.0 * np.sin(edges / 2.0)
    tol = 4.0 * unit_bound(xyz, 0.0)
    bz = np.zeros((kw["mmax"] + 1, nb, nb))
    outer = 0
    for i0 in range(0, xyz.shape[0], 500):
        c = np.linalg.norm(xyz[i0:i0 + 500, None, :] - xyz[None, :, :], axis=2)
        near = np.abs(c[..., None] - chords) < tol
        for pi, j, k in zip(*np.nonzero(near)):
            p = i0 + int(pi)
            if p == j:
                continue
            outer += int(k == 0 or k == nb)
            moved = [b for b in (k - 1, k) if 0 <= b < nb]
            A = oracle.zeta_sphere(xyz, np.abs(w), prim=np.array([p]), wprim=np.array([1.0]), **kw)["wpairs"]
            for b1 in range(nb):
                for b2 in range(nb):
                    t = (b1 in moved) * (A[b2] + abs(w[j])) + (b2 in moved) * (A[b1] + abs(w[j]))
                    bz[:, b1, b2] += abs(w[p] * w[j]) * t
    est = ctbmod.CTB.sphere(kw["theta_min"], kw["theta_max"], nb, kw["mmax"])
    est.set_points(xyz, w)
    z = est.compute()
    ref = oracle.zeta_sphere(xyz, w, **kw)
    err = zeta_err_with_flips(z, ref, bz)
    print(f"\n[sphere cap] pairs {ref['npairs']} ambiguous {int(np.count_nonzero(bz[0]) > 0)}+ (outer {outer}): "
          f"gram {zeta_err(z, ref):.2e}  gram after flip bound {err:.2e}")
    assert abs(est.pair_count() - ref["npairs"]) <= outer
    assert err < TOL_FP32
    est.close()
