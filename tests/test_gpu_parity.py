"""CUDA path vs the FP64 oracle, through the C ABI (GPU only).

Tolerance (FP32 pair kernel + FP32 contraction + FP64 reduction): 1e-5 on
the Gram-normalised metric of tests/parity.py, the FP32-mode bound the
estimator's accuracy target sets.  Inputs are the seeded synthetic
catalogues of paper_2604_08855_gb300.synth.
"""
import numpy as np
import pytest

import oracle
from paper_2604_08855_gb300 import synth
from tests.parity import alm_err, zeta_err

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
# Pair sums sum_p w_p sum_{j in b} w_j with positive weights: FP32 sums of at
# most a few thousand weights per (primary, bin) (relative error well under
# 1e-6 at random rounding), then FP64 over the primaries.
PAIRSUM_RTOL = 1e-5


@pytest.fixture(scope="module")
def ctbmod():
    from paper_2604_08855_gb300 import build
    build.build()
    from paper_2604_08855_gb300 import ctb
    return ctb


def make(ctbmod, box, rmin, rmax, nbins, lmax, **opts):
    est = ctbmod.CTB(box, rmin, rmax, nbins, lmax)
    for k, v in opts.items():
        est.set_option(getattr(ctbmod, "OPT_" + k.upper()), v)
    return est


def run_full(ctbmod, xyz, w, kw, **opts):
    est = make(ctbmod, **kw, **opts)
    est.set_points(xyz, w)
    z = est.compute()
    return z, est


# ----------------------------------------------------------------- small cases


@pytest.mark.parametrize("box", [400.0, 0.0])
@pytest.mark.parametrize("lmax", [0, 3, 10])
def test_small_thomas_vs_oracle(ctbmod, box, lmax):
    xyz, w = synth.thomas(4000, 400.0, 40, 5.0, seed=21, weights="u0.5-1.5")
    if box == 0.0:
        xyz = synth.snap_dyadic(xyz, 2.0 ** -16)
    kw = dict(box=box, rmin=2.0, rmax=60.0, nbins=7, lmax=lmax)
    z, est = run_full(ctbmod, xyz, w, kw)
    ref = oracle.zeta(xyz, w, **kw)
    assert est.pair_count() == ref["npairs"]
    assert zeta_err(z, ref) < TOL_FP32
    # the two-point pair sums of the same pass (a_00 column)
    np.testing.assert_allclose(est.pair_sums(), ref["wpairs"], rtol=PAIRSUM_RTOL)


def test_uniform_20k_full_vs_oracle(ctbmod):
    """20,000 uniform points, L = 1000, r in [10, 100], 10 bins, l_max = 10."""
    xyz, w = synth.uniform_20k()
    kw = synth.config_params(1)
    z, est = run_full(ctbmod, xyz, w, kw)
    ref = oracle.zeta(xyz, w, **kw)
    assert est.pair_count() == ref["npairs"]
    assert zeta_err(z, ref) < TOL_FP32


@pytest.mark.parametrize("lmax", [11, 12, 13, 14, 16, 17, 18, 20])
def test_multipass_lmax_vs_oracle(ctbmod, lmax):
    xyz, w = synth.thomas(3000, 300.0, 30, 5.0, seed=23, weights="u0.5-1.5")
    kw = dict(box=300.0, rmin=3.0, rmax=50.0, nbins=5, lmax=lmax)
    z, est = run_full(ctbmod, xyz, w, kw)
    ref = oracle.zeta(xyz, w, **kw)
    assert zeta_err(z, ref) < TOL_FP32


@pytest.mark.parametrize("prec", ["FP32", "BF16X3", "TF32"])
def test_caps_nbins64_lmax20_vs_oracle(ctbmod, prec):
    """The largest bin count and multipole order together, in every precision."""
    xyz, w = synth.thomas(2500, 200.0, 25, 6.0, seed=25, weights="u0.5-1.5")
    kw = dict(box=200.0, rmin=1.0, rmax=60.0, nbins=ctbmod.NBINS_CAP, lmax=ctbmod.LMAX_CAP)
    est = make(ctbmod, **kw)
    est.set_option(ctbmod.OPT_PRECISION, getattr(ctbmod, "PREC_" + prec))
    est.set_points(xyz, w)
    z = est.compute()
    ref = oracle.zeta(xyz, w, **kw)
    assert est.pair_count() == ref["npairs"]
    assert zeta_err(z, ref) < (TOL_FP32 if prec == "FP32" else 1e-3)


def test_alm_vs_oracle(ctbmod):
    xyz, w = synth.thomas(5000, 300.0, 50, 5.0, seed=24, weights="u0.5-1.5")
    kw = dict(box=300.0, rmin=2.0, rmax=45.0, nbins=6, lmax=10)
    est = make(ctbmod, **kw)
    est.set_points(xyz, w)
    prim = synth.sample_primaries(xyz.shape[0], 64, seed=3)
    a = est.get_alm(prim)
    a_ref = oracle.alm(xyz, w, prim=prim, **kw)
    w1 = oracle.alm(xyz, np.abs(w), prim=prim, **{**kw, "lmax": 0})[:, :, 0] * np.sqrt(4 * np.pi)
    assert alm_err(a, a_ref, w1, 10) < TOL_FP32


@pytest.mark.parametrize("cap", [0, 4096])
@pytest.mark.parametrize("cpr", [1, 3, 16])
def test_grid_and_list_capacity_do_not_change_result(ctbmod, cap, cpr):
    """Cell size and list capacity (4096 entries: hundreds of chunks of a few
    primaries, so chunk sizing, halving and bin-code buffer regrowth all run)."""
    xyz, w = synth.thomas(6000, 200.0, 30, 4.0, seed=25, weights="u0.5-1.5")
    kw = dict(box=200.0, rmin=1.0, rmax=40.0, nbins=4, lmax=4)
    z, est = run_full(ctbmod, xyz, w, kw, list_capacity=cap, cells_per_rmax=cpr)
    ref = oracle.zeta(xyz, w, **kw)
    assert est.pair_count() == ref["npairs"]
    assert zeta_err(z, ref) < TOL_FP32
    if cap:
        assert est.chunk_count() > 100


def test_autotune_picks_a_grid_and_keeps_the_result(ctbmod):
    xyz, w = synth.thomas(20000, 400.0, 100, 5.0, seed=31, weights="u0.5-1.5")
    kw = dict(box=400.0, rmin=2.0, rmax=60.0, nbins=8, lmax=6)
    plain = make(ctbmod, **kw)
    plain.set_points(xyz, w)
    assert plain.grid() == (8, int(np.floor(400.0 * 8 / 60.0)))
    est = make(ctbmod, **kw, autotune=1)
    est.set_points(xyz, w)
    k, nc = est.grid()
    assert k in (3, 4, 6, 8, 12, 16)
    assert nc == min(1024, int(np.floor(400.0 * k / 60.0)))
    z = est.compute()
    ref = oracle.zeta(xyz, w, **kw)
    assert est.pair_count() == ref["npairs"]
    assert zeta_err(z, ref) < TOL_FP32
    # the choice stays with the context for its next catalogue
    est.set_points(xyz[:10000], w[:10000])
    assert est.grid()[0] == k
    # an explicit cell size wins over the tuner
    fixed = make(ctbmod, **kw, autotune=1, cells_per_rmax=3)
    fixed.set_points(xyz, w)
    assert fixed.grid()[0] == 3


def test_list_capacity_below_one_primary_is_oom(ctbmod):
    xyz, w = synth.uniform(3000, 100.0, seed=26)
    est = make(ctbmod, box=100.0, rmin=1.0, rmax=45.0, nbins=3, lmax=2, list_capacity=4096)
    est.set_points(xyz, w)  # about 1130 neighbours per primary: fits
    est.compute()
    dense = np.concatenate([xyz, np.full((5000, 3), 50.0) + np.random.default_rng(3).uniform(-3, 3, (5000, 3))])
    est.set_points(dense, None)  # 5000 more points in a 6-unit cube: each of them has > 4096 pairs
    with pytest.raises(ctbmod.CTBError) as e:
        est.compute()
    assert e.value.code == ctbmod.ERR_OOM


def test_subset_and_partition(ctbmod):
    xyz, w = synth.thomas(5000, 300.0, 50, 5.0, seed=26, weights="u0.5-1.5")
    kw = dict(box=300.0, rmin=2.0, rmax=50.0, nbins=6, lmax=6)
    est = make(ctbmod, **kw)
    est.set_points(xyz, w)
    zfull = est.compute()
    perm = np.random.default_rng(0).permutation(xyz.shape[0])
    parts = [perm[:1000], perm[1000:3500], perm[3500:]]
    zs, ps = [], []
    for p in parts:
        zs.append(est.compute_subset(p))
        ps.append(est.pair_sums())
    ref = oracle.zeta(xyz, w, prim=parts[0], **kw)
    assert zeta_err(zs[0], ref) < TOL_FP32
    np.testing.assert_allclose(ps[0], ref["wpairs"], rtol=PAIRSUM_RTOL)
    reff = oracle.zeta(xyz, w, **kw)
    assert zeta_err(sum(zs), reff) < TOL_FP32
    assert zeta_err(zfull, reff) < TOL_FP32
    np.testing.assert_allclose(sum(ps), reff["wpairs"], rtol=PAIRSUM_RTOL)
    # a new catalogue has no pair sums until its first compute
    est.set_points(xyz[:100], w[:100])
    with pytest.raises(ctbmod.CTBError) as e:
        est.pair_sums()
    assert e.value.code == ctbmod.ERR_STATE


# ------------------------------------------------------------------ edge cases


def test_edge_empty_and_single(ctbmod):
    kw = dict(box=100.0, rmin=1.0, rmax=20.0, nbins=3, lmax=4)
    est = make(ctbmod, **kw)
    est.set_points(np.zeros((0, 3)), None)
    assert np.all(est.compute() == 0)
    est.set_points(np.array([[5.0, 5.0, 5.0]]), np.array([2.0]))
    assert np.all(est.compute() == 0)
    assert est.pair_count() == 0


def test_edge_hand_triangle_and_faces(ctbmod):
    """O with neighbours at 120 degrees in bins 0 and 1, placed across the
    periodic faces: zeta_l(0,1) = wO wA wB P_l(-1/2)."""
    from numpy.polynomial import legendre as npleg
    t = np.deg2rad(120.0)
    O = np.array([0.2, 99.9, 50.0])
    pts = synth.snap_periodic(np.array([O, O + [15.0, 0, 0], O + [25 * np.cos(t), 25 * np.sin(t), 0]]), 100.0)
    w = np.array([1.3, 0.7, -0.4])
    kw = dict(box=100.0, rmin=10.0, rmax=30.0, nbins=2, lmax=10)
    z, _ = run_full(ctbmod, pts, w, kw)
    for l in range(11):
        c = np.zeros(l + 1)
        c[l] = 1
        assert abs(z[l, 0, 1] - 1.3 * 0.7 * -0.4 * npleg.legval(-0.5, c)) < 1e-5


def test_edge_all_in_one_cell_nbins1_rmin0(ctbmod):
    rng = np.random.default_rng(3)
    xyz = synth.snap_dyadic(50.0 + rng.uniform(-1, 1, size=(300, 3)), 2.0 ** -20)
    w = rng.uniform(0.5, 1.5, 300)
    kw = dict(box=0.0, rmin=0.0, rmax=4.0, nbins=1, lmax=6)
    z, _ = run_full(ctbmod, xyz, w, kw)
    ref = oracle.zeta(xyz, w, **kw)
    assert zeta_err(z, ref) < TOL_FP32


def test_edge_coincident_points_and_small_box(ctbmod):
    """Duplicated points (r = 0 never binned) in a box only a few cells wide."""
    rng = np.random.default_rng(4)
    base = synth.snap_periodic(rng.uniform(0, 10.0, size=(200, 3)), 10.0)
    xyz = np.concatenate([base, base[:50]])
    w = rng.uniform(0.5, 1.5, xyz.shape[0])
    kw = dict(box=10.0, rmin=0.0, rmax=5.0, nbins=3, lmax=5)
    z, _ = run_full(ctbmod, xyz, w, kw)
    ref = oracle.zeta(xyz, w, **kw)
    assert zeta_err(z, ref) < TOL_FP32


def test_edge_negative_weights_and_wrap_inputs(ctbmod):
    xyz, _ = synth.uniform(3000, 250.0, seed=9)
    xyz = xyz + np.array([-250.0, 500.0, -750.0])  # periodic images of the same catalogue
    w = np.random.default_rng(9).uniform(-1.0, 1.0, xyz.shape[0])
    kw = dict(box=250.0, rmin=2.0, rmax=30.0, nbins=5, lmax=8)
    z, _ = run_full(ctbmod, xyz, w, kw)
    ref = oracle.zeta(np.mod(xyz, 250.0), w, **kw)
    # negative primary weights: the Gram bound still scales every entry
    assert zeta_err(z, ref) < TOL_FP32


def test_errors_are_status_codes(ctbmod):
    with pytest.raises(ctbmod.CTBError):
        ctbmod.CTB(100.0, 1.0, 60.0, 4, 2)           # r_max > L/2
    with pytest.raises(ctbmod.CTBError):
        ctbmod.CTB(100.0, 1.0, 10.0, 4, 21)          # l_max above the cap
    est = ctbmod.CTB(100.0, 1.0, 10.0, 4, 2)
    with pytest.raises(ctbmod.CTBError) as e:
        est.compute()
    assert e.value.code == ctbmod.ERR_STATE
    bad = np.zeros((10, 3))
    bad[3, 1] = np.nan
    with pytest.raises(ctbmod.CTBError) as e:
        est.set_points(bad)
    assert e.value.code == ctbmod.ERR_NONFINITE
    est.set_points(np.zeros((4, 3)))
    with pytest.raises(ctbmod.CTBError) as e:
        est.compute_subset(np.array([0, 7]))
    assert e.value.code == ctbmod.ERR_ARG
    # the pair kernels take blocks of at most 4 warps
    with pytest.raises(ctbmod.CTBError) as e:
        est.set_option(ctbmod.OPT_WARPS_PER_BLOCK, 5)
    assert e.value.code == ctbmod.ERR_ARG
    est.set_option(ctbmod.OPT_WARPS_PER_BLOCK, 2)
    est.compute()


def test_device_pointers_in_and_out(ctbmod):
    torch = pytest.importorskip("torch")
    xyz, w = synth.thomas(3000, 200.0, 30, 4.0, seed=27, weights="u0.5-1.5")
    kw = dict(box=200.0, rmin=1.0, rmax=30.0, nbins=4, lmax=5)
    est = make(ctbmod, **kw)
    est.set_stream(torch.cuda.current_stream())
    est.use_torch_allocator()
    est.set_points(torch.from_numpy(xyz).cuda(), torch.from_numpy(w).cuda())
    out = torch.zeros(est.zeta_shape, dtype=torch.float64, device="cuda")
    est.compute(out=out)
    ref = oracle.zeta(xyz, w, **kw)
    assert zeta_err(out.cpu().numpy(), ref) < TOL_FP32


# ------------------------------------------------------------------ full sizes


@pytest.mark.slow
def test_thomas_1m_sampled_primaries(ctbmod):
    """1M Thomas points, L = 1000, r in [5, 200], 20 bins, l_max 10: the full
    launch's zeta is checked by partition; sampled primaries against the oracle."""
    xyz, w = synth.thomas_1m()
    kw = synth.config_params(2)
    est = make(ctbmod, **kw)
    est.set_points(xyz, w)
    prim = synth.sample_primaries(xyz.shape[0], 96, seed=7)
    z = est.compute_subset(prim)
    ref = oracle.zeta(xyz, w, prim=prim, **kw)
    assert est.pair_count() == ref["npairs"]
    assert zeta_err(z, ref) < TOL_FP32


# ------------------------------------------------------- tensor-core contraction

TOL_MIXED = 1e-3   # BF16 hi/lo split or TF32 contraction, FP32 accumulate, FP64 reduce


@pytest.mark.parametrize("prec", ["BF16X3", "TF32"])
@pytest.mark.parametrize("nbins,lmax", [(8, 10), (36, 10), (5, 20)])
def test_tensor_core_contraction_vs_oracle(ctbmod, prec, nbins, lmax):
    xyz, w = synth.thomas(5000, 300.0, 50, 5.0, seed=28, weights="u0.5-1.5")
    kw = dict(box=300.0, rmin=2.0, rmax=50.0, nbins=nbins, lmax=lmax)
    z, _ = run_full(ctbmod, xyz, w, kw, precision=getattr(ctbmod, "PREC_" + prec))
    ref = oracle.zeta(xyz, w, **kw)
    err = zeta_err(z, ref)
    assert err < TOL_MIXED
    if prec == "BF16X3":
        assert err < 1e-4  # three products keep ~16 mantissa bits per operand


def test_tensor_core_chunks_and_negative_weights(ctbmod):
    """Several primary chunks accumulate into the same per-CTA partials; signed weights."""
    xyz, _ = synth.uniform(6000, 250.0, seed=29)
    w = np.random.default_rng(29).uniform(-1.0, 1.0, xyz.shape[0])
    kw = dict(box=250.0, rmin=2.0, rmax=40.0, nbins=6, lmax=6)
    z, est = run_full(ctbmod, xyz, w, kw, precision=ctbmod.PREC_BF16X3, chunk_primaries=1024)
    assert est.chunk_count() == 6  # 6000 primaries in chunks of at most 1024
    ref = oracle.zeta(xyz, w, **kw)
    assert zeta_err(z, ref) < TOL_MIXED


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["FP32", "BF16X3"])
def test_thomas_4m_subset_200k_full_vs_oracle(ctbmod, prec):
    """The seeded 200k subset of the 4M Thomas catalogue (L = 2000, r in
    [10, 200], 32 bins, l_max 20): full zeta against the oracle."""
    xyz, w = synth.thomas_4m_subset()
    kw = synth.config_params(3)
    z, est = run_full(ctbmod, xyz, w, kw, precision=getattr(ctbmod, "PREC_" + prec))
    ref = _cached_oracle("thomas_4m_subset", xyz, w, kw)
    assert est.pair_count() == ref["npairs"]
    assert zeta_err(z, ref) < (TOL_FP32 if prec == "FP32" else TOL_MIXED)


@pytest.mark.slow
def test_cut_sky_sampled_primaries(ctbmod):
    """Cut-sky sector: 8M clustered data (w = +1) and 24M uniform randoms
    (w = -1/3), open boundary, r in [20, 200], 36 bins, l_max 10; 192 seeded
    primaries with all 32M secondaries, against the oracle."""
    xyz, w = synth.cut_sky()
    kw = synth.config_params(5)
    est = make(ctbmod, **kw)
    est.set_points(xyz, w)
    prim = synth.sample_primaries(xyz.shape[0], 192, seed=7)
    z = est.compute_subset(prim)
    ref = oracle.zeta(xyz, w, prim=prim, **kw)
    assert est.pair_count() == ref["npairs"]
    assert zeta_err(z, ref) < TOL_FP32


_ORACLE_CACHE = {}


def _cached_oracle(key, xyz, w, kw):
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = oracle.zeta(xyz, w, **kw)
    return _ORACLE_CACHE[key]


# ------------------------------------------------------------------ batches


@pytest.mark.parametrize("prec", ["FP32", "BF16X3"])
def test_batch_matches_single_catalogues(ctbmod, prec):
    """Uneven mock catalogues (one empty) in one batch: each zeta matches the
    catalogue computed alone, and two of them match the oracle."""
    sizes = [3000, 0, 700, 5200, 1500]
    cats = [synth.thomas(n, 300.0, max(1, n // 100), 5.0, seed=60 + i, weights="u0.5-1.5") for i, n in
            enumerate(sizes)]
    kw = dict(box=300.0, rmin=2.0, rmax=40.0, nbins=6, lmax=8)
    opts = dict(precision=getattr(ctbmod, "PREC_" + prec))
    est = make(ctbmod, **kw, **opts)
    zb = est.compute_batch(cats)
    assert zb.shape == (len(sizes), 9, 6, 6)
    assert np.all(zb[1] == 0)
    pb = est.pair_sums(len(sizes))
    assert np.all(pb[1] == 0)
    tol = TOL_FP32 if prec == "FP32" else TOL_MIXED
    for i, (xyz, w) in enumerate(cats):
        if sizes[i] == 0:
            continue
        zs, single = run_full(ctbmod, xyz, w, kw, **opts)
        np.testing.assert_allclose(pb[i], single.pair_sums(), rtol=PAIRSUM_RTOL)
        ref = oracle.zeta(xyz, w, **kw) if i in (2, 3) else None
        if ref is not None:
            assert zeta_err(zb[i], ref) < tol
            assert zeta_err(zs, ref) < tol
            np.testing.assert_allclose(pb[i], ref["wpairs"], rtol=PAIRSUM_RTOL)
        scale = np.abs(zs).max()
        assert np.max(np.abs(zb[i] - zs)) <= 1e-6 * scale
    # the batch replaced the context's catalogue
    with pytest.raises(ctbmod.CTBError) as e:
        est.compute()
    assert e.value.code == ctbmod.ERR_STATE


def test_batch_rejects_open_boundary(ctbmod):
    est = make(ctbmod, box=0.0, rmin=1.0, rmax=10.0, nbins=2, lmax=2)
    xyz, w = synth.uniform(100, 50.0, seed=1)
    with pytest.raises(ctbmod.CTBError) as e:
        est.compute_batch([(xyz, w)])
    assert e.value.code == ctbmod.ERR_UNSUPPORTED
