"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks the oracle against what mathematics fixes independently of
its code: scipy's complex spherical harmonics, quadrature orthonormality, the
addition theorem with numpy's Legendre polynomials, an O(N^3) triplet sum
written here from the triangle-angle form of the estimator, the l = 0 closed
form with scipy's cKDTree neighbour counts, exact Legendre values for
hand-built triangles, and invariances of the estimator.
"""
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from scipy import special
from scipy.spatial import cKDTree

import oracle
from paper_2604_08855_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def real_ylm_scipy(lmax, dirs):
    """Real Y_lm from scipy's complex ones: sqrt2 Re / sqrt2 Im for m>0 / m<0."""
    x, y, z = dirs.T
    theta = np.arccos(np.clip(z, -1, 1))
    phi = np.arctan2(y, x)
    out = np.zeros((dirs.shape[0], (lmax + 1) ** 2))
    for l in range(lmax + 1):
        for m in range(0, l + 1):
            c = special.sph_harm_y(l, m, theta, phi)
            if m == 0:
                out[:, l * l + l] = c.real
            else:
                out[:, l * l + l + m] = np.sqrt(2) * c.real
                out[:, l * l + l - m] = np.sqrt(2) * c.imag
    return out


def random_dirs(n, seed):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


# ---------------------------------------------------------------- Y_lm pins

def test_ylm_matches_scipy():
    d = random_dirs(200, 11)
    d = np.concatenate([d, [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0]]])
    ours = oracle.ylm(20, d)
    ref = real_ylm_scipy(20, d)
    assert np.max(np.abs(ours - ref)) < 1e-12


def test_ylm_orthonormal_by_quadrature():
    lmax = 12
    xg, wg = npleg.leggauss(lmax + 2)
    nphi = 2 * lmax + 3
    phi = 2 * np.pi * np.arange(nphi) / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    wts = (wg[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y = oracle.ylm(lmax, dirs)
    gram = (Y * wts[:, None]).T @ Y
    assert np.max(np.abs(gram - np.eye(Y.shape[1]))) < 1e-12


def test_addition_theorem():
    lmax = 20
    a = random_dirs(100, 1)
    b = random_dirs(100, 2)
    Ya, Yb = oracle.ylm(lmax, a), oracle.ylm(lmax, b)
    mu = np.sum(a * b, axis=1)
    for l in range(lmax + 1):
        sl = slice(l * l, (l + 1) ** 2)
        lhs = np.sum(Ya[:, sl] * Yb[:, sl], axis=1)
        coef = np.zeros(l + 1)
        coef[l] = 1
        rhs = (2 * l + 1) / (4 * np.pi) * npleg.legval(mu, coef)
        assert np.max(np.abs(lhs - rhs)) < 1e-12
        # same direction: sum_m Y_lm^2 = (2l+1)/(4 pi)
        assert np.max(np.abs(np.sum(Ya[:, sl] ** 2, axis=1) - (2 * l + 1) / (4 * np.pi))) < 1e-12


# ---------------------------------------------------------------- zeta pins

def min_image(d, box):
    if box > 0:
        d = d - box * np.round(d / box)
    return d


def triplet_zeta(xyz, w, box, rmin, rmax, nbins, lmax):
    """sum_p w_p sum_{j,k} w_j w_k P_l(cos angle_jk) [b_j=b1][b_k=b2], j,k != p."""
    n = xyz.shape[0]
    edges = rmin + (rmax - rmin) * np.arange(nbins + 1) / nbins
    out = np.zeros((lmax + 1, nbins, nbins))
    for p in range(n):
        d = min_image(xyz - xyz[p], box)
        r = np.linalg.norm(d, axis=1)
        ok = (r >= rmin) & (r < rmax) & (np.arange(n) != p) & (r > 0)
        if not np.any(ok):
            continue
        u = d[ok] / r[ok, None]
        b = np.searchsorted(edges, r[ok], side="right") - 1
        onehot = np.zeros((u.shape[0], nbins))
        onehot[np.arange(u.shape[0]), b] = w[ok]
        cosm = np.clip(u @ u.T, -1, 1)
        for l in range(lmax + 1):
            coef = np.zeros(l + 1)
            coef[l] = 1
            out[l] += w[p] * onehot.T @ npleg.legval(cosm, coef) @ onehot
    return out


@pytest.mark.parametrize("box", [60.0, 0.0])
def test_zeta_equals_triplet_sum(box):
    rng = np.random.default_rng(5)
    n = 110
    xyz = rng.uniform(0, 60.0, size=(n, 3))
    w = rng.uniform(-0.5, 1.5, size=n)
    kw = dict(box=box, rmin=3.0, rmax=25.0, nbins=5, lmax=8)
    z = oracle.zeta(xyz, w, **kw)["zeta"]
    t = triplet_zeta(xyz, w, **kw)
    scale = np.max(np.abs(t))
    assert scale > 0
    assert np.max(np.abs(z - t)) < 1e-10 * scale


def test_l0_closed_form_with_kdtree_counts():
    """zeta_0(b1,b2) = sum_p w_p N_p(b1) N_p(b2), N_p(b) = sum_{j in b} w_j."""
    xyz, w = synth.thomas(3000, 400.0, 30, 5.0, seed=3, weights="u0.5-1.5")
    box, rmin, rmax, nbins = 400.0, 2.0, 60.0, 8
    tree = cKDTree(xyz, boxsize=box)
    sdm = tree.sparse_distance_matrix(tree, rmax, output_type="coo_matrix")
    i, j, r = sdm.row, sdm.col, sdm.data
    keep = (i != j) & (r >= rmin) & (r < rmax)
    i, j, r = i[keep], j[keep], r[keep]
    edges = rmin + (rmax - rmin) * np.arange(nbins + 1) / nbins
    b = np.searchsorted(edges, r, side="right") - 1
    N = np.zeros((xyz.shape[0], nbins))
    np.add.at(N, (i, b), w[j])
    expect = np.einsum("p,pa,pb->ab", w, N, N)
    got = oracle.zeta(xyz, w, box, rmin, rmax, nbins, 2)
    assert np.allclose(got["zeta"][0], expect, rtol=1e-12, atol=0)
    assert np.allclose(got["wpairs"], np.einsum("p,pb->b", w, N), rtol=1e-12)
    S = np.zeros((xyz.shape[0], nbins))
    np.add.at(S, (i, b), w[j] ** 2)
    assert np.allclose(got["selfw"], np.einsum("p,pb->b", w, S), rtol=1e-12)
    assert got["npairs"] == i.size


def load_golden_minus_half():
    vals = {}
    with open(os.path.join(GOLDEN, "legendre_minus_half.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            l, num, den = map(int, line.split())
            vals[l] = num / den
    return vals


def test_golden_fixture_is_legendre():
    vals = load_golden_minus_half()
    for l, v in vals.items():
        coef = np.zeros(l + 1)
        coef[l] = 1
        assert abs(npleg.legval(-0.5, coef) - v) < 1e-15


def three_points(theta_deg, rA, rB, wO, wA, wB, origin, rot=np.eye(3)):
    t = np.deg2rad(theta_deg)
    nA = np.array([1.0, 0.0, 0.0])
    nB = np.array([np.cos(t), np.sin(t), 0.0])
    pts = np.array([np.zeros(3), rA * nA, rB * nB]) @ rot.T + origin
    return pts, np.array([wO, wA, wB])


@pytest.mark.parametrize("box", [0.0, 200.0])
def test_hand_geometry_120_degrees(box):
    """O at the vertex, A (bin 0) and B (bin 1) at 120 degrees; |AB| > rmax so
    only O sees both.  zeta_l(0,1) = wO wA wB P_l(-1/2) (golden fixture); the
    diagonals collect the j = k terms: zeta_l(0,0) = wO wA^2 + wA wO^2."""
    lmax = 12
    vals = load_golden_minus_half()
    wO, wA, wB = 1.3, 0.7, -0.4
    pts, w = three_points(120.0, 15.0, 25.0, wO, wA, wB, origin=np.array([50.0, 60.0, 70.0]))
    res = oracle.zeta(pts, w, box, 10.0, 30.0, 2, lmax)["zeta"]
    for l in range(lmax + 1):
        assert abs(res[l, 0, 1] - wO * wA * wB * vals[l]) < 1e-13
        assert abs(res[l, 1, 0] - wO * wA * wB * vals[l]) < 1e-13
        assert abs(res[l, 0, 0] - (wO * wA ** 2 + wA * wO ** 2)) < 1e-13
        assert abs(res[l, 1, 1] - (wO * wB ** 2 + wB * wO ** 2)) < 1e-13


def test_hand_geometry_collinear():
    """A and B on opposite sides of O: P_l(-1) = (-1)^l."""
    lmax = 10
    rot = np.linalg.qr(np.random.default_rng(9).normal(size=(3, 3)))[0]
    pts, w = three_points(180.0, 12.0, 27.0, 2.0, 1.0, 1.0, origin=np.array([5.0, 5.0, 5.0]), rot=rot)
    res = oracle.zeta(pts, w, 0.0, 10.0, 30.0, 2, lmax)["zeta"]
    for l in range(lmax + 1):
        assert abs(res[l, 0, 1] - 2.0 * (-1) ** l) < 1e-12


def test_hand_geometry_alm_single_neighbour():
    """a_lm(O, b) = w_A Y_lm(nhat_A) with Y from scipy."""
    lmax = 10
    rot = np.linalg.qr(np.random.default_rng(4).normal(size=(3, 3)))[0]
    pts, w = three_points(150.0, 15.0, 25.0, 1.0, 0.8, 1.7, origin=np.zeros(3), rot=rot)
    a = oracle.alm(pts, w, 0.0, 10.0, 30.0, 2, lmax, prim=[0])[0]
    nA = (pts[1] - pts[0]) / 15.0
    nB = (pts[2] - pts[0]) / 25.0
    assert np.max(np.abs(a[0] - 0.8 * real_ylm_scipy(lmax, nA[None])[0])) < 1e-12
    assert np.max(np.abs(a[1] - 1.7 * real_ylm_scipy(lmax, nB[None])[0])) < 1e-12


def test_periodic_wrap_pair_across_faces():
    """Two points near opposite faces are neighbours through the boundary."""
    box = 100.0
    pts = np.array([[0.5, 50.0, 50.0], [99.0, 50.0, 50.0]])
    w = np.array([1.0, 2.0])
    a = oracle.alm(pts, w, box, 1.0, 3.0, 1, 2, prim=[0, 1])
    # separation 1.5 along -x from point 0 and +x from point 1
    assert np.allclose(a[0, 0], 2.0 * real_ylm_scipy(2, np.array([[-1.0, 0, 0]]))[0], atol=1e-13)
    assert np.allclose(a[1, 0], 1.0 * real_ylm_scipy(2, np.array([[1.0, 0, 0]]))[0], atol=1e-13)


# ---------------------------------------------------------------- invariances

KW = dict(rmin=4.0, rmax=40.0, nbins=6, lmax=6)


def small_cat(seed=0, n=700, box=200.0):
    return synth.thomas(n, box, 20, 4.0, seed=seed, weights="u0.5-1.5")


def test_permutation_invariance():
    xyz, w = small_cat()
    z1 = oracle.zeta(xyz, w, 200.0, **KW)["zeta"]
    perm = np.random.default_rng(1).permutation(xyz.shape[0])
    z2 = oracle.zeta(xyz[perm], w[perm], 200.0, **KW)["zeta"]
    assert np.allclose(z1, z2, rtol=1e-11, atol=1e-11 * np.abs(z1).max())


def test_periodic_translation_invariance():
    xyz, w = small_cat()
    z1 = oracle.zeta(xyz, w, 200.0, **KW)["zeta"]
    z2 = oracle.zeta(np.mod(xyz + np.array([73.1, -12.7, 151.9]), 200.0), w, 200.0, **KW)["zeta"]
    assert np.allclose(z1, z2, rtol=1e-10, atol=1e-10 * np.abs(z1).max())


def test_rotation_invariance_open_box():
    xyz, w = small_cat()
    rot = np.linalg.qr(np.random.default_rng(2).normal(size=(3, 3)))[0]
    z1 = oracle.zeta(xyz, w, 0.0, **KW)["zeta"]
    z2 = oracle.zeta(xyz @ rot.T + 17.0, w, 0.0, **KW)["zeta"]
    assert np.allclose(z1, z2, rtol=1e-10, atol=1e-10 * np.abs(z1).max())


def test_weight_scaling_symmetry_psd_and_gram_bound():
    xyz, w = small_cat(seed=3)
    r1 = oracle.zeta(xyz, w, 200.0, **KW)
    r2 = oracle.zeta(xyz, 1.7 * w, 200.0, **KW)
    z = r1["zeta"]
    assert np.allclose(r2["zeta"], 1.7 ** 3 * z, rtol=1e-12, atol=1e-12 * np.abs(z).max())
    assert np.allclose(z, np.transpose(z, (0, 2, 1)), rtol=0, atol=1e-12 * np.abs(z).max())
    for l in range(z.shape[0]):
        ev = np.linalg.eigvalsh(z[l])
        assert ev.min() > -1e-9 * ev.max()
    g = r1["gram"]
    d = np.sqrt(np.einsum("lii->li", g))
    s = d[:, :, None] * d[:, None, :]
    assert np.all(np.abs(z) <= s * (1 + 1e-12))


def test_primary_subsets_add_up():
    xyz, w = small_cat(seed=4)
    z = oracle.zeta(xyz, w, 200.0, **KW)["zeta"]
    idx = np.random.default_rng(0).permutation(xyz.shape[0])
    za = oracle.zeta(xyz, w, 200.0, prim=idx[:300], **KW)["zeta"]
    zb = oracle.zeta(xyz, w, 200.0, prim=idx[300:], **KW)["zeta"]
    assert np.allclose(za + zb, z, rtol=1e-12, atol=1e-12 * np.abs(z).max())


def test_alm_contracts_to_zeta():
    xyz, w = small_cat(seed=6, n=300)
    kw = dict(rmin=4.0, rmax=40.0, nbins=4, lmax=5)
    a = oracle.alm(xyz, w, 200.0, **kw)
    z = oracle.zeta(xyz, w, 200.0, **kw)["zeta"]
    for l in range(6):
        sl = slice(l * l, (l + 1) ** 2)
        zz = 4 * np.pi / (2 * l + 1) * np.einsum("p,pac,pbc->ab", w, a[:, :, sl], a[:, :, sl])
        assert np.allclose(zz, z[l], rtol=1e-12, atol=1e-12 * np.abs(z).max())


def test_contract_reproduces_zeta():
    """oracle.contract on the oracle's own a_lm rows gives oracle.zeta, for a
    primary subset with negative weights and in open space."""
    xyz, w = small_cat(seed=9, n=400)
    w = w * np.where(np.arange(w.size) % 3 == 0, -1.0, 1.0)
    kw = dict(rmin=3.0, rmax=45.0, nbins=5, lmax=6)
    prim = np.random.default_rng(3).choice(xyz.shape[0], 150, replace=False)
    for box in (200.0, 0.0):
        a = oracle.alm(xyz, w, box, prim=prim, **kw)
        z = oracle.zeta(xyz, w, box, prim=prim, **kw)["zeta"]
        zc = oracle.contract(a, w[prim], kw["lmax"])
        assert np.allclose(zc, z, rtol=1e-12, atol=1e-12 * np.abs(z).max())
    with pytest.raises(ValueError):
        oracle.contract(a[:, :, :-1], w[prim], kw["lmax"])


def test_argument_checks():
    xyz, w = small_cat(n=50)
    with pytest.raises(ValueError):
        oracle.zeta(xyz, w, 200.0, rmin=4.0, rmax=150.0, nbins=4, lmax=2)  # rmax > L/2
    with pytest.raises(ValueError):
        oracle.zeta(xyz, w, 200.0, rmin=5.0, rmax=4.0, nbins=4, lmax=2)
    with pytest.raises(ValueError):
        oracle.zeta(xyz, w, 200.0, rmin=1.0, rmax=4.0, nbins=0, lmax=2)


def test_ambiguous_pair_count():
    """A pair placed exactly on an interior bin edge is counted as ambiguous."""
    pts = np.array([[0.0, 0.0, 0.0], [20.0, 0.0, 0.0]])
    r = oracle.zeta(pts, None, 0.0, 10.0, 30.0, 2, 0, amb_tol=1e-9)
    assert r["namb"] == 2 and r["npairs"] == 2
    # half-open bins: r = 20 belongs to bin 1
    assert r["wpairs"][1] == 2.0 and r["wpairs"][0] == 0.0


def test_generators_are_on_the_fixed_point_grid():
    """Snapped catalogues: x / L * 2^32 is an exact integer (periodic), and
    x * 2^20 an exact integer (open space)."""
    for box in (1000.0, 2000.0, 400.0, 250.0):
        xyz, _ = synth.thomas(5000, box, 50, 5.0, seed=1)
        k = xyz / box * 4294967296.0
        assert np.all(k == np.floor(k)) and np.all(k >= 0) and np.all(k < 4294967296.0)
    s = synth.sector_randoms(5000, seed=6)
    assert np.all(s * 2.0 ** 20 == np.floor(s * 2.0 ** 20))
    assert np.all(synth.in_sector(s))


# ------------------------------------------------- edge-ambiguous pairs

def test_ambiguous_hand_pairs():
    """Pairs placed at and near edges are listed with the right edge index,
    and their count equals zeta's namb for the same tolerance."""
    rmin, rmax, nb = 10.0, 30.0, 4          # edges 10, 15, 20, 25, 30
    pts = np.array([[0.0, 0.0, 0.0],
                    [15.0 + 1e-9, 0.0, 0.0],    # edge 1, just above
                    [0.0, 25.0 - 1e-9, 0.0],    # edge 3, just below
                    [0.0, 0.0, 30.0],           # edge 4 (r_max), on it
                    [0.0, 0.0, -17.5]])         # mid-bin: not ambiguous
    idx, d, r, edge = oracle.ambiguous(pts, 0.0, rmin, rmax, nb, 1e-8, prim=np.array([0]))
    assert [tuple(x) for x in idx] == [(0, 1), (0, 2), (0, 3)]
    assert list(edge) == [1, 3, 4]
    np.testing.assert_allclose(r, [15.0 + 1e-9, 25.0 - 1e-9, 30.0])
    np.testing.assert_allclose(d[2], [0.0, 0.0, 30.0])
    full = oracle.ambiguous(pts, 0.0, rmin, rmax, nb, 1e-8)
    z = oracle.zeta(pts, None, 0.0, rmin, rmax, nb, 0, amb_tol=1e-8)
    assert len(full[0]) == z["namb"]


def test_bin_flip_bound_covers_planted_flips():
    """Secondaries planted just above edges, then moved just below them (a
    binning of rounded coordinates could do that): the change of zeta stays
    within the bound built from the unmoved catalogue's ambiguous pairs."""
    from tests.parity import bin_flip_bound
    rng = np.random.default_rng(12)
    box = 200.0
    kw = dict(box=box, rmin=4.0, rmax=40.0, nbins=6, lmax=6)
    xyz, w = small_cat(seed=13, n=400, box=box)
    prim = np.array([3, 50, 51, 200])
    edges = kw["rmin"] + np.arange(kw["nbins"] + 1) * (kw["rmax"] - kw["rmin"]) / kw["nbins"]
    planted, moved = [], []
    for k, p in enumerate(prim):
        for e in (edges[0], edges[2], edges[6], edges[(k % 5) + 1]):
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            planted.append(np.mod(xyz[p] + (e + 2e-9) * u, box))
            moved.append(np.mod(xyz[p] + (e - 2e-9) * u, box))
    x0 = np.vstack([xyz, planted])
    x1 = np.vstack([xyz, moved])
    ww = np.concatenate([w, rng.uniform(0.5, 1.5, len(planted))])
    z0 = oracle.zeta(x0, ww, prim=prim, **kw)
    z1 = oracle.zeta(x1, ww, prim=prim, **kw)
    amb = oracle.ambiguous(x0, box, kw["rmin"], kw["rmax"], kw["nbins"], 1e-8 / kw["rmin"], prim=prim)
    assert len(amb[0]) >= len(planted)
    bz, bp, outer = bin_flip_bound(x0, ww, kw, prim, amb)
    dz = np.abs(z1["zeta"] - z0["zeta"])
    assert dz.max() > 1e-3 * np.abs(z0["zeta"]).max()      # the flips do change zeta
    assert np.all(dz <= bz * (1 + 1e-9) + 1e-9 * np.abs(z0["zeta"]).max())
    assert np.all(np.abs(z1["wpairs"] - z0["wpairs"]) <= bp * (1 + 1e-9) + 1e-12)
    assert abs(z1["npairs"] - z0["npairs"]) <= outer
