"""Pins of the oracle's shared-neighbour-list estimate and its bound (CPU).

The pins do not go through the shared estimator's own code path:

- hand-placed points with their pivot cells, wrap and representatives;
- one-point groups give oracle.zeta, and so do groups of coincident points
  (a catalogue and a copy with other weights);
- an O(N^3) triplet sum, with scipy's Legendre polynomials and independent
  binning, gives the signed difference from the exact estimate.  Its
  absolute version lies between |dzeta| and the bound;
- the bound holds on clustered catalogues, periodic and open, with weights
  of both signs;
- with no membership change the bound's l = 0 entry is zero and the rest is
  linear in the displacement;
- the primary-weight override of oracle.zeta is exact and linear.
"""
import numpy as np
import pytest

import oracle
from oracle import shared
from paper_2604_08855_gb300 import synth


def test_pivot_groups_hand():
    xyz = np.array([
        [0.2, 0.2, 0.2],    # cell (0, 0, 0)
        [1.0, 0.1, 0.1],    # (1, 0, 0): a point on a cell face belongs to the upper cell
        [0.9, 0.1, 0.5],    # (0, 0, 0)
        [-0.1, 0.5, 0.5],   # (-1, 0, 0); periodic box 4: wraps to 3.9, cell (3, 0, 0)
        [1.5, 0.99, 0.0],   # (1, 0, 0)
        [3.95, 0.5, 0.5],   # (3, 0, 0)
    ])
    w = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    label, rep, W = shared.pivot_groups(xyz, 1.0, w=w)
    assert label.tolist() == [0, 1, 0, 2, 1, 3]
    assert rep.tolist() == [0, 1, 3, 5]
    assert W.tolist() == [4.0, 7.0, 4.0, 6.0]
    label, rep, W = shared.pivot_groups(xyz, 1.0, box=4.0, w=w)
    assert label.tolist() == [0, 1, 0, 2, 1, 2]
    assert rep.tolist() == [0, 1, 3]
    assert W.tolist() == [4.0, 7.0, 10.0]
    label, rep, W = shared.pivot_groups(xyz, 10.0, w=w)  # one cell holds all but the negative x
    assert rep.tolist() == [0, 3]
    assert W.tolist() == [17.0, 4.0]
    with pytest.raises(ValueError):
        shared.pivot_groups(xyz, 0.0)


def test_mean_separation():
    xyz = np.array([[0.0, 0.0, 0.0], [2.0, 1.0, 4.0], [1.0, 0.5, 0.0], [0.0, 0.0, 1.0]])
    assert shared.mean_separation(xyz, box=8.0) == pytest.approx(8.0 / 4 ** (1 / 3), rel=1e-15)
    # open: sides 2, 1, 4, each at least rmax = 1.5 -> 2 * 1.5 * 4
    assert shared.mean_separation(xyz, rmax=1.5) == pytest.approx((12.0 / 4) ** (1 / 3), rel=1e-15)


def test_primary_weight_override():
    xyz, w = synth.thomas(600, 60.0, 12, 3.0, seed=501, weights="u0.5-1.5")
    kw = dict(box=60.0, rmin=1.0, rmax=15.0, nbins=4, lmax=4)
    prim = np.arange(0, 600, 7)
    a = oracle.zeta(xyz, w, prim=prim, **kw)
    b = oracle.zeta(xyz, w, prim=prim, wprim=w[prim], **kw)
    assert np.array_equal(a["zeta"], b["zeta"])
    c = oracle.zeta(xyz, w, prim=prim, wprim=-2.0 * w[prim], **kw)
    np.testing.assert_allclose(c["zeta"], -2.0 * a["zeta"], rtol=1e-13, atol=1e-13 * np.abs(a["zeta"]).max())
    np.testing.assert_allclose(c["gram"], 2.0 * a["gram"], rtol=1e-13, atol=1e-13 * np.abs(a["gram"]).max())


def test_singleton_groups_are_exact():
    xyz, w = synth.uniform(400, 50.0, seed=502, weights="u0.5-1.5")
    kw = dict(box=50.0, rmin=2.0, rmax=15.0, nbins=5, lmax=6)
    s = shared.zeta_shared(xyz, w, h=1e-4, **kw)
    assert s["rep"].shape[0] == 400
    e = oracle.zeta(xyz, w, **kw)
    np.testing.assert_allclose(s["zeta"], e["zeta"], rtol=1e-12, atol=1e-12 * np.abs(e["zeta"]).max())
    assert s["npairs"] == e["npairs"]
    assert not np.any(shared.shared_bound(xyz, w, h=1e-4, **kw))


@pytest.mark.parametrize("box", [40.0, 0.0])
def test_coincident_groups_are_exact(box):
    xyz, w1 = synth.thomas(250, 40.0, 8, 2.0, seed=503, weights="u0.5-1.5")
    w2 = np.random.default_rng(504).uniform(-1.0, 1.0, 250)
    xyz2 = np.concatenate([xyz, xyz])
    w = np.concatenate([w1, w2])
    kw = dict(box=box, rmin=1.0, rmax=12.0, nbins=4, lmax=5)
    s = shared.zeta_shared(xyz2, w, h=1e-3, **kw)
    label, _, _ = shared.pivot_groups(xyz2, 1e-3, box)
    assert np.array_equal(label[:250], label[250:])   # a point and its copy share a group
    assert np.array_equal(s["rep"], np.arange(250))
    np.testing.assert_allclose(s["W"], w1 + w2, rtol=1e-15)
    e = oracle.zeta(xyz2, w, **kw)
    np.testing.assert_allclose(s["zeta"], e["zeta"], rtol=1e-11, atol=1e-11 * np.abs(e["zeta"]).max())
    assert not np.any(shared.shared_bound(xyz2, w, h=1e-3, **kw))


def test_sphere_singletons_and_coincident_groups():
    xyz = synth.snap_dyadic(synth.fibonacci_sphere(700))
    w = synth.sphere_field(xyz, seed=505)
    kw = dict(theta_min=0.01, theta_max=0.3, nbins=4, mmax=6)
    s = shared.zeta_shared_sphere(xyz, w, h=1e-4, **kw)
    e = oracle.zeta_sphere(xyz, w, **kw)
    assert s["rep"].shape[0] == 700
    np.testing.assert_allclose(s["zeta"], e["zeta"], rtol=1e-12, atol=1e-12 * np.abs(e["zeta"]).max())
    xyz2 = np.concatenate([xyz, xyz])
    w2 = np.concatenate([w, 0.5 - w])
    s = shared.zeta_shared_sphere(xyz2, w2, h=1e-4, **kw)
    e = oracle.zeta_sphere(xyz2, w2, **kw)
    assert s["rep"].shape[0] == 700
    np.testing.assert_allclose(s["zeta"], e["zeta"], rtol=1e-11, atol=1e-11 * np.abs(e["zeta"]).max())


def _triplet_difference(xyz, w, box, rmin, rmax, nbins, lmax, rep_of):
    """sum_p w_p sum_{j,k} w_j w_k (T_c - T_p) and the same with absolute values,
    T_x = P_l(cos angle(x_j - x, x_k - x)) [bin_x(j) = b1][bin_x(k) = b2];
    binning by plain comparison with the edges, P_l from scipy."""
    from scipy.special import eval_legendre
    n = xyz.shape[0]
    edges = rmin + (rmax - rmin) * np.arange(nbins + 1) / nbins

    def view(x):
        d = xyz - xyz[x]
        if box > 0:
            d -= box * np.rint(d / box)
        r = np.linalg.norm(d, axis=1)
        b = np.full(n, -1)
        for k in range(nbins):
            b[(r >= edges[k]) & (r < edges[k + 1]) & (r > 0)] = k
        b[x] = -1
        u = d / np.where(r > 0, r, 1.0)[:, None]
        cosg = np.clip(u @ u.T, -1.0, 1.0)
        P = np.stack([eval_legendre(l, cosg) for l in range(lmax + 1)])
        ind = np.stack([b == k for k in range(nbins)]).astype(float)   # [nbins][n]
        return P, ind

    sig = np.zeros((lmax + 1, nbins, nbins))
    ab = np.zeros_like(sig)
    for p in range(n):
        c = rep_of[p]
        if c == p:
            continue
        Pp, Ip = view(p)
        Pc, Ic = view(c)
        for b1 in range(nbins):
            for b2 in range(nbins):
                Tp = Pp * np.outer(Ip[b1], Ip[b2])[None]
                Tc = Pc * np.outer(Ic[b1], Ic[b2])[None]
                ww = np.outer(w, w)[None]
                sig[:, b1, b2] += w[p] * np.sum(ww * (Tc - Tp), axis=(1, 2))
                ab[:, b1, b2] += abs(w[p]) * np.sum(np.abs(ww) * np.abs(Tc - Tp), axis=(1, 2))
    return sig, ab


def test_bound_against_triplet_sum():
    rng = np.random.default_rng(506)
    xyz = synth.snap_dyadic(rng.uniform(0.0, 10.0, (45, 3)))
    w = rng.uniform(-0.5, 1.5, 45)
    kw = dict(box=0.0, rmin=1.0, rmax=6.0, nbins=3, lmax=4)
    h = 2.5
    label, rep, _ = shared.pivot_groups(xyz, h)
    assert rep.shape[0] < 40   # several groups with more than one member
    sig, ab = _triplet_difference(xyz, w, rep_of=rep[label], **kw)
    s = shared.zeta_shared(xyz, w, h=h, **kw)
    e = oracle.zeta(xyz, w, **kw)
    dz = s["zeta"] - e["zeta"]
    scale = np.abs(e["zeta"]).max()
    # the shared estimate is the exact one with each member's terms taken from its representative
    np.testing.assert_allclose(dz, sig, rtol=1e-9, atol=1e-11 * scale)
    B = shared.shared_bound(xyz, w, h=h, **kw)
    assert np.all(np.abs(dz) <= ab + 1e-11 * scale)
    assert np.all(ab <= B + 1e-11 * scale)
    assert np.any(np.abs(dz) > 1e-6 * scale)


@pytest.mark.parametrize("box,wmode", [(100.0, "u0.5-1.5"), (0.0, "signed")])
@pytest.mark.parametrize("hfac", [0.5, 1.0, 2.0])
def test_bound_holds_on_clustered_catalogues(box, wmode, hfac):
    xyz, w = synth.thomas(1200, 100.0, 25, 3.0, seed=507, weights="u0.5-1.5")
    if wmode == "signed":
        w = np.random.default_rng(508).uniform(-1.0, 1.0, xyz.shape[0])
    kw = dict(box=box, rmin=2.0, rmax=20.0, nbins=5, lmax=6)
    h = hfac * shared.mean_separation(xyz, box, kw["rmax"])
    s = shared.zeta_shared(xyz, w, h=h, **kw)
    e = oracle.zeta(xyz, w, **kw)
    B = shared.shared_bound(xyz, w, h=h, **kw)
    dz = np.abs(s["zeta"] - e["zeta"])
    scale = np.sqrt(np.einsum("lii,ljj->lij", e["gram"], e["gram"]))
    assert np.all(dz <= B + 1e-10 * scale)
    assert np.any(dz > 1e-8 * scale)
    assert s["rep"].shape[0] < xyz.shape[0]


def test_bound_linear_without_membership_change():
    # representative c, member p displaced by delta along x, 30 neighbours mid-bin
    # in distinct cells: only the angular term of the bound is present
    dirs = synth.fibonacci_sphere(30)
    radii = 2.5 + np.arange(30) % 4
    c = np.array([0.1, 0.1, 0.1])
    nb = c + dirs * radii[:, None]
    w = np.random.default_rng(509).uniform(0.5, 1.5, 32)
    kw = dict(box=0.0, rmin=2.0, rmax=6.0, nbins=4, lmax=8)
    Bs = []
    for delta in (0.02, 0.01):
        xyz = np.concatenate([[c, c + [delta, 0.0, 0.0]], nb])
        label, rep, _ = shared.pivot_groups(xyz, 0.5)
        assert rep.tolist() == [0] + list(range(2, 32))   # only the pivot pair shares a cell
        B = shared.shared_bound(xyz, w, h=0.5, **kw)
        s = shared.zeta_shared(xyz, w, h=0.5, **kw)
        e = oracle.zeta(xyz, w, **kw)
        assert not np.any(B[0])
        np.testing.assert_allclose(s["zeta"][0], e["zeta"][0], rtol=1e-12)
        assert np.all(np.abs(s["zeta"] - e["zeta"]) <= B + 1e-12 * np.abs(e["zeta"]).max())
        Bs.append(B)
    ratio = Bs[0][1:] / Bs[1][1:]
    assert np.all((ratio > 1.98) & (ratio < 2.02))


def test_bound_hand_geometry():
    # representative c, member p = c + 0.1 x; neighbour j at 3 along y stays in
    # bin [2, 4) from both; neighbour k at 4.05 along x is in [4, 6) from c and
    # at 3.95, in [2, 4), from p.  By hand: alpha_j = atan(0.1 / 3); from p and c
    # S = (3, 0), A = (3 alpha_j, 0), D = (5, 5), U = (8, 5), and w_p = 2.
    c = np.array([0.05, 0.05, 0.05])
    xyz = np.array([c, c + [0.1, 0, 0], c + [0, 3.0, 0], c + [4.05, 0, 0]])
    w = np.array([1.0, 2.0, 3.0, 5.0])
    kw = dict(box=0.0, rmin=2.0, rmax=6.0, nbins=2, lmax=4)
    label, rep, _ = shared.pivot_groups(xyz, 1.0)
    assert label.tolist() == [0, 0, 1, 2]
    B = shared.shared_bound(xyz, w, h=1.0, **kw)
    aj = np.arctan(0.1 / 3.0)
    for l in range(5):
        np.testing.assert_allclose(B[l], 2.0 * np.array([[18 * l * aj + 80, 65], [65, 50]]), rtol=1e-13)


def _cap(n, seed, theta=0.25, centre=(0.3, -0.2, 0.93)):
    rng = np.random.default_rng(seed)
    c = np.asarray(centre, float)
    c /= np.linalg.norm(c)
    mu = rng.uniform(np.cos(theta), 1.0, n)
    ph = rng.uniform(0.0, 2 * np.pi, n)
    s = np.sqrt(1 - mu * mu)
    local = np.stack([s * np.cos(ph), s * np.sin(ph), mu], axis=1)
    z = np.array([0.0, 0.0, 1.0])
    v = np.cross(z, c)
    sn, cs = np.linalg.norm(v), z @ c
    k = v / sn
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return synth.snap_dyadic(local @ (np.eye(3) + sn * K + (1 - cs) * K @ K).T)


def test_sphere_bound_zero_for_singletons_and_coincident_groups():
    xyz = _cap(300, 510)
    w = np.random.default_rng(511).uniform(-1.0, 1.0, 300)
    kw = dict(theta_min=0.01, theta_max=0.3, nbins=4, mmax=5)
    assert not np.any(shared.shared_bound_sphere(xyz, w, h=1e-5, **kw))
    xyz2 = np.concatenate([xyz, xyz])
    w2 = np.concatenate([w, 1.0 - w])
    assert shared.pivot_groups(xyz2, 1e-5)[1].shape[0] == 300
    assert not np.any(shared.shared_bound_sphere(xyz2, w2, h=1e-5, **kw))


def _sphere_triplet_difference(xyz, w, theta_min, theta_max, nbins, mmax, rep_of):
    """sum_p w_p sum_{j,k} w_j w_k (T_c - T_p) and its absolute version; T_x =
    cos(m (phi_xj - phi_xk)) [bins], phi in a tangent frame built here."""
    import math
    n = xyz.shape[0]
    edges = np.array([2.0 * math.sin(0.5 * (theta_min + b * (theta_max - theta_min) / nbins))
                      for b in range(nbins + 1)])

    def view(x):
        nx = xyz[x] / np.linalg.norm(xyz[x])
        e1 = np.cross(nx, [0.3, 0.5, 0.8])
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(nx, e1)
        d = xyz - xyz[x]
        chord = np.linalg.norm(d, axis=1)
        b = np.full(n, -1)
        ok = (chord > 0) & (chord >= edges[0]) & (chord < edges[-1])
        b[ok] = np.searchsorted(edges, chord[ok], side="right") - 1
        b[x] = -1
        u, v = d @ e1, d @ e2
        phi = np.where((u == 0) & (v == 0), 0.0, np.arctan2(v, u))
        C = np.stack([np.cos(m * (phi[:, None] - phi[None, :])) for m in range(mmax + 1)])
        ind = np.stack([b == k for k in range(nbins)]).astype(float)
        return C, ind

    sig = np.zeros((mmax + 1, nbins, nbins))
    ab = np.zeros_like(sig)
    ww = np.outer(w, w)[None]
    for p in range(n):
        c = rep_of[p]
        if c == p:
            continue
        Cp, Ip = view(p)
        Cc, Ic = view(c)
        for b1 in range(nbins):
            for b2 in range(nbins):
                Tp = Cp * np.outer(Ip[b1], Ip[b2])[None]
                Tc = Cc * np.outer(Ic[b1], Ic[b2])[None]
                sig[:, b1, b2] += w[p] * np.sum(ww * (Tc - Tp), axis=(1, 2))
                ab[:, b1, b2] += abs(w[p]) * np.sum(np.abs(ww) * np.abs(Tc - Tp), axis=(1, 2))
    return sig, ab


def test_sphere_bound_against_triplet_sum():
    xyz = _cap(45, 512, theta=0.2)
    w = np.random.default_rng(513).uniform(-0.5, 1.5, 45)
    kw = dict(theta_min=0.01, theta_max=0.2, nbins=3, mmax=4)
    h = 0.05
    label, rep, _ = shared.pivot_groups(xyz, h)
    assert rep.shape[0] < 40
    sig, ab = _sphere_triplet_difference(xyz, w, rep_of=rep[label], **kw)
    s = shared.zeta_shared_sphere(xyz, w, h=h, **kw)
    e = oracle.zeta_sphere(xyz, w, **kw)
    dz = s["zeta"] - e["zeta"]
    scale = np.abs(e["zeta"]).max()
    np.testing.assert_allclose(dz, sig, rtol=1e-9, atol=1e-11 * scale)
    B = shared.shared_bound_sphere(xyz, w, h=h, **kw)
    assert np.all(np.abs(dz) <= ab + 1e-11 * scale)
    assert np.all(ab <= B + 1e-11 * scale)
    assert np.any(np.abs(dz) > 1e-6 * scale)


@pytest.mark.parametrize("h", [0.01, 0.03])
def test_sphere_bound_holds_on_a_field(h):
    xyz = _cap(900, 514, theta=0.3)
    w = synth.sphere_field(xyz / np.linalg.norm(xyz, axis=1, keepdims=True), seed=515, width=0.05)
    kw = dict(theta_min=0.005, theta_max=0.15, nbins=4, mmax=6)
    s = shared.zeta_shared_sphere(xyz, w, h=h, **kw)
    e = oracle.zeta_sphere(xyz, w, **kw)
    B = shared.shared_bound_sphere(xyz, w, h=h, **kw)
    dz = np.abs(s["zeta"] - e["zeta"])
    scale = np.abs(e["zeta"]).max()
    assert np.all(dz <= B + 1e-10 * scale)
    assert np.any(dz > 1e-8 * scale)


def test_sphere_bound_hand_geometry():
    # c at the pole and p = delta along the meridian phi = 0 share a cell.
    # j is at colatitude theta on the meridian phi = 90 deg.  In the right
    # spherical triangle (c, p, j) Napier's rule gives tan A = tan(theta) /
    # sin(delta) at p, so the transported direction (east) and p's direction
    # to j differ by beta_j = atan(sin(delta) / tan(theta)).  k lies on the
    # great circle through c and p, so beta_k = 0.  Bins [0.05, 0.15) and
    # [0.15, 0.25) hold j and k from both; w = (1, 2, 3, 5), so S = (3, 5),
    # A = (3 beta_j, 0), D = 0, and only p (|w_p| = 2) contributes.
    delta, theta, theta_k = 0.01, 0.1, 0.2
    pts = np.array([
        [0.0, 0.0, 1.0],
        [np.sin(delta), 0.0, np.cos(delta)],
        [0.0, np.sin(theta), np.cos(theta)],
        [-np.sin(theta_k), 0.0, np.cos(theta_k)],
    ])
    # the whole configuration rotated a little, so that c is off the cell faces
    g = 0.3
    R = np.array([[np.cos(g), 0.0, np.sin(g)], [0.0, 1.0, 0.0], [-np.sin(g), 0.0, np.cos(g)]])
    xyz = pts @ R.T
    w = np.array([1.0, 2.0, 3.0, 5.0])
    h = 0.04
    label, rep, _ = shared.pivot_groups(xyz, h)
    assert label[0] == label[1] and len({label[0], label[2], label[3]}) == 3
    kw = dict(theta_min=0.05, theta_max=0.25, nbins=2, mmax=4)
    B = shared.shared_bound_sphere(xyz, w, h=h, **kw)
    bj = np.arctan(np.sin(delta) / np.tan(theta))
    for m in range(5):
        want = 2.0 * np.array([[min(m * 18 * bj, 18.0), min(m * 15 * bj, 30.0)],
                               [min(m * 15 * bj, 30.0), 0.0]])
        np.testing.assert_allclose(B[m], want, rtol=1e-9, atol=1e-12)
