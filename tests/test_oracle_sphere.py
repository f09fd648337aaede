"""Pins of the oracle's projected (angular) multipoles on the sphere (CPU).

zeta_m(b1,b2) = sum_p w_p sum_{j in b1, k in b2} w_j w_k cos(m (phi_pj - phi_pk)),
bins in the angle theta = 2 asin(chord / 2).  The pins do not use the
oracle's tangent frame:

- a frame-free triplet sum: the angle between the tangent projections of
  n_j - n_p and n_k - n_p at p;
- m = 0: sum_p w_p N_p(b1) N_p(b2) with N_p from scipy's cKDTree;
- hand geometries: a pivot at the pole and one on the equator, two
  neighbours at known position angles;
- invariance under a random rotation, symmetry, PSD for w >= 0.
"""
import numpy as np
import pytest

import oracle


def cap_points(n, seed, theta_cap=0.3, centre=(0.2, -0.3, 0.93)):
    """n unit vectors uniform in a spherical cap (so that most pairs fall in range)."""
    rng = np.random.default_rng(seed)
    c = np.asarray(centre, float)
    c /= np.linalg.norm(c)
    cosmax = np.cos(theta_cap)
    mu = rng.uniform(cosmax, 1.0, n)
    ph = rng.uniform(0, 2 * np.pi, n)
    s = np.sqrt(1 - mu * mu)
    local = np.stack([s * np.cos(ph), s * np.sin(ph), mu], axis=1)
    # rotate z to c
    z = np.array([0.0, 0.0, 1.0])
    v = np.cross(z, c)
    sn, cs = np.linalg.norm(v), z @ c
    if sn < 1e-12:
        return local
    k = v / sn
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    R = np.eye(3) + sn * K + (1 - cs) * K @ K
    return local @ R.T


def chord_edges(tmin, tmax, nbins):
    return 2.0 * np.sin(0.5 * np.linspace(tmin, tmax, nbins + 1))


def triplets(xyz, w, tmin, tmax, nbins, mmax):
    e = chord_edges(tmin, tmax, nbins)
    n = xyz.shape[0]
    z = np.zeros((mmax + 1, nbins, nbins))
    for p in range(n):
        d = xyz - xyz[p]
        c = np.linalg.norm(d, axis=1)
        ok = (c > 0) & (c >= e[0]) & (c < e[-1])
        ok[p] = False
        idx = np.nonzero(ok)[0]
        if idx.size == 0:
            continue
        b = np.searchsorted(e, c[idx], side="right") - 1
        nh = xyz[p] / np.linalg.norm(xyz[p])
        t = d[idx] - np.outer(d[idx] @ nh, nh)          # tangent projections at p
        tn = t / np.linalg.norm(t, axis=1)[:, None]
        cosd = np.clip(tn @ tn.T, -1.0, 1.0)
        sind = np.einsum("i,jki->jk", nh, np.cross(tn[:, None, :], tn[None, :, :]))
        dphi = np.arctan2(sind, cosd)                   # signed angle between the two sides
        ww = w[idx][:, None] * w[idx][None, :]
        for m in range(mmax + 1):
            val = w[p] * ww * np.cos(m * dphi)
            np.add.at(z[m], (b[:, None].repeat(idx.size, 1), b[None, :].repeat(idx.size, 0)), val)
    return z


@pytest.mark.parametrize("seed", [0, 1])
def test_against_frame_free_triplets(seed):
    xyz = cap_points(120, seed)
    w = np.random.default_rng(seed + 10).uniform(-1.0, 2.0, xyz.shape[0])
    kw = dict(theta_min=0.02, theta_max=0.5, nbins=4, mmax=6)
    got = oracle.zeta_sphere(xyz, w, **kw)["zeta"]
    want = triplets(xyz, w, kw["theta_min"], kw["theta_max"], kw["nbins"], kw["mmax"])
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-10 * np.abs(want).max())


def test_m0_is_the_product_of_neighbour_counts():
    scipy_spatial = pytest.importorskip("scipy.spatial")
    xyz = cap_points(400, 3)
    w = np.random.default_rng(4).uniform(0.5, 1.5, xyz.shape[0])
    tmin, tmax, nb = 0.01, 0.4, 5
    e = chord_edges(tmin, tmax, nb)
    tree = scipy_spatial.cKDTree(xyz)
    nbr = np.zeros((xyz.shape[0], nb))
    for p in range(xyz.shape[0]):
        for b in range(nb):
            inner = set(tree.query_ball_point(xyz[p], e[b] * (1 - 1e-12)))
            outer = set(tree.query_ball_point(xyz[p], e[b + 1] * (1 - 1e-12)))
            js = [j for j in outer - inner if j != p]
            nbr[p, b] = w[js].sum()
    want = np.einsum("p,pa,pb->ab", w, nbr, nbr)
    got = oracle.zeta_sphere(xyz, w, tmin, tmax, nb, 0)["zeta"][0]
    np.testing.assert_allclose(got, want, rtol=1e-12)


@pytest.mark.parametrize("pivot", [(0.0, 0.0, 1.0), (1.0, 0.0, 0.0)])
def test_hand_geometry(pivot):
    p = np.asarray(pivot)
    # tangent directions at the pivot, any orthonormal pair
    a = np.cross(p, [0.3, 0.4, 0.5])
    a /= np.linalg.norm(a)
    bvec = np.cross(p, a)
    th1, th2, phi1, phi2 = 0.10, 0.25, 0.7, 2.3
    def at(theta, phi):
        return np.cos(theta) * p + np.sin(theta) * (np.cos(phi) * a + np.sin(phi) * bvec)
    xyz = np.stack([p, at(th1, phi1), at(th2, phi2)])
    w = np.array([2.0, 3.0, 5.0])
    # bins [0.05, 0.15), [0.15, 0.3): j1 in bin 0, j2 in bin 1; only the pivot
    # has both neighbours in range
    r = oracle.zeta_sphere(xyz, w, 0.05, 0.3, 2, 5, prim=[0])
    for m in range(6):
        z = r["zeta"][m]
        assert z[0, 1] == pytest.approx(2 * 3 * 5 * np.cos(m * (phi1 - phi2)), abs=1e-12)
        assert z[1, 0] == pytest.approx(z[0, 1], abs=1e-12)
        assert z[0, 0] == pytest.approx(2 * 9.0, abs=1e-12)
        assert z[1, 1] == pytest.approx(2 * 25.0, abs=1e-12)
    assert r["npairs"] == 2
    np.testing.assert_allclose(r["wpairs"], [6.0, 10.0])


def test_rotation_invariance_symmetry_psd():
    xyz = cap_points(300, 7, theta_cap=0.4, centre=(0.0, 0.01, 1.0))  # straddles the pole
    w = np.random.default_rng(8).uniform(0.5, 1.5, xyz.shape[0])
    kw = dict(theta_min=0.01, theta_max=0.45, nbins=5, mmax=8)
    z0 = oracle.zeta_sphere(xyz, w, **kw)["zeta"]
    q, _ = np.linalg.qr(np.random.default_rng(9).normal(size=(3, 3)))
    z1 = oracle.zeta_sphere(xyz @ q.T, w, **kw)["zeta"]
    np.testing.assert_allclose(z1, z0, rtol=1e-9, atol=1e-9 * np.abs(z0).max())
    np.testing.assert_allclose(z0, np.swapaxes(z0, 1, 2), rtol=1e-13)
    for m in range(kw["mmax"] + 1):
        assert np.linalg.eigvalsh(z0[m]).min() > -1e-9 * np.abs(z0[m]).max()
