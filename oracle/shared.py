"""Shared neighbour lists for close pivots: FP64 oracle (test infrastructure).

Paper, "Implementation": pivots that lie close to one another share one
neighbour list.  Closeness is a pivot radius, set from the catalogue's mean
separation unless the user gives one.  The paper gives no formula for the
resulting estimate, so these functions state the reading the library
implements:

- Groups.  A point belongs to the pivot cell (floor(x/h), floor(y/h),
  floor(z/h)) of side h, with cells aligned at the origin of coordinates.
  Periodic coordinates are wrapped into [0, box) first.
- Representative.  Each group is represented by its member of smallest
  catalogue index, c_g.  Its weight is W_g = sum of the members' weights.
- Estimate.  Every member takes the representative's neighbour list and
  multipoles:

      zeta_l(b1, b2) ~= 4 pi/(2l+1) sum_g W_g sum_m a_lm(c_g, b1) a_lm(c_g, b2)

  The neighbour sums keep their own weights.  On the sphere the same holds
  with the projected a_m of ``oracle.zeta_sphere``.
- Error bound.  ``shared_bound`` bounds |shared - exact| entry by entry.
  Take a member p with representative c, and neighbours j and k.  Both
  estimates are sums over (p, j, k) of w_p w_j w_k P_l(cos gamma), where
  gamma is the angle between the two separations (addition theorem).  The
  shared one takes the separations from c instead of p.
  - When j and k are in bins b1 and b2 as seen from both p and c, the two
    angles differ by at most alpha_j + alpha_k.  Here alpha_j is the angle
    between x_j - x_p and x_j - x_c.  P_l(cos gamma) is a trigonometric
    polynomial of degree l in gamma with modulus at most 1, so by
    Bernstein's inequality its derivative is at most l in modulus.  The
    term therefore changes by at most l (alpha_j + alpha_k), and never by
    more than 2.
  - When one of j, k changes bin membership between p and c, the term
    changes by at most |w_p w_j w_k|.
  Summed, with S_b, A_b the |w|-sums (plain and times alpha) over j in bin b
  from both points, D_b over j in b from exactly one, and U_b over j in b
  from either:

      |dzeta_l(b1, b2)| <= sum_p |w_p| [ min(l (A1 S2 + S1 A2), 2 S1 S2)
                                         + D1 U2 + U1 D2 ]

  A representative contributes nothing.

Parity status (what pins each function is in tests/test_oracle_shared.py):
  pivot_groups    pinned: hand-placed points with their cells, wrap and
                  representatives written out.
  zeta_shared     pinned: equals oracle.zeta when every group is one point,
                  and when each group is a pair of coincident points (a
                  catalogue and its copy); it lies within shared_bound of
                  oracle.zeta.
  shared_bound    pinned: an O(N^3) triplet sum of |term differences| with
                  scipy's Legendre polynomials lies between |dzeta| and the
                  bound.  The bound is zero for singleton and coincident
                  groups, and linear in the displacement where no
                  membership changes.
  zeta_shared_sphere  pinned: equals oracle.zeta_sphere for singleton groups
                  and coincident pairs; lies within shared_bound_sphere of it.
  shared_bound_sphere  pinned: an O(N^3) triplet sum of |term differences|,
                  with each pivot's angles taken from its own tangent frame,
                  lies between |dzeta| and the bound; zero for singleton and
                  coincident groups.

Sphere bound.  zeta_m = sum_p w_p sum_{j,k} w_j w_k cos(m psi_p(j,k)), psi_p
the signed angle between the tangent-plane projections at p of n_j - n_p
and n_k - n_p.  The rotation R that takes c's normal to p's maps c's tangent
plane onto p's and keeps signed angles.  So psi_c - psi_p is at most
beta_j + beta_k (mod 2 pi), beta_j being the angle between p's projection
of j and R applied to c's.  |d/dpsi cos(m psi)| <= m, so the same sum as in
3-D holds, with beta for alpha and m for l (beta = pi where a projection
vanishes).
"""
from __future__ import annotations

import numpy as np

from .oracle import zeta, zeta_sphere


def pivot_groups(xyz, h, box=0.0, w=None):
    """Groups of the catalogue by pivot cell of side h.

    Returns ``(label, rep, W)``.  ``label[i]`` is the group of point i.
    ``rep[g]`` is the smallest index in group g.  ``W[g]`` is the sum of the
    members' weights (1 each when ``w`` is None).  Groups are numbered in
    order of their representatives.
    """
    return _groups(np.asarray(xyz, dtype=np.float64), w, float(h), float(box))


def _groups(xyz, w, h, box):
    if not (h > 0.0) or not np.isfinite(h):
        raise ValueError("pivot cell side must be positive and finite")
    x = xyz
    if box > 0.0:
        x = np.mod(x, box)
        x = np.where(x >= box, 0.0, x)
    cells = np.floor(x / h).astype(np.int64)
    n = x.shape[0]
    _, first, inv = np.unique(cells, axis=0, return_index=True, return_inverse=True)
    inv = inv.reshape(-1)
    rep_u = np.full(first.shape[0], n, dtype=np.int64)
    np.minimum.at(rep_u, inv, np.arange(n, dtype=np.int64))
    order = np.argsort(rep_u, kind="stable")  # number groups by representative
    relabel = np.empty_like(order)
    relabel[order] = np.arange(order.shape[0])
    label = relabel[inv]
    rep = rep_u[order]
    W = np.zeros(rep.shape[0])
    ww = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    for i in range(n):  # members in index order, FP64
        W[label[i]] += ww[i]
    return label, rep, W


def mean_separation(xyz, box=0.0, rmax=0.0):
    """The automatic pivot cell side: (V / n)^(1/3), with V = box^3 (periodic),
    else the product of the bounding box's sides, each at least rmax."""
    xyz = np.asarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    if box > 0.0:
        vol = box ** 3
    else:
        vol = float(np.prod(np.maximum(xyz.max(axis=0) - xyz.min(axis=0), rmax)))
    return float(np.cbrt(vol / n))


def zeta_shared(xyz, w, box, rmin, rmax, nbins, lmax, h, nthreads=0):
    """The shared-list estimate of zeta_l(b1, b2) (module docstring).

    Returns ``oracle.zeta``'s dict (its ``gram`` with |W_g|) plus ``rep``,
    ``W`` and ``label``.
    """
    xyz = np.asarray(xyz, dtype=np.float64)
    label, rep, W = _groups(xyz, w, float(h), float(box))
    res = zeta(xyz, w, box, rmin, rmax, nbins, lmax, prim=rep, nthreads=nthreads, wprim=W)
    res.update(rep=rep, W=W, label=label)
    return res


def zeta_shared_sphere(xyz, w, theta_min, theta_max, nbins, mmax, h, nthreads=0):
    """The shared-list estimate of the projected zeta_m on the sphere; the
    pivot cells are cubes of side h in the embedding space."""
    xyz = np.asarray(xyz, dtype=np.float64)
    label, rep, W = _groups(xyz, w, float(h), 0.0)
    res = zeta_sphere(xyz, w, theta_min, theta_max, nbins, mmax, prim=rep, nthreads=nthreads, wprim=W)
    res.update(rep=rep, W=W, label=label)
    return res


def _separations(xyz, i, box):
    """x_j - x_i for every j (minimum image when periodic)."""
    d = xyz - xyz[i]
    if box > 0.0:
        d = d - box * np.rint(d / box)
    return d


def _bins(d, self_idx, rmin, rmax, nbins):
    """Bin of every separation as oracle.zeta decides it (-1: not binned)."""
    dr = (rmax - rmin) / nbins
    r = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2])
    ok = (r >= rmin) & (r < rmax) & (r != 0.0)
    ok[self_idx] = False
    b = np.clip(np.floor((r - rmin) / dr), 0, nbins - 1).astype(np.int64)
    for _ in range(4):  # settle rounding at an edge against the edge values
        down = (b > 0) & (r < rmin + b * dr)
        b = b - down
        up = (b + 1 < nbins) & (r >= rmin + (b + 1) * dr)
        b = b + up
    return np.where(ok, b, -1)


def _angle(u, v):
    cr = np.cross(u, v)
    return np.arctan2(np.sqrt(np.sum(cr * cr, axis=1)), np.sum(u * v, axis=1))


def shared_bound(xyz, w, box, rmin, rmax, nbins, lmax, h):
    """Entrywise bound [lmax+1][nbins][nbins] on |zeta_shared - zeta| (module
    docstring), by brute force over every member and every neighbour."""
    xyz = np.asarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    ww = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    aw = np.abs(ww)
    label, rep, _ = _groups(xyz, ww, float(h), float(box))
    ells = np.arange(lmax + 1, dtype=np.float64)[:, None, None]
    B = np.zeros((lmax + 1, nbins, nbins))
    for p in range(n):
        c = int(rep[label[p]])
        if c == p:
            continue
        dp = _separations(xyz, p, box)
        dc = _separations(xyz, c, box)
        bp = _bins(dp, p, rmin, rmax, nbins)
        bc = _bins(dc, c, rmin, rmax, nbins)
        same = (bp == bc) & (bp >= 0)
        alpha = np.zeros(n)
        alpha[same] = _angle(dp[same], dc[same])
        S = np.zeros(nbins)
        A = np.zeros(nbins)
        D = np.zeros(nbins)
        U = np.zeros(nbins)
        for b in range(nbins):
            ip = bp == b
            ic = bc == b
            both = ip & ic
            S[b] = aw[both].sum()
            A[b] = (aw[both] * alpha[both]).sum()
            D[b] = aw[ip ^ ic].sum()
            U[b] = aw[ip | ic].sum()
        ang = np.minimum(ells * (np.outer(A, S) + np.outer(S, A))[None], 2.0 * np.outer(S, S)[None])
        mem = np.outer(D, U) + np.outer(U, D)
        B += aw[p] * (ang + mem[None])
    return B


def _sphere_edges(theta_min, theta_max, nbins):
    """Chord edges 2 sin(theta_b / 2), computed as oracle.zeta_sphere does (libm sin)."""
    import math
    return np.array([2.0 * math.sin(0.5 * (theta_min + b * (theta_max - theta_min) / nbins))
                     for b in range(nbins + 1)])


def _sphere_bins(xyz, i, edges):
    """Bin of every chord from point i as oracle.zeta_sphere decides it (-1: none)."""
    d = xyz - xyz[i]
    c = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2])
    ok = (c > 0.0) & (c >= edges[0]) & (c < edges[-1])
    ok[i] = False
    b = np.searchsorted(edges, c, side="right") - 1
    return np.where(ok, b, -1)


def _tangent_dirs(xyz, i):
    """Unit tangent-plane directions at point i of x_j - x_i, and where they exist."""
    n = xyz[i] / np.linalg.norm(xyz[i])
    d = xyz - xyz[i]
    t = d - np.outer(d @ n, n)
    nt = np.linalg.norm(t, axis=1)
    ok = nt > 0.0
    t[ok] /= nt[ok, None]
    return t, ok


def _rotation(a, b):
    """Rotation taking the unit vector a to the unit vector b (about a x b)."""
    v = np.cross(a, b)
    s = np.linalg.norm(v)
    c = float(a @ b)
    if s == 0.0:
        if c > 0.0:
            return np.eye(3)
        p = np.array([1.0, 0.0, 0.0]) if abs(a[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        k = np.cross(a, p)
        k /= np.linalg.norm(k)
        return 2.0 * np.outer(k, k) - np.eye(3)  # half turn about k, which is orthogonal to a
    k = v / s
    K = np.array([[0.0, -k[2], k[1]], [k[2], 0.0, -k[0]], [-k[1], k[0], 0.0]])
    return np.eye(3) + s * K + (1.0 - c) * (K @ K)


def shared_bound_sphere(xyz, w, theta_min, theta_max, nbins, mmax, h):
    """Entrywise bound [mmax+1][nbins][nbins] on |zeta_shared_sphere -
    zeta_sphere| (module docstring), by brute force over every member and
    every neighbour."""
    xyz = np.asarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    ww = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    aw = np.abs(ww)
    label, rep, _ = _groups(xyz, ww, float(h), 0.0)
    edges = _sphere_edges(theta_min, theta_max, nbins)
    ms = np.arange(mmax + 1, dtype=np.float64)[:, None, None]
    B = np.zeros((mmax + 1, nbins, nbins))
    for p in range(n):
        c = int(rep[label[p]])
        if c == p:
            continue
        bp = _sphere_bins(xyz, p, edges)
        bc = _sphere_bins(xyz, c, edges)
        same = (bp == bc) & (bp >= 0)
        tp, okp = _tangent_dirs(xyz, p)
        tc, okc = _tangent_dirs(xyz, c)
        R = _rotation(xyz[c] / np.linalg.norm(xyz[c]), xyz[p] / np.linalg.norm(xyz[p]))
        tcr = tc @ R.T
        beta = np.full(n, np.pi)
        good = same & okp & okc
        cr = np.cross(tp[good], tcr[good])
        beta[good] = np.arctan2(np.sqrt(np.sum(cr * cr, axis=1)), np.sum(tp[good] * tcr[good], axis=1))
        S = np.zeros(nbins)
        A = np.zeros(nbins)
        D = np.zeros(nbins)
        U = np.zeros(nbins)
        for b in range(nbins):
            ip = bp == b
            ic = bc == b
            both = ip & ic
            S[b] = aw[both].sum()
            A[b] = (aw[both] * beta[both]).sum()
            D[b] = aw[ip ^ ic].sum()
            U[b] = aw[ip | ic].sum()
        ang = np.minimum(ms * (np.outer(A, S) + np.outer(S, A))[None], 2.0 * np.outer(S, S)[None])
        mem = np.outer(D, U) + np.outer(U, D)
        B += aw[p] * (ang + mem[None])
    return B
