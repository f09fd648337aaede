"""Error metrics for comparing a zeta or a_lm against the FP64 oracle.

zeta: max over (l, b1, b2) of |zeta - zeta_ref| / s, with
s = sqrt(G_l(b1,b1) G_l(b2,b2)) and G the oracle's |w_p|-weighted Gram
(the same contraction with |w_p|).  By Cauchy-Schwarz s >= |zeta_ref| when
w_p >= 0, and s stays meaningful for the near-zero off-diagonal l > 0 entries
that make a plain elementwise relative error ill-defined.
"""
import numpy as np


def zeta_err(z, ref):
    g = ref["gram"]
    d = np.sqrt(np.maximum(np.einsum("lii->li", g), 0.0))
    s = d[:, :, None] * d[:, None, :]
    diff = np.abs(np.asarray(z) - ref["zeta"])
    zero = s == 0
    assert np.all(diff[zero] == 0), "non-zero zeta where the oracle's Gram bound is zero"
    s = np.where(zero, 1.0, s)
    return float(np.max(diff / s))


def alm_err(a, a_ref, w1_sum, lmax):
    """|a - a_ref| / (sqrt((2l+1)/(4 pi)) sum_{j in b} |w_j|) per (p, b, l, m), max.

    w1_sum[p, b] = sum of |w_j| over the bin's secondaries, so the scale is
    the bound on every term's magnitude summed: the scale of the forward
    error of a floating-point sum (sum |terms| times the unit roundoff and
    the evaluation's conditioning).  A root-sum-square scale would assume
    that rounding errors cancel at random; the moments of a factored
    polynomial basis do not guarantee that (their conversion to a_lm
    cancels, by up to a few tens at l = 10).
    """
    err = 0.0
    for l in range(lmax + 1):
        sl = slice(l * l, (l + 1) ** 2)
        scale = (np.sqrt((2 * l + 1) / (4 * np.pi)) * w1_sum)[:, :, None]
        diff = np.abs(np.asarray(a[:, :, sl], dtype=np.float64) - a_ref[:, :, sl])
        ok = scale > 0
        assert np.all(diff[~np.broadcast_to(ok, diff.shape)] < 1e-30)
        err = max(err, float(np.max(np.where(ok, diff / np.where(ok, scale, 1.0), 0.0))))
    return err


def zeta_err_elementwise(z, ref, floor=1e-3):
    """Plain relative error max |dzeta| / |zeta_ref| over the entries with
    |zeta_ref| >= floor * max_l |zeta_ref| (a secondary metric beside the Gram one)."""
    zr = ref["zeta"]
    big = np.abs(zr) >= floor * np.abs(zr).max(axis=(1, 2), keepdims=True)
    big &= np.abs(zr) > 0
    d = np.abs(np.asarray(z) - zr)
    return float(np.max(np.where(big, d / np.where(big, np.abs(zr), 1.0), 0.0)))


def zeta_err_normwise(z, ref):
    """Per-l normwise error max_(b1,b2) |dzeta_l| / max_(b1,b2) |zeta_ref_l|,
    the largest over l (the other secondary metric)."""
    zr = ref["zeta"]
    d = np.abs(np.asarray(z) - zr).max(axis=(1, 2))
    m = np.abs(zr).max(axis=(1, 2))
    return float(np.max(np.where(m > 0, d / np.where(m > 0, m, 1.0), np.where(d > 0, np.inf, 0.0))))


def bin_flip_bound(xyz, w, kw, prim, amb):
    """Elementwise bound on |zeta - zeta_ref| from pairs that a binning of
    rounded coordinates may put across a bin edge from the FP64 oracle.

    amb = oracle.ambiguous(...) for the same primaries.  For each primary
    with ambiguous pairs, its own a_lm rows (oracle.alm) are modified by
    every subset of those pairs switching to the other side of their edge
    (leaving or entering the bin range at the outer edges), and the largest
    change of its zeta term per entry is taken; the bound is the sum over
    primaries.  Also returns the bound on the pair sums per bin and the
    number of ambiguous pairs at the outer edges (the most the pair counts
    can differ by).
    """
    import oracle
    idx, d, r, edge = amb
    lmax, nb = kw["lmax"], kw["nbins"]
    box, rmin, rmax = kw["box"], kw["rmin"], kw["rmax"]
    dr = (rmax - rmin) / nb
    wv = np.ones(xyz.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    bz = np.zeros((lmax + 1, nb, nb))
    bp = np.zeros(nb)
    outer = int(np.sum((edge == 0) | (edge == nb)))
    for i in np.unique(idx[:, 0]) if len(idx) else []:
        sel = np.nonzero(idx[:, 0] == i)[0]
        if len(sel) > 10:
            raise ValueError("too many ambiguous pairs for one primary to enumerate")
        p = int(prim[i]) if prim is not None else int(i)
        a = oracle.alm(xyz, wv, box, rmin, rmax, nb, lmax, prim=np.array([p]))[0]
        z0 = oracle.contract(a[None], np.array([wv[p]]), lmax)
        moves = []
        for t in sel:
            k, j = int(edge[t]), int(idx[t, 1])
            below = k - 1 if k >= 1 else None
            above = k if k < nb else None
            cur, alt = (above, below) if r[t] >= rmin + k * dr else (below, above)
            y = wv[j] * oracle.ylm(lmax, d[t] / r[t])[0]
            moves.append((cur, alt, y))
            bp += abs(wv[p] * wv[j]) * np.array([(b == cur or b == alt) for b in range(nb)], dtype=float)
        worst = np.zeros_like(bz)
        for mask in range(1, 1 << len(moves)):
            a2 = a.copy()
            for bit, (cur, alt, y) in enumerate(moves):
                if mask >> bit & 1:
                    if cur is not None:
                        a2[cur] -= y
                    if alt is not None:
                        a2[alt] += y
            worst = np.maximum(worst, np.abs(oracle.contract(a2[None], np.array([wv[p]]), lmax) - z0))
        bz += worst
    return bz, bp, outer


def zeta_err_with_flips(z, ref, flip):
    """The Gram-normalised error after granting each entry its bin-flip
    bound: max over entries of max(0, |dzeta| - bound) / s."""
    g = ref["gram"]
    dg = np.sqrt(np.maximum(np.einsum("lii->li", g), 0.0))
    s = dg[:, :, None] * dg[:, None, :]
    diff = np.maximum(np.abs(np.asarray(z) - ref["zeta"]) - flip, 0.0)
    zero = s == 0
    assert np.all(diff[zero] == 0), "non-zero zeta where the oracle's Gram bound is zero"
    return float(np.max(diff / np.where(zero, 1.0, s)))
