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


def alm_err(a, a_ref, w2_sum, lmax):
    """|a - a_ref| / sqrt((2l+1)/(4 pi) sum_{j in b} w_j^2) per (p, b, l, m), max.

    w2_sum[p, b] = sum of squared secondary weights in the bin: the natural
    scale of a sum of |w_j| sqrt((2l+1)/4pi)-bounded terms with random signs.
    """
    err = 0.0
    for l in range(lmax + 1):
        sl = slice(l * l, (l + 1) ** 2)
        scale = np.sqrt((2 * l + 1) / (4 * np.pi) * w2_sum)[:, :, None]
        diff = np.abs(np.asarray(a[:, :, sl], dtype=np.float64) - a_ref[:, :, sl])
        ok = scale > 0
        assert np.all(diff[~np.broadcast_to(ok, diff.shape)] < 1e-30)
        err = max(err, float(np.max(np.where(ok, diff / np.where(ok, scale, 1.0), 0.0))))
    return err
