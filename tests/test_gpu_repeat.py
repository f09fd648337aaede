"""Bitwise repeatability (GPU).

Every reduction on the path has a fixed order: the neighbour lists are
written in candidate order, each (primary, bin) list is summed by one warp,
each contraction block owns its partial rows, and the FP64 partials are
added in a fixed order.  So the same inputs with the same configuration give
the same bits, whichever warp takes which primary.  These tests run each mode
twice on one context and once on a fresh one, and compare bit for bit.
Compute-sanitizer's race detection is not available here; a race in any of
these reductions would show up as a difference.
"""
import numpy as np
import pytest

from paper_2604_08855_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctbmod():
    from paper_2604_08855_gb300 import build
    build.build()
    from paper_2604_08855_gb300 import ctb
    return ctb


def three(ctbmod, make, run):
    outs = []
    est = make()
    outs.append(run(est))
    outs.append(run(est))
    outs.append(run(make()))
    return outs


@pytest.mark.parametrize("box,prec", [(300.0, "FP32"), (0.0, "FP32"), (300.0, "BF16X3")])
def test_zeta_pair_sums_alm_repeat_bitwise(ctbmod, box, prec):
    xyz, w = synth.thomas(20000, 300.0, 200, 5.0, seed=91, weights="u0.5-1.5")
    prim = synth.sample_primaries(xyz.shape[0], 50, seed=9)

    def make():
        est = ctbmod.CTB(box, 2.0, 40.0, 8, 8)
        est.set_option(ctbmod.OPT_CELLS_PER_RMAX, 6)
        est.set_option(ctbmod.OPT_PRECISION, getattr(ctbmod, "PREC_" + prec))
        est.set_points(xyz, w)
        return est

    def run(est):
        z = est.compute()
        return z, est.pair_sums(), est.get_alm(prim), est.pair_count()

    outs = three(ctbmod, make, run)
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0])
        assert np.array_equal(o[1], outs[0][1])
        assert np.array_equal(o[2], outs[0][2])
        assert o[3] == outs[0][3]


def test_sphere_repeat_bitwise(ctbmod):
    xyz = synth.fibonacci_sphere(30000)
    w = synth.sphere_field(xyz, seed=92)

    def make():
        est = ctbmod.CTB.sphere(0.0, 0.12, 6, 8)
        est.set_option(ctbmod.OPT_CELLS_PER_RMAX, 4)
        est.set_points(xyz, w)
        return est

    outs = three(ctbmod, make, lambda est: est.compute())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_batch_repeat_bitwise(ctbmod):
    cats = [synth.thomas(n, 300.0, max(1, n // 100), 5.0, seed=93 + i) for i, n in enumerate([4000, 900, 2500])]

    def make():
        return ctbmod.CTB(300.0, 2.0, 40.0, 5, 6)

    outs = three(ctbmod, make, lambda est: est.compute_batch(cats))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_shared_lists_repeat_bitwise(ctbmod):
    xyz, w = synth.thomas(20000, 300.0, 200, 5.0, seed=94, weights="u0.5-1.5")

    def make():
        est = ctbmod.CTB(300.0, 2.0, 40.0, 8, 8)
        est.set_points(xyz, w)
        return est

    def run(est):
        return est.compute_shared(0.0), est.pair_sums(), est.pivot_groups()

    outs = three(ctbmod, make, run)
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0])
        assert np.array_equal(o[1], outs[0][1])
        assert o[2] == outs[0][2]
