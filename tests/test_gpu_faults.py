"""Failure detection through the C ABI, without faulting the GPU.

A bounded device wait is made to run out (the tensor-core contraction waits on
a barrier that nothing signals, with a ~10 ms limit), and device allocations
are made to fail on the host side.  Each returns its status code, and the same
context then computes the right answer.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2604_08855_gb300 import synth
from tests.parity import zeta_err

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-3


@pytest.fixture(scope="module")
def ctbmod():
    from paper_2604_08855_gb300 import build
    build.build()
    from paper_2604_08855_gb300 import ctb
    return ctb


def small():
    xyz, w = synth.uniform(300, 100.0, seed=40)
    kw = dict(box=100.0, rmin=1.0, rmax=30.0, nbins=3, lmax=2)
    return xyz, w, kw


def test_injected_wait_timeout_is_reported_and_context_recovers(ctbmod):
    xyz, w, kw = small()
    est = ctbmod.CTB(**kw)
    est.set_option(ctbmod.OPT_PRECISION, ctbmod.PREC_BF16X3)
    est.set_points(xyz, w)
    est.set_option(ctbmod.OPT_FAULT_INJECT, ctbmod.INJECT_STALL)
    t0 = time.perf_counter()
    with pytest.raises(ctbmod.CTBError) as e:
        est.compute()
    assert e.value.code == ctbmod.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    est.set_option(ctbmod.OPT_FAULT_INJECT, 0)
    z = est.compute()
    assert zeta_err(z, oracle.zeta(xyz, w, **kw)) < TOL_MIXED


def test_injected_allocation_failure_is_oom_and_context_recovers(ctbmod):
    xyz, w, kw = small()
    est = ctbmod.CTB(**kw)
    est.set_option(ctbmod.OPT_FAULT_INJECT, ctbmod.INJECT_ALLOC)
    with pytest.raises(ctbmod.CTBError) as e:
        est.set_points(xyz, w)
    assert e.value.code == ctbmod.ERR_OOM
    with pytest.raises(ctbmod.CTBError) as e:
        est.compute()
    assert e.value.code == ctbmod.ERR_STATE
    est.set_option(ctbmod.OPT_FAULT_INJECT, 0)
    est.set_points(xyz, w)
    z = est.compute()
    assert np.isfinite(z).all()
    assert zeta_err(z, oracle.zeta(xyz, w, **kw)) < 1e-5


def test_unknown_fault_is_rejected(ctbmod):
    est = ctbmod.CTB(box=100.0, rmin=1.0, rmax=30.0, nbins=3, lmax=2)
    with pytest.raises(ctbmod.CTBError) as e:
        est.set_option(ctbmod.OPT_FAULT_INJECT, 7)
    assert e.value.code == ctbmod.ERR_ARG
