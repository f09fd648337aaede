"""ctb_contract_noalloc: zeta from device-resident a_lm rows with no device
allocation by the library.

It serves callers that must not allocate device memory when they call in: a
service that reserves the whole device in its own pool up front and hands out
only fixed buffers, or a loop with a latency budget in which an allocation,
or its failure, is not acceptable.  Its scratch is a fixed array inside the
library, shared by all calls.

This file is collected last (pytest orders test files by name), so a run that
stops at the first failure has run every other test before it.
"""
import numpy as np
import pytest

import oracle
from paper_2604_08855_gb300 import synth
from tests.parity import zeta_err

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5   # the FP32-path tolerance of the other parity tests


def test_noalloc_matches_compute_subset_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_2604_08855_gb300 import build
    build.build()
    from paper_2604_08855_gb300 import ctb

    nbins, lmax = 8, 10
    xyz, w = synth.thomas(6000, 300.0, 60, 5.0, seed=41, weights="u0.5-1.5")
    kw = dict(box=300.0, rmin=2.0, rmax=45.0, nbins=nbins, lmax=lmax)
    est = ctb.CTB(**kw)
    est.set_points(xyz, w)
    prim = synth.sample_primaries(xyz.shape[0], 700, seed=4)
    z_existing = est.compute_subset(prim)  # the existing entry point

    dev = torch.device("cuda")
    alm = torch.empty((prim.size, nbins, (lmax + 1) ** 2), dtype=torch.float32, device=dev)
    est.get_alm(torch.from_numpy(prim).to(dev), out=alm)
    wp = torch.from_numpy(w[prim].astype(np.float32)).to(dev)  # the library's float32 weights
    scale = {"zeta": z_existing, "gram": oracle.zeta(xyz, w, prim=prim, **kw)["gram"]}

    for _ in range(2):  # the shared scratch keeps the previous call's contents
        out = torch.full((lmax + 1, nbins, nbins), float("nan"), dtype=torch.float64, device=dev)
        ctb.contract_noalloc(alm, wp, nbins, lmax, out)
        torch.cuda.synchronize()
        z = out.cpu().numpy()
        assert np.all(np.isfinite(z))
        assert zeta_err(z, scale) < TOL_FP32

    # sizes beyond the fixed scratch are rejected with CTB_ERR_ARG
    big = torch.zeros((1, 64, 441), dtype=torch.float32, device=dev)
    with pytest.raises(ctb.CTBError) as e:
        ctb.contract_noalloc(big, wp[:1], 64, 20, torch.zeros((21, 64, 64), dtype=torch.float64, device=dev))
    assert e.value.code == ctb.ERR_ARG
