"""ctb_contract_noalloc: zeta from device-resident a_lm rows with no device
allocation by the library.

It serves callers that must not allocate device memory when they call in: a
service that reserves the whole device in its own pool up front and hands out
only fixed buffers, or a loop with a latency budget in which an allocation,
or its failure, is not acceptable.  Its scratch is a fixed array inside the
library, shared by all calls.

Every case is held to the FP64 oracle (oracle.zeta for a real catalogue's
primaries, oracle.contract for given a_lm rows) and, where a catalogue
exists, to the existing entry point ctb_compute_subset.

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


def _lib():
    torch = pytest.importorskip("torch")
    from paper_2604_08855_gb300 import build
    build.build()
    from paper_2604_08855_gb300 import ctb
    return torch, ctb


def _contract_ref(alm, w, lmax):
    """The oracle's FP64 contraction of the given rows and its |w| Gram."""
    a = alm.double().cpu().numpy()
    wp = w.double().cpu().numpy()
    return {"zeta": oracle.contract(a, wp, lmax), "gram": oracle.contract(a, np.abs(wp), lmax)}


def test_noalloc_matches_oracle_and_compute_subset_on_two_calls():
    torch, ctb = _lib()
    nbins, lmax = 8, 10
    xyz, w = synth.thomas(6000, 300.0, 60, 5.0, seed=41, weights="u0.5-1.5")
    kw = dict(box=300.0, rmin=2.0, rmax=45.0, nbins=nbins, lmax=lmax)
    est = ctb.CTB(**kw)
    est.set_points(xyz, w)
    prim = synth.sample_primaries(xyz.shape[0], 700, seed=4)
    ref = oracle.zeta(xyz, w, prim=prim, **kw)
    z_existing = est.compute_subset(prim)  # the existing entry point
    assert zeta_err(z_existing, ref) < TOL_FP32

    dev = torch.device("cuda")
    alm = torch.empty((prim.size, nbins, (lmax + 1) ** 2), dtype=torch.float32, device=dev)
    est.get_alm(torch.from_numpy(prim).to(dev), out=alm)
    wp = torch.from_numpy(w[prim].astype(np.float32)).to(dev)  # the library's float32 weights

    for _ in range(2):  # the shared scratch keeps the previous call's contents
        out = torch.full((lmax + 1, nbins, nbins), float("nan"), dtype=torch.float64, device=dev)
        ctb.contract_noalloc(alm, wp, nbins, lmax, out)
        torch.cuda.synchronize()
        z = out.cpu().numpy()
        assert np.all(np.isfinite(z))
        assert zeta_err(z, ref) < TOL_FP32
        assert zeta_err(z, {"zeta": z_existing, "gram": ref["gram"]}) < TOL_FP32
    est.close()


def test_noalloc_200k_primaries_against_oracle_and_compute_subset():
    """Long per-block FP32 runs: 2e5 primaries of a real catalogue."""
    torch, ctb = _lib()
    nbins, lmax = 4, 6
    xyz, w = synth.thomas(200_000, 400.0, 2000, 3.0, seed=43, weights="u0.5-1.5")
    kw = dict(box=400.0, rmin=1.0, rmax=9.0, nbins=nbins, lmax=lmax)
    est = ctb.CTB(**kw)
    est.set_points(xyz, w)
    prim = np.arange(xyz.shape[0], dtype=np.int64)
    z_existing = est.compute_subset(prim)
    dev = torch.device("cuda")
    alm = torch.empty((prim.size, nbins, (lmax + 1) ** 2), dtype=torch.float32, device=dev)
    est.get_alm(torch.from_numpy(prim).to(dev), out=alm)
    wp = torch.from_numpy(w.astype(np.float32)).to(dev)
    ref = _contract_ref(alm, wp, lmax)
    for _ in range(2):
        out = torch.full((lmax + 1, nbins, nbins), float("nan"), dtype=torch.float64, device=dev)
        ctb.contract_noalloc(alm, wp, nbins, lmax, out)
        torch.cuda.synchronize()
        z = out.cpu().numpy()
        assert zeta_err(z, ref) < TOL_FP32
        assert zeta_err(z, {"zeta": z_existing, "gram": ref["gram"]}) < TOL_FP32
    est.close()


def test_noalloc_at_the_size_limit_on_a_side_stream():
    """(l_max+1) nbins^2 = 16 * 32^2 = 16384, the largest accepted shape, on a
    non-default stream, after a call with a smaller shape."""
    torch, ctb = _lib()
    dev = torch.device("cuda")
    g = torch.Generator(device="cpu").manual_seed(5)
    s = torch.cuda.Stream(device=dev)
    for nbins, lmax, npr in ((5, 3, 3000), (32, 15, 1500)):
        alm = torch.randn((npr, nbins, (lmax + 1) ** 2), generator=g, dtype=torch.float32).to(dev)
        wp = (torch.rand((npr,), generator=g, dtype=torch.float32) * 2.0 - 0.5).to(dev)
        ref = _contract_ref(alm, wp, lmax)
        out = torch.full((lmax + 1, nbins, nbins), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            ctb.contract_noalloc(alm, wp, nbins, lmax, out)  # defaults to the current (side) stream
        s.synchronize()
        assert zeta_err(out.cpu().numpy(), ref) < TOL_FP32


def test_noalloc_zero_primaries_and_argument_checks():
    torch, ctb = _lib()
    dev = torch.device("cuda")
    nbins, lmax = 6, 4
    alm = torch.zeros((0, nbins, (lmax + 1) ** 2), dtype=torch.float32, device=dev)
    wp = torch.zeros((0,), dtype=torch.float32, device=dev)
    out = torch.full((lmax + 1, nbins, nbins), float("nan"), dtype=torch.float64, device=dev)
    ctb.contract_noalloc(alm, wp, nbins, lmax, out)
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 0.0)

    # sizes beyond the fixed scratch are rejected with CTB_ERR_ARG
    big = torch.zeros((1, 33, 256), dtype=torch.float32, device=dev)
    with pytest.raises(ctb.CTBError) as e:
        ctb.contract_noalloc(big, wp.new_zeros(1), 33, 15, torch.zeros((16, 33, 33), dtype=torch.float64, device=dev))
    assert e.value.code == ctb.ERR_ARG

    # arguments the kernel could not read safely are refused before the call
    good = torch.zeros((3, nbins, (lmax + 1) ** 2), dtype=torch.float32, device=dev)
    w3 = torch.ones((3,), dtype=torch.float32, device=dev)
    bad = [
        (good.cpu(), w3, out),                          # host tensor
        (good.double(), w3, out),                       # wrong dtype
        (good.transpose(1, 2).contiguous().transpose(1, 2), w3, out),  # not contiguous
        (good[:, :, :-1].contiguous(), w3, out),        # wrong coefficient count
        (good, w3[:2], out),                            # one weight short
        (good, w3, out.float()),                        # out not float64
        (good, w3, out[:, :-1]),                        # wrong out shape
    ]
    for a, ww, o in bad:
        with pytest.raises(ValueError):
            ctb.contract_noalloc(a, ww, nbins, lmax, o)


@pytest.mark.parametrize("nbins,lmax,npr", [(1, 0, 50), (3, 2, 200), (4, 3, 300), (7, 5, 130), (20, 8, 400),
                                            (40, 9, 100), (64, 3, 64), (12, 1, 1000)])
def test_noalloc_shapes_against_oracle(nbins, lmax, npr):
    """The contraction's shape-dependent paths (threads per task, stage size,
    two blocks per SM, the scalar staging of rows whose length is not a
    multiple of 4) on random rows with weights of both signs."""
    torch, ctb = _lib()
    dev = torch.device("cuda")
    g = torch.Generator(device="cpu").manual_seed(1000 * nbins + lmax)
    alm = torch.randn((npr, nbins, (lmax + 1) ** 2), generator=g, dtype=torch.float32).to(dev)
    wp = (torch.rand((npr,), generator=g, dtype=torch.float32) * 2.0 - 0.5).to(dev)
    ref = _contract_ref(alm, wp, lmax)
    out = torch.full((lmax + 1, nbins, nbins), float("nan"), dtype=torch.float64, device=dev)
    ctb.contract_noalloc(alm, wp, nbins, lmax, out)
    torch.cuda.synchronize()
    z = out.cpu().numpy()
    assert np.all(np.isfinite(z))
    assert zeta_err(z, ref) < TOL_FP32
