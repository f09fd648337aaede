"""Benchmark: Legendre-multipole 3PCF on one GB300 (prints one JSON line).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision mixed|fp32|bf16x3|tf32] [--workload thomas_4m]

A step is one full pass of the hot path over the workload: ingest + cell sort
(ctb_set_points from device-resident float64 inputs), pair multipoles,
contraction and the FP64 reduction (ctb_compute).  Default workload: the
precision configuration, 4,000,000 Thomas-process points in a periodic cube
L = 2000 (40,000 parents, sigma = 5, weights U[0.5, 1.5], seed 2), r in
[10, 200] with 32 linear bins, l_max = 20.

Default precision "mixed": the same catalogue is timed in plain FP32 (FP32
pair kernel and contraction) and then with the BF16 hi/lo tensor-core
contraction; the line's value is the mixed form, `plain_fp32` holds the plain
form and `mixed_over_plain` their ratio; a short TF32 run is an extra field.

value  pair-multipole updates/s = binned ordered pairs x (l_max+1)^2 / step time
e2e    the same through the C ABI with HOST float64 inputs and a HOST zeta
       (host->device copies and the result read-back inside the timed region)

Under torchrun (N > 1) each rank computes its shard of the primaries of the
one catalogue (every point a secondary) and the ranks sum zeta with one FP64
all-reduce: one zeta per step over all GPUs (strong scaling).

--impl reference times the FP64 CPU oracle (the slow, obviously correct
restatement of the method) on a bounded sample of primaries of the same
workload, on the host cores.  Under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pair-multipole updates/s and ms per zeta_ell at 1 GB300 (mixed vs plain FP32, <=1e-3 rel err)"
UNIT = "updates/s"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 152
# Algorithmic work of the accumulation step per (pair, coefficient) update:
# about one FMA to accumulate plus the recurrence share, in FP32 instructions.
INST_PER_UPDATE = 2.6
# DRAM bytes per pair of the accumulation kernel from one ncu capture of the
# current k_alm (dram__bytes_read.sum + dram__bytes_write.sum over the pairs of
# the captured launches, summed over the m-pass launches of one chunk: one at
# l_max 10, three at l_max 20).  Keyed by l_max; a missing entry reports null
# traffic.
K_ALM_DRAM_BYTES_PER_PAIR = {10: 4.383, 20: 21.17}
FP32_LANES_PER_SM = 128


def workload(name: str):
    from paper_2604_08855_gb300 import synth
    if name == "thomas_1m":
        xyz, w = synth.thomas_1m()
        return xyz, w, synth.config_params(2), {
            "workload": "thomas_1m", "n_points": 1_000_000, "box": 1000.0, "r_min": 5.0, "r_max": 200.0,
            "nbins": 20, "ell_max": 10, "periodic": True, "clustering": "Thomas, 10k parents, sigma 5",
            "weights": "U[0.5,1.5]"}
    if name == "uniform_20k":
        xyz, w = synth.uniform_20k()
        return xyz, w, synth.config_params(1), {
            "workload": "uniform_20k", "n_points": 20_000, "box": 1000.0, "r_min": 10.0, "r_max": 100.0,
            "nbins": 10, "ell_max": 10, "periodic": True, "weights": "unit"}
    if name == "cut_sky":
        xyz, w = synth.cut_sky()
        return xyz, w, synth.config_params(5), {
            "workload": "cut_sky", "n_points": 32_000_000, "box": "open", "r_min": 20.0, "r_max": 200.0,
            "nbins": 36, "ell_max": 10, "periodic": False,
            "clustering": "8M Thomas data (w=+1) + 24M uniform randoms (w=-1/3) in an RA 0-60, Dec -30..30 deg, "
                          "r 500-1500 sector"}
    if name == "thomas_4m":
        xyz, w = synth.thomas_4m()
        return xyz, w, synth.config_params(3), {
            "workload": "thomas_4m", "n_points": 4_000_000, "box": 2000.0, "r_min": 10.0, "r_max": 200.0,
            "nbins": 32, "ell_max": 20, "periodic": True, "clustering": "Thomas, 40k parents, sigma 5",
            "weights": "U[0.5,1.5]"}
    if name == "sphere_nside1024":
        xyz, w = synth.sphere_map(1024)
        arcmin = np.pi / (180.0 * 60.0)
        return xyz, w, dict(sphere=True, theta_min=0.0, theta_max=200.0 * arcmin, nbins=20, mmax=8), {
            "workload": "sphere_nside1024", "n_points": int(xyz.shape[0]), "geometry": "unit sphere",
            "theta_arcmin": [0.0, 200.0], "nbins": 20, "m_max": 8,
            "points": "12 * 1024^2 Fibonacci-spiral directions (equal-area, HEALPix-like)",
            "weights": "smooth random field: 64 von Mises blobs (width 0.05 rad) + 0.1 white noise"}
    if name == "mock_batch":
        sizes = synth.mock_sizes()
        cats = [synth.mock_catalogue(i, n) for i, n in enumerate(sizes)]
        return [c[0] for c in cats], [np.ones(c[0].shape[0]) for c in cats], synth.config_params(4), {
            "workload": "mock_batch", "catalogues": len(sizes), "n_points": int(sizes.sum()), "box": 1000.0,
            "r_min": 10.0, "r_max": 150.0, "nbins": 20, "ell_max": 10, "periodic": True,
            "clustering": "Thomas per catalogue, N_i/100 parents, sigma 5", "weights": "unit",
            "mode": "see batch_mode"}
    raise SystemExit(f"unknown workload {name}")


PASS_CAP = 184          # accumulators per pass of the accumulation kernel
SINGLE_PASS_LMAX = 10   # up to here one pass holds every coefficient
FIRST_PASS_M1 = 2       # above it the first (Chebyshev) pass ends at m = 2


def _coefs(L: int, m0: int, m1: int) -> int:
    return sum((L - m + 1) * (1 if m == 0 else 2) for m in range(m0, min(m1, L) + 1))


def _pass_end(L: int, m0: int, cap: int) -> int:
    """End column of the pass starting at m0, as the library splits them:
    one pass up to l_max 10; above, a first pass [0, 2], then columns are
    added while a pass holds at most `cap` coefficients."""
    if L <= SINGLE_PASS_LMAX:
        return L
    if m0 == 0:
        return FIRST_PASS_M1
    s, m = 0, m0
    while m <= L:
        c = (L - m + 1) * (1 if m == 0 else 2)
        if s + c > cap and m > m0:
            break
        s += c
        m += 1
    return m - 1


def _passes(L: int, cap: int):
    out, m0 = [], 0
    while m0 <= L:
        m1 = _pass_end(L, m0, cap)
        out.append((m0, m1))
        m0 = m1 + 1
    return out


def pass_split(L: int):
    """The m-passes of the accumulation kernel for l_max L: the smallest cap
    that keeps the pass count of filling each to PASS_CAP coefficients."""
    target = len(_passes(L, PASS_CAP))
    lo, hi = 1, PASS_CAP
    while lo < hi:
        mid = (lo + hi) // 2
        if len(_passes(L, mid)) <= target:
            hi = mid
        else:
            lo = mid + 1
    return _passes(L, lo)


def _cpow_flops(e: int) -> int:
    """FLOPs of (x + iy)^e by repeated squaring (FMA = 2)."""
    if e == 1:
        return 0
    if e % 2 == 0:
        return _cpow_flops(e // 2) + 5
    return _cpow_flops(e - 1) + 6


def flops_per_pair(lmax: int) -> int:
    """Algorithmic FP32 FLOPs per pair of the accumulation kernel (FMA = 2),
    counted from its formulation: per m-range pass the separation norm and
    direction (8), the pass's basis sequence (Chebyshev: one FMA per degree;
    the first column's monic recurrence: MUL + FMA per degree), the pass's
    first power w (x+iy)^m0 by squaring, one complex multiplication (6) per
    further column, and one FMA per moment (an ADD for degree 0)."""
    L = lmax
    f = 0
    for m0, m1 in pass_split(L):
        f += 8
        K = L - m0
        if K >= 2:
            f += (K - 1) * (2 if m0 == 0 else 3)
        ms = max(m0, 1)
        if m0 == 0:
            f += 1 + 2 * L                                # column 0
        if ms <= min(m1, L):
            f += 2 + _cpow_flops(ms)                      # w (x+iy)^ms
            for m in range(ms, min(m1, L) + 1):
                if m > ms:
                    f += 6
                f += 2 + 4 * (L - m)                      # (+m, -m) moments
    return f


def traffic_per_launch(lmax: int, npairs: int, chunks: int):
    """DRAM bytes of one mean k_alm launch of this run (a chunk runs one
    launch per m-pass), scaled from the captured launches by their pairs (the
    traffic is the list words and the gathers' misses, which grow with the
    pairs), or None when no capture of the current kernel exists."""
    per_pair = K_ALM_DRAM_BYTES_PER_PAIR.get(lmax)
    if per_pair is None or chunks <= 0:
        return None
    return per_pair * npairs / (chunks * len(pass_split(lmax)))


def contraction_roofline(prec, kw, stages_ms, pk, pk_kind, npts, negw):
    """Roofline of the tcgen05 contraction (mixed precisions only).  It reads
    each operand element once, at about 48 FLOP per byte for BF16x3 against a
    machine balance near 290, so it is bound by HBM: the algorithmic bytes
    are the operand tensors (BF16x3: H and 2L, plus sign(w) H when a weight is
    negative, 2 bytes an element; TF32: H, plus sign(w) H, 4 bytes), primaries
    x nbins x (l_max+1)^2 elements each, over the contraction stage's event
    time against the measured copy bandwidth.  The tensor-pipe rate (2 x
    primaries x (l_max+1)^2 x nbins^2 FLOPs, x3 for the BF16 hi/lo split,
    against the measured dense BF16 peak; TF32 x 1.1/2.25) and the pack
    stage's HBM rate (reads the FP32 coefficient, writes the operand
    elements) ride along."""
    if prec == "fp32" or kw.get("sphere") or stages_ms.get("contraction", 0.0) <= 0.0:
        return {}
    nc = ncoef(kw)
    elems = float(npts) * nc * kw["nbins"]
    if prec == "bf16x3":
        op_bytes = elems * 2.0 * (3 if negw else 2)
    else:
        op_bytes = elems * 4.0 * (2 if negw else 1)
    hbm = float(pk.get("hbm_gbs", 6800.0))
    t = stages_ms["contraction"] / 1e3
    achieved = op_bytes / t / 1e9
    flops = 2.0 * npts * nc * kw["nbins"] ** 2 * (3 if prec == "bf16x3" else 1)
    peak_tc = float(pk.get("bf16_tflops", 1900.0)) * (1.0 if prec == "bf16x3" else 1.1 / 2.25)
    out = {"bound": "hbm", "kernel": "k_contract_tc", "achieved": achieved, "peak": hbm, "unit": "GB/s",
           "frac": achieved / hbm, "bytes_per_step": op_bytes,
           "peak_note": f"HBM copy bandwidth ({pk_kind})",
           "tensor_tflops": flops / t / 1e12, "tensor_peak": peak_tc,
           "tensor_frac": flops / t / 1e12 / peak_tc,
           "tensor_peak_note": f"dense BF16 ({pk_kind}, burst)" + (" x 1.1/2.25 for TF32" if prec == "tf32" else "")}
    if stages_ms.get("pack", 0.0) > 0.0:
        pack_bytes = elems * 4.0 + op_bytes
        out["pack"] = {"kernel": "k_pack", "achieved": pack_bytes / (stages_ms["pack"] / 1e3) / 1e9,
                       "bytes_per_step": pack_bytes,
                       "frac": pack_bytes / (stages_ms["pack"] / 1e3) / 1e9 / hbm}
    return {"roofline_contraction": out}


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def sum_over_ranks(world, v: float) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(world, v: float) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)


def ncoef(kw) -> int:
    """Real coefficients per pair: (l_max+1)^2 in 3-D, 2 m_max + 1 on the sphere."""
    return 2 * kw["mmax"] + 1 if kw.get("sphere") else (kw["lmax"] + 1) ** 2


def oracle_zeta(xyz, w, kw, prim):
    import oracle
    if kw.get("sphere"):
        return oracle.zeta_sphere(xyz, w, kw["theta_min"], kw["theta_max"], kw["nbins"], kw["mmax"], prim=prim)
    return oracle.zeta(xyz, w, prim=prim, **kw)


def make_estimator(ctb, kw):
    if kw.get("sphere"):
        return ctb.CTB.sphere(kw["theta_min"], kw["theta_max"], kw["nbins"], kw["mmax"])
    return ctb.CTB(**kw)


def zeta_err(z, ref) -> float:
    """max over (l, b1, b2) of |z - zeta_ref| / sqrt(G_l(b1,b1) G_l(b2,b2)), G the
    same contraction with |w_p| (a Cauchy-Schwarz bound on every entry)."""
    g = np.abs(np.diagonal(ref["gram"], axis1=1, axis2=2))
    s = np.sqrt(g[:, :, None] * g[:, None, :])
    d = np.abs(np.asarray(z) - ref["zeta"])
    return float(np.max(np.where(s > 0, d / np.where(s > 0, s, 1.0), np.where(d > 0, np.inf, 0.0))))


def zeta_err_elementwise(z, ref, floor=1e-3) -> float:
    """Plain relative error over the entries with |zeta_ref| >= floor * max_l |zeta_ref|."""
    zr = ref["zeta"]
    big = (np.abs(zr) >= floor * np.abs(zr).max(axis=(1, 2), keepdims=True)) & (np.abs(zr) > 0)
    d = np.abs(np.asarray(z) - zr)
    return float(np.max(np.where(big, d / np.where(big, np.abs(zr), 1.0), 0.0)))


def zeta_err_normwise(z, ref) -> float:
    """max over l of max |dzeta_l| / max |zeta_ref_l|."""
    zr = ref["zeta"]
    d = np.abs(np.asarray(z) - zr).max(axis=(1, 2))
    m = np.abs(zr).max(axis=(1, 2))
    return float(np.max(np.where(m > 0, d / np.where(m > 0, m, 1.0), np.where(d > 0, np.inf, 0.0))))


def oracle_rate(xyz, w, kw, target_s: float, seed: int = 7, full: bool = False):
    """Time the oracle on a growing sample of primaries until ~target_s of CPU work."""
    import oracle
    from paper_2604_08855_gb300 import synth
    oracle.build()
    nc = ncoef(kw)
    k = 32
    while True:
        prim = synth.sample_primaries(xyz.shape[0], k, seed=seed)
        t0 = time.perf_counter()
        res = oracle_zeta(xyz, w, kw, prim)
        dt = time.perf_counter() - t0
        if dt >= 0.25 * target_s or k >= xyz.shape[0]:
            break
        k = min(xyz.shape[0], int(k * max(2.0, min(16.0, 0.5 * target_s / max(dt, 1e-3)))))
    if full:
        return res["npairs"] * nc / dt, k, dt, res["npairs"], res
    return res["npairs"] * nc / dt, k, dt, res["npairs"]


def run_reference(args):
    world, rank, _ = dist_init(args)
    if rank != 0:
        return
    xyz, w, kw, cfg = workload(args.workload)
    if isinstance(xyz, list):  # a batch: the oracle samples catalogue 0
        xyz, w = xyz[0], w[0]
        cfg = {**cfg, "note": "oracle sample from catalogue 0"}
    import oracle
    oracle.build()
    from paper_2604_08855_gb300 import synth
    nc = ncoef(kw)
    cores = oracle.max_threads()
    # size the per-step sample to about 2 s of CPU work
    rate, k0, _, np0 = oracle_rate(xyz, w, kw, target_s=2.0)
    per_pair = max(1.0, np0 / max(k0, 1))  # pairs per primary of the sample
    k = int(max(8, min(xyz.shape[0], 2.0 * rate / nc / per_pair)))
    times, pairs = [], []
    for step in range(args.warmup + args.steps):
        prim = synth.sample_primaries(xyz.shape[0], k, seed=1000 + step)
        t0 = time.perf_counter()
        res = oracle_zeta(xyz, w, kw, prim)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            pairs.append(res["npairs"])
    total_t = sum(times)
    value = sum(pairs) * nc / total_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{k} seeded primaries per step x all {xyz.shape[0]} secondaries"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm


PREC_OPT = {"fp32": 0, "bf16x3": 1, "tf32": 2}


def run_ours(args):
    world, rank, local = dist_init(args)
    import torch
    from paper_2604_08855_gb300 import build as ctb_build
    if rank == 0 or world == 1:
        ctb_build.build()
    barrier(world)
    from paper_2604_08855_gb300 import ctb
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    xyz, w, kw, cfg = workload(args.workload)
    nc = ncoef(kw)
    sphere = bool(kw.get("sphere"))
    batch = isinstance(xyz, list)  # several catalogues, one ctb_compute_batch per step
    negw = bool(any(np.any(v < 0) for v in w)) if batch else bool(np.any(w < 0))
    # precisions timed in this run: "mixed" = plain FP32, then the BF16 hi/lo
    # tensor-core contraction (the line's headline), then a short TF32 extra
    if args.precision == "mixed":
        modes = ["fp32"] if sphere else ["fp32", "bf16x3"]
    else:
        modes = [args.precision]
    headline = modes[-1]
    est = make_estimator(ctb, kw)
    stream = torch.cuda.current_stream(dev)
    est.set_stream(stream)
    if args.cells_per_rmax:
        est.set_option(ctb.OPT_CELLS_PER_RMAX, args.cells_per_rmax)
    else:
        # tuned on the first set_points or batch (a warm-up step); a batch
        # tunes on its largest catalogue
        est.set_option(ctb.OPT_AUTOTUNE, 1)
    if batch:
        d_cats = [(torch.from_numpy(x).to(dev), torch.from_numpy(v).to(dev)) for x, v in zip(xyz, w)]
        d_zeta = torch.zeros((len(xyz),) + est.zeta_shape, dtype=torch.float64, device=dev)
    else:
        d_xyz = torch.from_numpy(xyz).to(dev)
        d_w = torch.from_numpy(w).to(dev)
        d_zeta = torch.zeros(est.zeta_shape, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    d_prim = None
    if args.primaries and not batch:
        # profiling case: the same catalogue and kernels, fewer primaries
        from paper_2604_08855_gb300 import synth
        d_prim = torch.from_numpy(synth.sample_primaries(xyz.shape[0], args.primaries, seed=7)).to(dev)
        cfg = {**cfg, "primaries": args.primaries, "note": "primary subset (profiling case)"}
    elif world > 1 and not batch:
        # several GPUs: each rank takes its shard of one catalogue's primaries
        # (every point stays a secondary) and one FP64 all-reduce sums zeta
        from paper_2604_08855_gb300 import shard
        d_prim = torch.from_numpy(shard.shard_primaries(xyz.shape[0], rank, world)).to(dev)

    seq = batch and args.batch_mode == "sequential"
    seq_stats = {}
    shared_h = args.shared if args.shared >= 0 and not batch and not args.primaries else None

    def step():
        if seq:
            # the same catalogues as plain launches, one set_points + compute each
            tm, launches_, pairs_, chunks_ = np.zeros(9), 0, 0, 0
            for i, (x, v) in enumerate(d_cats):
                est.set_points(x, v)
                est.compute(out=d_zeta[i])
                tm += np.array(est.timings())
                launches_ += est.launch_count()
                pairs_ += est.pair_count()
                chunks_ += est.chunk_count()
            seq_stats.update(timings=list(tm), launches=launches_, pairs=pairs_, chunks=chunks_)
            return
        if batch:
            est.compute_batch(d_cats, out=d_zeta)
            return
        est.set_points(d_xyz, d_w)
        if shared_h is not None:
            est.compute_shared(shared_h, out=d_zeta)
        elif d_prim is None:
            est.compute(out=d_zeta)
        else:
            est.compute_subset(d_prim, out=d_zeta)
            if world > 1 and not args.primaries:
                import torch.distributed as dist
                dist.all_reduce(d_zeta, op=dist.ReduceOp.SUM)

    def stats():
        if seq:
            return seq_stats["timings"], seq_stats["launches"], seq_stats["pairs"], seq_stats["chunks"]
        return est.timings(), est.launch_count(), est.pair_count(), est.chunk_count()

    def time_mode(prec, steps, warmup):
        est.set_option(ctb.OPT_PRECISION, PREC_OPT[prec])
        for _ in range(warmup):
            flush.zero_()
            step()
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        launches, stages = 0, []
        barrier(world)
        torch.cuda.synchronize(dev)
        wall0 = time.perf_counter()
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            tm, ln, npairs, chunks = stats()
            launches += ln
            stages.append(tm)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - wall0
        barrier(world)
        step_ms = [a.elapsed_time(b) for a, b in ev]
        t_total = max_over_ranks(world, sum(step_ms) / 1e3)
        npairs_all = int(sum_over_ranks(world, float(npairs))) if world > 1 and d_prim is not None \
            and not args.primaries else npairs
        return {"t_total": t_total, "stages": np.mean(np.array(stages), axis=0), "launches": launches,
                "npairs": npairs, "npairs_all": npairs_all, "chunks": chunks, "wall": wall,
                "pair_ms": float(np.mean([s[7] for s in stages]))}

    shared_info = None
    if shared_h is not None:
        est.set_option(ctb.OPT_PRECISION, PREC_OPT[headline])
        for _ in range(args.warmup):
            flush.zero_()
            step()
        # the exact estimator on the same catalogue, once, for the speed and the deviation
        est.set_points(d_xyz, d_w)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        flush.zero_()
        t0.record(stream)
        z_exact = est.compute()
        t1.record(stream)
        torch.cuda.synchronize(dev)
        exact_ms, exact_pairs = t0.elapsed_time(t1), est.pair_count()
        z_sh = est.compute_shared(shared_h)
        h_used, n_groups_sh = est.pivot_groups()
        if np.all(w > 0):
            # positive weights: zeta itself is the Gram matrix of the tests' metric
            diag = np.abs(np.einsum("lii->li", z_exact))
            scale = np.sqrt(diag[:, :, None] * diag[:, None, :])
            dev_metric = "max |zeta_shared - zeta_exact| / sqrt(zeta(b1,b1) zeta(b2,b2))"
        else:
            scale = np.broadcast_to(np.abs(z_exact).max(axis=(1, 2), keepdims=True), z_exact.shape)
            dev_metric = "max over l of max |zeta_shared - zeta_exact| / max |zeta_exact|"
        shared_info = {"pivot_cell": h_used, "groups": n_groups_sh, "points": int(xyz.shape[0]),
                       "exact_pairs": exact_pairs, "exact_ms": exact_ms,
                       "max_dev_vs_exact": float(np.max(np.abs(z_sh - z_exact) / np.where(scale > 0, scale, 1.0))),
                       "dev_metric": dev_metric + ", against the exact path on the GPU"}
        torch.cuda.synchronize(dev)

    with ClockSampler(local) as clk:
        res = {}
        for prec in modes:
            res[prec] = time_mode(prec, args.steps, args.warmup)
        clocks = clk.summary()
    extra_tf32 = None
    if args.precision == "mixed" and not sphere and not batch and shared_h is None and args.tf32_steps > 0:
        extra_tf32 = time_mode("tf32", args.tf32_steps, 1)
    est.set_option(ctb.OPT_PRECISION, PREC_OPT[headline])

    pk, pk_kind = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    # FP32 lane-instruction peak (one FMA-pipe instruction per lane per clock)
    peak_tinst = SM_COUNT * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    n_groups = (kw["mmax"] if sphere else kw["lmax"]) + 1
    names = ["ingest", "sort_grid", "pair_total", "pack", "contraction", "reduce", "enumerate", "accumulate",
             "group"]

    def summarise(prec, r):
        updates = r["npairs_all"] * nc
        value = args.steps_of(prec) * updates / r["t_total"]
        ms = 1e3 * r["t_total"] / args.steps_of(prec)
        pair_s = r["pair_ms"] / 1e3
        if sphere:
            inst_pair = 4 * kw["mmax"] + 11
            achieved = r["npairs"] * inst_pair / pair_s / 1e12
            roof = {"kernel": "k_am", "work_per_unit": f"{inst_pair} FP32 instructions per pair (4 m_max + 11)"}
        else:
            # algorithmic work of the accumulation: INST_PER_UPDATE FP32 instructions
            # per (pair, coefficient) update, over the kernel's own event time
            achieved = r["npairs"] * nc * INST_PER_UPDATE / pair_s / 1e12
            impl_tflops = r["npairs"] * flops_per_pair(kw["lmax"]) / pair_s / 1e12
            roof = {"kernel": "k_alm", "work_per_unit": f"{INST_PER_UPDATE} FP32 instructions per update",
                    "traffic": traffic_per_launch(kw["lmax"], r["npairs"], r["chunks"]),
                    "impl_flops_per_pair": flops_per_pair(kw["lmax"]), "impl_tflops": impl_tflops,
                    "impl_frac": impl_tflops / (2 * peak_tinst)}
        stages_ms = {k: round(float(v), 3) for k, v in zip(names, r["stages"])}
        out = {
            "value": value, "ms_per_step": ms, "ms_per_zeta_ell": ms / n_groups,
            "pairs_per_step": r["npairs_all"], "pairs_per_s": args.steps_of(prec) * r["npairs_all"] / r["t_total"],
            "stages_ms": stages_ms, "gpu_launches": r["launches"],
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tinst, "unit": "Tinst/s",
                         "frac": achieved / peak_tinst, "traffic": None, **roof,
                         "launches_per_step": r["chunks"] * (1 if sphere else len(pass_split(kw["lmax"]))),
                         "peak_note": f"FP32 pipe: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x "
                                      f"{sm_max:.0f} MHz ({pk_kind} max clock), burst",
                         "kernel_ms": 1e3 * pair_s},
        }
        n_prim_step = (sum(a.shape[0] for a in xyz) if batch else xyz.shape[0]) if not args.primaries \
            else args.primaries
        if world > 1 and d_prim is not None and not args.primaries:
            n_prim_step = int(d_prim.shape[0])
        out.update(contraction_roofline(prec, kw, stages_ms, pk, pk_kind, npts=n_prim_step, negw=negw))
        return out

    args.steps_of = lambda prec: args.steps
    head = summarise(headline, res[headline])
    # end to end through the public API with host buffers (the headline precision)
    zh = np.zeros(tuple(d_zeta.shape))
    e2e_t = []
    for k in range(0 if args.no_e2e else max(2, min(args.steps, 5)) + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        if seq:
            for i, (x, v) in enumerate(zip(xyz, w)):
                est.set_points(x, v)
                est.compute(out=zh[i])
        elif batch:
            est.compute_batch(list(zip(xyz, w)), out=zh)
        else:
            est.set_points(xyz, w)
            if shared_h is not None:
                est.compute_shared(shared_h, out=zh)
            elif d_prim is None:
                est.compute(out=zh)
            else:
                est.compute_subset(d_prim.cpu().numpy(), out=zh)
                if world > 1 and not args.primaries:
                    from paper_2604_08855_gb300 import shard
                    zh[...] = shard.allreduce_zeta(zh)
        dt = time.perf_counter() - t0
        if k > 0:
            e2e_t.append(dt)
    e2e_s = max_over_ranks(world, float(np.mean(e2e_t)) if e2e_t else float("nan"))
    in_bytes = sum(a.nbytes for a in xyz) + sum(a.nbytes for a in w) if batch else xyz.nbytes + w.nbytes
    e2e = {"value": res[headline]["npairs_all"] * nc / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(in_bytes), "d2h_bytes_per_step": int(zh.nbytes + 8)}

    dtype = {"fp32": "f32", "bf16x3": "f32+bf16x3", "tf32": "f32+tf32"}[headline]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "strong" if (world > 1 and d_prim is not None and not args.primaries) else "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {**cfg, "precision": headline,
                   "precision_note": {"fp32": "FP32 pair kernel and contraction, FP64 reduce",
                                      "bf16x3": "FP32 pair kernel, BF16 hi/lo x3 tcgen05 contraction with FP32 "
                                                "accumulate, FP64 reduce",
                                      "tf32": "FP32 pair kernel, TF32 tcgen05 contraction with FP32 accumulate, "
                                              "FP64 reduce"}[headline],
                   **({"batch_mode": args.batch_mode} if batch else {}),
                   "cells_per_rmax": est.grid()[0],
                   "grid": "fixed" if args.cells_per_rmax else "autotuned",
                   "l2": "flushed (256 MB write) before every step",
                   "inputs": "device-resident float64 xyz, w",
                   **({"parallelism": f"primaries sharded over {world} GPUs, one FP64 all-reduce of zeta"}
                      if world > 1 and d_prim is not None and not args.primaries else {})},
        "e2e": e2e,
        "gpu_launches": head["gpu_launches"],
        "roofline": head["roofline"],
        **({"roofline_contraction": head["roofline_contraction"]} if "roofline_contraction" in head else {}),
        "stages_ms": head["stages_ms"],
        "pairs_per_step": head["pairs_per_step"],
        "pairs_per_s": head["pairs_per_s"],
        "ms_per_zeta_ell": head["ms_per_zeta_ell"],
        "wall_s": res[headline]["wall"],
        "clocks": clocks,
    }
    if len(modes) > 1:
        plain = summarise("fp32", res["fp32"])
        line["plain_fp32"] = {k: plain[k] for k in ("value", "ms_per_step", "ms_per_zeta_ell", "stages_ms",
                                                    "gpu_launches", "roofline")}
        line["plain_fp32"]["dtype"] = "f32"
        line["mixed_over_plain"] = head["value"] / plain["value"]
        line["mixed_over_plain_contraction"] = (
            (plain["stages_ms"]["contraction"] + plain["stages_ms"]["pack"])
            / max(head["stages_ms"]["contraction"] + head["stages_ms"]["pack"], 1e-9))
    if extra_tf32 is not None:
        args.steps_of = lambda prec: args.tf32_steps
        t = summarise("tf32", extra_tf32)
        line["tf32"] = {"value": t["value"], "ms_per_step": t["ms_per_step"], "stages_ms": t["stages_ms"],
                        "steps": args.tf32_steps, "warmup": 1, "dtype": "f32+tf32",
                        **({"roofline_contraction": t["roofline_contraction"]} if "roofline_contraction" in t else {})}
    if shared_info is not None:
        shared_info["speedup_vs_exact"] = shared_info["exact_ms"] / head["ms_per_step"]
        line["config"]["estimator"] = "shared neighbour lists for close pivots (approximate)"
        line["shared"] = shared_info
    if rank == 0 and not args.no_cpu_baseline:
        sx, sw = (xyz[0], w[0]) if batch else (xyz, w)
        rate, k, dt, _, ref = oracle_rate(sx, sw, kw, target_s=args.cpu_seconds, full=True)
        import oracle
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                                "sample": f"{k} seeded primaries x all {sx.shape[0]} secondaries"
                                          + (" of catalogue 0" if batch else "") + f", {dt:.1f} s"}
        # the same primaries through the library, against the oracle, in every precision timed
        from paper_2604_08855_gb300 import synth
        prim = synth.sample_primaries(sx.shape[0], k, seed=7)
        est.set_points(sx, sw)
        par = {"metric": "max |dzeta| / sqrt(G(b1,b1) G(b2,b2)), G the |w_p| Gram",
               "secondary": "elementwise: max |dzeta|/|zeta| over |zeta| >= 1e-3 max_l |zeta|; "
                            "normwise: max over l of max |dzeta_l| / max |zeta_l|",
               "sample": f"the cpu_baseline's {k} primaries"}
        for prec in modes + (["tf32"] if extra_tf32 is not None else []):
            est.set_option(ctb.OPT_PRECISION, PREC_OPT[prec])
            z = est.compute_subset(prim)
            par[prec] = {"value": zeta_err(z, ref), "tolerance": 1e-5 if prec == "fp32" else 1e-3,
                         "elementwise": zeta_err_elementwise(z, ref), "normwise": zeta_err_normwise(z, ref),
                         "pairs_match": est.pair_count() == ref["npairs"]}
        par["value"] = par[headline]["value"]
        par["tolerance"] = par[headline]["tolerance"]
        par["pairs_match"] = all(par[p]["pairs_match"] for p in modes)
        line["parity"] = par
    if rank == 0:
        print(json.dumps(line), flush=True)
    est.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32", "bf16x3", "tf32"],
                    help="mixed (default): time plain FP32, then the BF16 hi/lo tensor-core contraction (the "
                         "line's value), then a short TF32 extra; or one precision alone")
    ap.add_argument("--tf32-steps", type=int, default=2, help="timed steps of the TF32 extra (0: skip)")
    ap.add_argument("--workload", default="thomas_4m")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--primaries", type=int, default=0,
                    help="profiling case: time ctb_compute_subset over this many seeded primaries")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-mode", default="batched", choices=["batched", "sequential"],
                    help="mock_batch: one ctb_compute_batch per step, or one set_points + compute per catalogue")
    ap.add_argument("--shared", type=float, default=-1.0,
                    help="time ctb_compute_shared (shared neighbour lists for close pivots) with this pivot "
                         "cell side; 0 = the mean separation; negative = off (the exact estimator)")
    ap.add_argument("--cells-per-rmax", type=int, default=0,
                    help="grid cells per r_max (0: the library's autotuner picks)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
