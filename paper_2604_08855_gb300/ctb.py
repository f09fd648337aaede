"""Thin ctypes binding to libctb (include/ctb.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module converts
numpy arrays / torch tensors to pointers and status codes to exceptions.  It
raises ImportError when the library has not been built: there is no CPU
fallback.

    from paper_2604_08855_gb300.ctb import CTB
    est = CTB(box=1000.0, rmin=5.0, rmax=200.0, nbins=20, lmax=10)
    est.set_points(xyz, w)            # numpy (host) or torch CUDA tensors
    zeta = est.compute()              # numpy float64 [(lmax+1), nbins, nbins]
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libctb.so")

OK = 0
ERR_ARG, ERR_NONFINITE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_STATE, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6, -7
OPT_PRECISION, OPT_CELLS_PER_RMAX, OPT_LIST_CAPACITY, OPT_WARPS_PER_BLOCK, OPT_CHUNK_PRIMARIES, \
    OPT_DETERMINISTIC, OPT_AUTOTUNE, OPT_FAULT_INJECT = 1, 2, 3, 4, 5, 6, 7, 8
INJECT_STALL, INJECT_ALLOC = 1, 2
PREC_FP32, PREC_BF16X3, PREC_TF32 = 0, 1, 2
LMAX_CAP, NBINS_CAP, MMAX_CAP = 20, 64, 16

# every symbol include/ctb.h declares
EXPORTS = ("ctb_create", "ctb_create_sphere", "ctb_set_points", "ctb_compute", "ctb_compute_subset",
           "ctb_compute_shared", "ctb_get_pivot_groups", "ctb_get_alm",
           "ctb_compute_batch", "ctb_set_option", "ctb_set_stream", "ctb_set_allocator",
           "ctb_get_timings", "ctb_get_pair_count", "ctb_get_chunk_count", "ctb_get_grid",
           "ctb_get_2pcf", "ctb_edge_correct", "ctb_get_launch_count", "ctb_contract_noalloc", "ctb_destroy", "ctb_last_error", "ctb_version")

_lib = None


class CTBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def load(path: str | None = None):
    """Load libctb.so (ImportError if it is missing; build it with build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libctb.so not built at {path}: run paper_2604_08855_gb300.build")
    lib = ctypes.CDLL(path)
    vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.ctb_create.argtypes = [d, d, d, i32, i32]
    lib.ctb_create_sphere.argtypes = [d, d, i32, i32]
    lib.ctb_create_sphere.restype = vp
    lib.ctb_create.restype = vp
    lib.ctb_set_points.argtypes = [vp, vp, vp, i64]
    lib.ctb_compute.argtypes = [vp, vp]
    lib.ctb_compute_subset.argtypes = [vp, vp, i64, vp]
    lib.ctb_get_alm.argtypes = [vp, vp, i64, vp]
    lib.ctb_compute_shared.argtypes = [vp, d, vp]
    lib.ctb_get_pivot_groups.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(i64)]
    lib.ctb_compute_batch.argtypes = [vp, vp, vp, vp, i32, vp]
    lib.ctb_set_option.argtypes = [vp, i32, i64]
    lib.ctb_set_stream.argtypes = [vp, vp]
    lib.ctb_set_allocator.argtypes = [vp, vp, vp, vp]
    lib.ctb_get_timings.argtypes = [vp, vp, i32]
    lib.ctb_get_pair_count.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.ctb_get_chunk_count.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.ctb_get_grid.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.ctb_get_2pcf.argtypes = [vp, vp, i32]
    lib.ctb_edge_correct.argtypes = [vp, vp, vp, vp]
    lib.ctb_get_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.ctb_contract_noalloc.argtypes = [vp, vp, i64, i32, i32, vp, vp]
    lib.ctb_destroy.argtypes = [vp]
    lib.ctb_destroy.restype = None
    lib.ctb_last_error.argtypes = [vp]
    lib.ctb_last_error.restype = ctypes.c_char_p
    lib.ctb_version.argtypes = []
    lib.ctb_version.restype = ctypes.c_char_p
    for name in ("ctb_set_points", "ctb_compute", "ctb_compute_subset", "ctb_compute_shared",
                 "ctb_get_pivot_groups", "ctb_get_alm", "ctb_compute_batch",
                 "ctb_set_option", "ctb_set_stream", "ctb_set_allocator", "ctb_get_timings",
                 "ctb_get_pair_count", "ctb_get_chunk_count", "ctb_get_grid", "ctb_get_2pcf",
                 "ctb_edge_correct", "ctb_get_launch_count", "ctb_contract_noalloc"):
        getattr(lib, name).restype = i32
    _lib = lib
    return lib


def _ptr(x):
    """Pointer of a numpy array or torch tensor (host or CUDA), or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return x.ctypes.data_as(ctypes.c_void_p)


def _as_f64(x, shape_tail=None):
    if x is None or hasattr(x, "data_ptr"):
        if x is not None:
            import torch
            if x.dtype != torch.float64 or not x.is_contiguous():
                raise TypeError("torch inputs must be contiguous float64")
        return x
    return np.ascontiguousarray(x, dtype=np.float64)


class CTB:
    """One estimator configuration on the current CUDA device.

    CTB(box, rmin, rmax, nbins, lmax): 3-D Legendre multipoles (box <= 0: open).
    CTB.sphere(theta_min, theta_max, nbins, mmax): projected multipoles on the
    unit sphere (ctb_create_sphere); ``lmax`` then holds m_max.
    """

    def __init__(self, box: float, rmin: float, rmax: float, nbins: int, lmax: int, _sphere: bool = False):
        self.lib = load()
        self.box, self.rmin, self.rmax, self.nbins, self.lmax = float(box), float(rmin), float(rmax), int(nbins), int(lmax)
        self.is_sphere = bool(_sphere)
        if self.is_sphere:
            h = self.lib.ctb_create_sphere(self.rmin, self.rmax, self.nbins, self.lmax)
        else:
            h = self.lib.ctb_create(self.box, self.rmin, self.rmax, self.nbins, self.lmax)
        if not h:
            raise CTBError(ERR_ARG, self.lib.ctb_last_error(None).decode())
        self._h = ctypes.c_void_p(h)
        self.n = None
        self._keep = []

    @classmethod
    def sphere(cls, theta_min: float, theta_max: float, nbins: int, mmax: int):
        """Projected multipoles zeta_m, m = 0..mmax, of directions on the unit
        sphere, bins linear in the angle [theta_min, theta_max) (radians)."""
        return cls(0.0, theta_min, theta_max, nbins, mmax, _sphere=True)

    @property
    def ncoef(self) -> int:
        """Coefficients per (primary, bin) of get_alm."""
        return 2 * self.lmax + 1 if self.is_sphere else (self.lmax + 1) ** 2

    def close(self):
        if getattr(self, "_h", None):
            self.lib.ctb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc):
        if rc < 0:
            raise CTBError(rc, self.lib.ctb_last_error(self._h).decode())
        return rc

    @property
    def zeta_shape(self):
        return (self.lmax + 1, self.nbins, self.nbins)

    def set_option(self, key: int, value: int):
        self._check(self.lib.ctb_set_option(self._h, int(key), int(value)))

    def set_stream(self, stream):
        """stream: torch.cuda.Stream, an integer cudaStream_t, or None."""
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self._check(self.lib.ctb_set_stream(self._h, ctypes.c_void_p(stream or 0)))

    def use_torch_allocator(self, device=None):
        """Route device allocations through torch's caching allocator."""
        import torch
        dev = torch.cuda.current_device() if device is None else int(device)
        AF = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
        FF = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

        def _alloc(nbytes, _user):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev)
            except Exception:
                return None

        def _free(ptr, _user):
            torch.cuda.caching_allocator_delete(ptr)

        af, ff = AF(_alloc), FF(_free)
        self._keep = [af, ff]
        self._check(self.lib.ctb_set_allocator(self._h, ctypes.cast(af, ctypes.c_void_p),
                                               ctypes.cast(ff, ctypes.c_void_p), None))

    def set_points(self, xyz, w=None):
        xyz = _as_f64(xyz)
        w = _as_f64(w)
        n = int(xyz.shape[0])
        if tuple(xyz.shape[1:]) != (3,):
            raise ValueError("xyz must be (n, 3)")
        if w is not None and tuple(w.shape) != (n,):
            raise ValueError("w must be (n,)")
        self._check(self.lib.ctb_set_points(self._h, _ptr(xyz), _ptr(w), n))
        self.n = n

    def _out(self, out, shape, dtype):
        if out is None:
            return np.zeros(shape, dtype=dtype)
        return out

    def compute(self, out=None):
        z = self._out(out, self.zeta_shape, np.float64)
        self._check(self.lib.ctb_compute(self._h, _ptr(z)))
        return z

    def compute_subset(self, primaries, out=None):
        p = primaries if hasattr(primaries, "data_ptr") else np.ascontiguousarray(primaries, dtype=np.int64)
        z = self._out(out, self.zeta_shape, np.float64)
        self._check(self.lib.ctb_compute_subset(self._h, _ptr(p), int(p.shape[0]), _ptr(z)))
        return z

    def compute_shared(self, pivot_cell=0.0, out=None):
        """Shared neighbour lists for close pivots: the approximation of zeta in
        which every point takes the neighbour list of its pivot cell's
        representative (include/ctb.h states it and its error bound).
        pivot_cell: the cell side h, 0 for the mean separation."""
        z = self._out(out, self.zeta_shape, np.float64)
        self._check(self.lib.ctb_compute_shared(self._h, float(pivot_cell), _ptr(z)))
        return z

    def pivot_groups(self):
        """(h, groups) of the last compute_shared."""
        h = ctypes.c_double(0.0)
        g = ctypes.c_int64(0)
        self._check(self.lib.ctb_get_pivot_groups(self._h, ctypes.byref(h), ctypes.byref(g)))
        return float(h.value), int(g.value)

    def get_alm(self, primaries, out=None):
        p = primaries if hasattr(primaries, "data_ptr") else np.ascontiguousarray(primaries, dtype=np.int64)
        a = self._out(out, (int(p.shape[0]), self.nbins, self.ncoef), np.float32)
        self._check(self.lib.ctb_get_alm(self._h, _ptr(p), int(p.shape[0]), _ptr(a)))
        return a

    def compute_batch(self, cats, out=None):
        """cats: list of (xyz, w) pairs (numpy or torch); returns [k, lmax+1, nbins, nbins]."""
        k = len(cats)
        xs = [_as_f64(c[0]) for c in cats]
        ws = [_as_f64(c[1]) if len(c) > 1 else None for c in cats]
        xp = (ctypes.c_void_p * k)(*[_ptr(x).value for x in xs])
        wp = (ctypes.c_void_p * k)(*[(_ptr(w).value if w is not None else None) for w in ws])
        ns = np.ascontiguousarray([x.shape[0] for x in xs], dtype=np.int64)
        z = self._out(out, (k,) + self.zeta_shape, np.float64)
        self._check(self.lib.ctb_compute_batch(self._h, ctypes.cast(xp, ctypes.c_void_p),
                                               ctypes.cast(wp, ctypes.c_void_p), _ptr(ns), k, _ptr(z)))
        return z

    def timings(self):
        """ms per stage: ingest, sort+grid, pair, pack, contraction, reduce, enumeration, accumulation,
        pivot grouping."""
        buf = (ctypes.c_double * 9)()
        k = self._check(self.lib.ctb_get_timings(self._h, ctypes.cast(buf, ctypes.c_void_p), 9))
        return list(buf)[:k]

    def launch_count(self) -> int:
        """Kernels launched by the last set_points plus the last compute."""
        v = ctypes.c_uint64(0)
        self._check(self.lib.ctb_get_launch_count(self._h, ctypes.byref(v)))
        return int(v.value)

    def pair_count(self) -> int:
        v = ctypes.c_uint64(0)
        self._check(self.lib.ctb_get_pair_count(self._h, ctypes.byref(v)))
        return int(v.value)

    def edge_correct(self, zeta_nnn, zeta_rrr, out=None):
        """Edge-corrected Legendre coefficients from a data-minus-randoms zeta
        and the randoms' zeta (numpy or torch, host or device)."""
        zn, zr = _as_f64(zeta_nnn), _as_f64(zeta_rrr)
        for z in (zn, zr):
            if tuple(z.shape) != self.zeta_shape:
                raise CTBError(ERR_ARG, f"zeta shape {tuple(z.shape)} != {self.zeta_shape}")
        o = self._out(out, self.zeta_shape, np.float64)
        self._check(self.lib.ctb_edge_correct(self._h, _ptr(zn), _ptr(zr), _ptr(o)))
        return o

    def pair_sums(self, catalogues: int = 1) -> np.ndarray:
        """Weighted pair sums sum_p w_p sum_{j in b} w_j of the last compute
        ([nbins]), or of each catalogue of the last batch ([k, nbins])."""
        out = np.zeros((catalogues, self.nbins), dtype=np.float64)
        r = self.lib.ctb_get_2pcf(self._h, out.ctypes.data_as(ctypes.c_void_p), out.size)
        if r < 0:
            self._check(r)
        if r != out.size:
            raise CTBError(ERR_ARG, f"{r // self.nbins} catalogues hold pair sums, asked for {catalogues}")
        return out[0] if catalogues == 1 else out

    def grid(self) -> tuple[int, int]:
        """(cells per r_max, cells per axis) of the current catalogue's grid."""
        k, nc = ctypes.c_int32(0), ctypes.c_int32(0)
        self._check(self.lib.ctb_get_grid(self._h, ctypes.byref(k), ctypes.byref(nc)))
        return int(k.value), int(nc.value)

    def chunk_count(self) -> int:
        """Primary chunks (launches of each pair kernel) of the last compute."""
        v = ctypes.c_uint64(0)
        self._check(self.lib.ctb_get_chunk_count(self._h, ctypes.byref(v)))
        return int(v.value)


def contract_noalloc(alm, w, nbins: int, lmax: int, out, stream=None) -> None:
    """zeta from device a_lm rows [np][nbins][(lmax+1)^2] and device weights [np]
    (float32 CUDA tensors) into `out` (float64 CUDA tensor [(lmax+1), nbins,
    nbins]), with no device allocation by the library; see
    ctb_contract_noalloc in include/ctb.h.  `stream` defaults to torch's
    current stream on the tensors' device."""
    import torch
    lib = load()
    nc = (int(lmax) + 1) ** 2
    checks = (
        (all(isinstance(t, torch.Tensor) and t.is_cuda for t in (alm, w, out)), "alm, w and out must be CUDA tensors"),
        (alm.device == w.device == out.device, "alm, w and out must be on one device"),
        (alm.dtype == torch.float32 and w.dtype == torch.float32, "alm and w must be float32"),
        (out.dtype == torch.float64, "out must be float64"),
        (alm.is_contiguous() and w.is_contiguous() and out.is_contiguous(), "alm, w and out must be contiguous"),
        (alm.dim() == 3 and tuple(alm.shape[1:]) == (int(nbins), nc), f"alm must be [np][{nbins}][{nc}]"),
        (w.dim() == 1 and w.shape[0] == alm.shape[0], "w needs one weight per primary"),
        (tuple(out.shape) == (int(lmax) + 1, int(nbins), int(nbins)), f"out must be [{lmax + 1}][{nbins}][{nbins}]"),
    ) if isinstance(alm, torch.Tensor) else ((False, "alm, w and out must be CUDA tensors"),)
    for ok, msg in checks:
        if not ok:
            raise ValueError(msg)
    if stream is None:
        stream = torch.cuda.current_stream(alm.device)
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    np_ = int(alm.shape[0])
    rc = lib.ctb_contract_noalloc(_ptr(alm), _ptr(w), np_, int(nbins), int(lmax), _ptr(out),
                                  ctypes.c_void_p(stream or 0))
    if rc < 0:
        raise CTBError(rc, "ctb_contract_noalloc failed")


def version() -> str:
    return load().ctb_version().decode()
