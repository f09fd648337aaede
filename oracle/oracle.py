"""ctypes wrapper around ``ctb_oracle.c`` (FP64 brute force; test infrastructure).

The shared object is compiled with the host gcc into ``oracle/_build`` on first
use (or by ``__graft_entry__.build()``).  No function here touches a GPU.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ctb_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "ctb_oracle_sphere.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libctb_oracle.so")
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, IEEE arithmetic)."""
    with _lock:
        if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(s) for s in _SRCS):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                   "-fno-fast-math", "-ffp-contract=off", "-o", tmp, *_SRCS, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        vp = ctypes.c_void_p
        lib.oracle_ylm.argtypes = [i32, d, d, d, vp]
        lib.oracle_ylm.restype = None
        lib.oracle_alm.argtypes = [vp, vp, i64, d, d, d, i32, i32, vp, i64, vp, vp, i32]
        lib.oracle_alm.restype = i32
        lib.oracle_zeta.argtypes = [vp, vp, i64, d, d, d, i32, i32, vp, i64,
                                    vp, vp, vp, vp, vp, vp, d, i32, vp]
        lib.oracle_zeta.restype = i32
        lib.oracle_zeta_sphere.argtypes = [vp, vp, i64, d, d, i32, i32, vp, i64, vp, vp, vp, vp, i32, vp]
        lib.oracle_zeta_sphere.restype = i32
        lib.oracle_ambiguous.argtypes = [vp, i64, d, d, d, i32, vp, i64, d, vp, vp, i64]
        lib.oracle_ambiguous.restype = i64
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = i32
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _points(xyz, w):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    if xyz.ndim != 2 or xyz.shape[1] != 3:
        raise ValueError("xyz must be (n, 3)")
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float64)
        if w.shape != (xyz.shape[0],):
            raise ValueError("w must be (n,)")
    return xyz, w


def _prim(prim):
    if prim is None:
        return None
    return np.ascontiguousarray(prim, dtype=np.int64)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def ylm(lmax: int, dirs) -> np.ndarray:
    """Real orthonormal Y_lm, index l*l + l + m, at each unit direction."""
    lib = _load()
    dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
    nc = (lmax + 1) ** 2
    out = np.zeros((dirs.shape[0], nc))
    row = np.zeros(nc)
    for i, (x, y, z) in enumerate(dirs):
        lib.oracle_ylm(lmax, float(x), float(y), float(z), _ptr(row))
        out[i] = row
    return out


def alm(xyz, w, box, rmin, rmax, nbins, lmax, prim=None, nthreads=0):
    """a_lm(p, b) for the given primaries: array [np][nbins][(lmax+1)^2]."""
    lib = _load()
    xyz, w = _points(xyz, w)
    prim = _prim(prim)
    n = xyz.shape[0]
    np_ = n if prim is None else prim.shape[0]
    nc = (lmax + 1) ** 2
    out = np.zeros((np_, nbins, nc))
    npairs = ctypes.c_int64(0)
    rc = lib.oracle_alm(_ptr(xyz), _ptr(w), n, float(box), float(rmin), float(rmax),
                        int(nbins), int(lmax), _ptr(prim), np_, _ptr(out),
                        ctypes.byref(npairs), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_alm rejected its arguments (rc={rc})")
    return out


def ambiguous(xyz, box, rmin, rmax, nbins, amb_tol, prim=None, cap=4096):
    """Pairs (i, j) -- i the index into ``prim`` (or the primary itself) --
    whose separation lies within amb_tol * r of a bin edge rmin + k D
    (k = 0..nbins), where a binning that is not exact in FP64 may disagree
    with this oracle's.  Returns (idx [m][2] int64, d [m][3], r [m],
    edge [m] int); raises if more than ``cap`` pairs qualify."""
    lib = _load()
    xyz, _ = _points(xyz, None)
    prim = _prim(prim)
    n = xyz.shape[0]
    np_ = n if prim is None else prim.shape[0]
    ri = np.zeros((cap, 2), dtype=np.int64)
    rd = np.zeros((cap, 5))
    m = lib.oracle_ambiguous(_ptr(xyz), n, float(box), float(rmin), float(rmax), int(nbins), _ptr(prim), np_,
                             float(amb_tol), _ptr(ri), _ptr(rd), cap)
    if m < 0:
        raise ValueError("oracle_ambiguous rejected its arguments")
    if m > cap:
        raise ValueError(f"{m} ambiguous pairs, more than cap = {cap}")
    return ri[:m], rd[:m, :3], rd[:m, 3], rd[:m, 4].astype(int)


def contract(alm_rows, wprim, lmax):
    """zeta_l(b1, b2) = 4 pi / (2l+1) sum_p w_p sum_{m=-l..l} a_lm(p, b1) a_lm(p, b2)
    from given a_lm rows [np][nbins][(lmax+1)^2] (index l*l + l + m) and
    primary weights [np], in float64: the contraction step of the estimator
    definition alone (the same formula ``zeta`` applies to its own a_lm)."""
    a = np.asarray(alm_rows, dtype=np.float64)
    wp = np.asarray(wprim, dtype=np.float64)
    if a.ndim != 3 or a.shape[2] != (lmax + 1) ** 2 or wp.shape != (a.shape[0],):
        raise ValueError("alm_rows must be [np][nbins][(lmax+1)^2] and wprim [np]")
    nb = a.shape[1]
    z = np.zeros((lmax + 1, nb, nb))
    for l in range(lmax + 1):
        sl = a[:, :, l * l:(l + 1) * (l + 1)]          # [np][nbins][2l+1]
        z[l] = 4.0 * np.pi / (2 * l + 1) * np.einsum("p,pim,pjm->ij", wp, sl, sl)
    return z


def _wprim(wprim, np_):
    if wprim is None:
        return None
    wprim = np.ascontiguousarray(wprim, dtype=np.float64)
    if wprim.shape != (np_,):
        raise ValueError("wprim needs one weight per primary")
    return wprim


def zeta(xyz, w, box, rmin, rmax, nbins, lmax, prim=None, amb_tol=0.0, nthreads=0, wprim=None):
    """zeta_l(b1, b2) and its diagnostics, summed over the given primaries.

    ``wprim`` (one per primary, optional) replaces each primary's own weight
    in the sum over primaries.  Returns a dict with ``zeta`` and ``gram`` ([lmax+1][nbins][nbins]),
    ``wpairs`` and ``selfw`` ([nbins]), ``npairs`` and ``namb`` (ints).
    """
    lib = _load()
    xyz, w = _points(xyz, w)
    prim = _prim(prim)
    n = xyz.shape[0]
    np_ = n if prim is None else prim.shape[0]
    wprim = _wprim(wprim, np_)
    shape = (lmax + 1, nbins, nbins)
    z = np.zeros(shape)
    g = np.zeros(shape)
    wp = np.zeros(nbins)
    sw = np.zeros(nbins)
    npairs = ctypes.c_int64(0)
    namb = ctypes.c_int64(0)
    rc = lib.oracle_zeta(_ptr(xyz), _ptr(w), n, float(box), float(rmin), float(rmax),
                         int(nbins), int(lmax), _ptr(prim), np_, _ptr(z), _ptr(g),
                         _ptr(wp), _ptr(sw), ctypes.byref(npairs), ctypes.byref(namb),
                         float(amb_tol), int(nthreads), _ptr(wprim))
    if rc != 0:
        raise ValueError(f"oracle_zeta rejected its arguments (rc={rc})")
    return {"zeta": z, "gram": g, "wpairs": wp, "selfw": sw,
            "npairs": int(npairs.value), "namb": int(namb.value)}


def zeta_sphere(xyz, w, theta_min, theta_max, nbins, mmax, prim=None, nthreads=0, wprim=None):
    """Projected (angular) multipoles zeta_m(b1, b2) on the unit sphere, summed
    over the given primaries (ctb_oracle_sphere.c states the definition);
    ``wprim`` as in ``zeta``.

    Returns a dict with ``zeta`` and ``gram`` ([mmax+1][nbins][nbins]),
    ``wpairs`` ([nbins]) and ``npairs``.
    """
    lib = _load()
    xyz, w = _points(xyz, w)
    prim = _prim(prim)
    n = xyz.shape[0]
    np_ = n if prim is None else prim.shape[0]
    wprim = _wprim(wprim, np_)
    shape = (mmax + 1, nbins, nbins)
    z = np.zeros(shape)
    g = np.zeros(shape)
    wp = np.zeros(nbins)
    npairs = ctypes.c_int64(0)
    rc = lib.oracle_zeta_sphere(_ptr(xyz), _ptr(w), n, float(theta_min), float(theta_max), int(nbins),
                                int(mmax), _ptr(prim), np_, _ptr(z), _ptr(g), _ptr(wp),
                                ctypes.byref(npairs), int(nthreads), _ptr(wprim))
    if rc != 0:
        raise ValueError(f"oracle_zeta_sphere rejected its arguments (rc={rc})")
    return {"zeta": z, "gram": g, "wpairs": wp, "npairs": int(npairs.value)}
