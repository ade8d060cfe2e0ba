"""Brute-force CPU oracle and the gridded CPU baseline (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this package.  It compiles ``oracle.c`` (and ``gridded.c``) with gcc
(``-ffp-contract=off``: no fused multiply-add, so every operation is one
correctly rounded binary64 operation) and wraps them with ctypes.

Functions (all inputs are numpy arrays; float32 positions are promoted exactly
to float64 before the call):

* ``xi(...)``    DD(r) of Sec. 1.1 (Code 1, Eq. "separations"), brute force;
* ``rppi(...)``  DD(rp, pi), rp-major 2-D histogram, line of sight = z, brute force;
* ``gridded_xi(...)``  DD(r) by cell lists (Sec. 1.2 / 2.1 / 2.2, scalar, OpenMP):
  the plain gridded CPU count the benchmark reports as its CPU baseline; the
  tests pin it to ``xi`` bit for bit.

``xi`` and ``rppi`` return ``(npairs[uint64], wsum[float64] or None, rsum[float64]
or None)``; ``gridded_xi`` returns ``npairs``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_GSRC = os.path.join(_HERE, "gridded.c")
_GOUT = os.path.join(_HERE, "_build", "libgridded.so")
_lock = threading.Lock()
_lib = None
_glib = None

_D = ctypes.POINTER(ctypes.c_double)
_U = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False, src: str = _SRC, out: str = _OUT, opt: str = "-O2") -> str:
    """Compile the oracle shared library (gcc, OpenMP, no FP contraction)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", opt, "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build_gridded(force: bool = False) -> str:
    """Compile the gridded CPU counter (gcc -O3, OpenMP, no FP contraction)."""
    return build(force=force, src=_GSRC, out=_GOUT, opt="-O3")


def _bind(path: str):
    lib = ctypes.CDLL(path)
    common = [ctypes.c_int, ctypes.c_int64, _D, _D, _D, _D, ctypes.c_int64, _D, _D, _D, _D,
              ctypes.c_int, _D]
    lib.oracle_xi.argtypes = common + [_D, ctypes.c_int, _U, _D, _D]
    lib.oracle_xi.restype = ctypes.c_int
    lib.oracle_rppi.argtypes = common + [_D, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                         _U, _D, _D]
    lib.oracle_rppi.restype = ctypes.c_int
    lib.oracle_num_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _f64(a):
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_D)


def _cat(x, y, z, w):
    x, y, z, w = _f64(x), _f64(y), _f64(z), _f64(w)
    n = 0 if x is None else x.size
    return n, (x, y, z, w)


def _call(fn, autocorr, c1, c2, periodic, box, edges, extra, nslots, want_r):
    n1, a1 = c1
    n2, a2 = c2 if c2 is not None else (0, (None, None, None, None))
    edges = _f64(edges)
    boxa = None if box is None else _f64(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    npairs = np.zeros(nslots, dtype=np.uint64)
    weighted = a1[3] is not None
    wsum = np.zeros(nslots) if weighted else None
    rsum = np.zeros(nslots) if want_r else None
    st = fn(int(autocorr), n1, *map(_ptr, a1), n2, *map(_ptr, a2), int(periodic), _ptr(boxa),
            _ptr(edges), int(edges.size), *extra, npairs.ctypes.data_as(_U), _ptr(wsum), _ptr(rsum))
    if st != 0:
        raise ValueError(f"oracle returned status {st}")
    return npairs, wsum, rsum


class Oracle:
    """Bound oracle functions of one compiled library (the default build, or a
    test build of a modified source)."""

    def __init__(self, lib):
        self._lib = lib

    def xi(self, x1, y1, z1, *, edges, w1=None, x2=None, y2=None, z2=None, w2=None,
           autocorr=True, periodic=True, box=None, want_r=False):
        """DD(r) histogram (ordered pairs), see ``oracle.c``."""
        c1 = _cat(x1, y1, z1, w1)
        c2 = None if autocorr else _cat(x2, y2, z2, w2)
        nb = len(edges) - 1
        return _call(self._lib.oracle_xi, autocorr, c1, c2, periodic, box, edges, (), nb, want_r)

    def rppi(self, x1, y1, z1, *, rp_edges, pimax, npibins, w1=None, x2=None, y2=None, z2=None,
             w2=None, autocorr=True, periodic=True, box=None, want_r=False):
        """DD(rp, pi) histogram, shape (len(rp_edges)-1, npibins), see ``oracle.c``."""
        c1 = _cat(x1, y1, z1, w1)
        c2 = None if autocorr else _cat(x2, y2, z2, w2)
        nb = (len(rp_edges) - 1) * int(npibins)
        npairs, wsum, rsum = _call(self._lib.oracle_rppi, autocorr, c1, c2, periodic, box,
                                   rp_edges, (ctypes.c_double(float(pimax)), int(npibins)), nb,
                                   want_r)
        shp = (len(rp_edges) - 1, int(npibins))
        return (npairs.reshape(shp), None if wsum is None else wsum.reshape(shp),
                None if rsum is None else rsum.reshape(shp))


def load_variant(path: str) -> Oracle:
    """Oracle bound to another compiled build (used to plant mistakes in tests)."""
    return Oracle(_bind(path))


def xi(*args, **kw):
    return Oracle(_load()).xi(*args, **kw)


def rppi(*args, **kw):
    return Oracle(_load()).rppi(*args, **kw)


xi.__doc__ = Oracle.xi.__doc__
rppi.__doc__ = Oracle.rppi.__doc__


def _load_gridded():
    global _glib
    with _lock:
        if _glib is None:
            lib = ctypes.CDLL(build_gridded())
            lib.gridded_xi.argtypes = [ctypes.c_int, ctypes.c_int64, _D, _D, _D, ctypes.c_int64, _D,
                                       _D, _D, ctypes.c_int, _D, _D, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), _U]
            lib.gridded_xi.restype = ctypes.c_int
            lib.gridded_num_threads.restype = ctypes.c_int
            _glib = lib
    return _glib


def gridded_num_threads() -> int:
    return int(_load_gridded().gridded_num_threads())


def gridded_xi(x1, y1, z1, *, edges, x2=None, y2=None, z2=None, autocorr=True, periodic=True,
               box=None, refine=(2, 2, 1)):
    """DD(r) histogram (ordered pairs) by cell lists, see ``gridded.c``."""
    lib = _load_gridded()
    n1, a1 = _cat(x1, y1, z1, None)
    n2, a2 = (0, (None, None, None, None)) if autocorr else _cat(x2, y2, z2, None)
    edges = _f64(edges)
    boxa = None if box is None else _f64(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    ref = (ctypes.c_int * 3)(*[int(v) for v in refine])
    npairs = np.zeros(edges.size - 1, dtype=np.uint64)
    st = lib.gridded_xi(int(autocorr), n1, *map(_ptr, a1[:3]), n2, *map(_ptr, a2[:3]),
                        int(periodic), _ptr(boxa), _ptr(edges), int(edges.size), ref,
                        npairs.ctypes.data_as(_U))
    if st != 0:
        raise ValueError(f"gridded counter returned status {st}")
    return npairs
