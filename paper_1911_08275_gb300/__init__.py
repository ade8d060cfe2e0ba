"""cfgpu: exact cell-list pair counting on NVIDIA GB300 (sm_103a).

Python binding of the C ABI in ``include/cf.h`` (ctypes; argument marshalling
only -- every step of the computation runs in the CUDA library).  The
operation is the pair-separation histogram of Sinha & Garrison,
arXiv:1911.08275 (Sec. 1.1, Code 1 and Eq. "separations").

    import paper_1911_08275_gb300 as cf
    r = cf.countpairs_xi(x, y, z, edges, boxsize=420.0)         # auto, periodic
    r.npairs                                                    # uint64 histogram

Inputs are torch tensors (CUDA or CPU) or numpy arrays, float32 or float64,
one per coordinate.  There is no CPU fallback: if the CUDA library cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

CF_OK, CF_EINVAL, CF_ENOMEM, CF_ECUDA, CF_ETIMEOUT, CF_EDEVICE = 0, -1, -2, -3, -4, -5
CF_FLOAT32, CF_FLOAT64 = 0, 1
CF_MODE_FP64, CF_MODE_FP32_RECHECK = 0, 1
CF_FLAG_COUNT_EVALS = 1 << 0
CF_FLAG_NO_PRUNE = 1 << 1
CF_FLAG_VERIFY_BAND = 1 << 2
CF_FLAG_DEBUG_STALL = 1 << 3

_STATUS = {CF_EINVAL: "CF_EINVAL", CF_ENOMEM: "CF_ENOMEM", CF_ECUDA: "CF_ECUDA",
           CF_ETIMEOUT: "CF_ETIMEOUT", CF_EDEVICE: "CF_EDEVICE"}

# Names exported by the library; they must match include/cf.h.
EXPORTS = ("cf_countpairs_xi", "cf_countpairs_rp_pi", "cf_last_error", "cf_version",
           "cf_countpairs_xi_noalloc", "cf_tune_save", "cf_tune_load", "cf_tune_clear",
           "cf_tune_count", "cf_batch_create", "cf_batch_add_xi", "cf_batch_add_rp_pi",
           "cf_batch_run", "cf_batch_destroy", "cf_debug_bin_tables", "cf_debug_pi_band")


class cf_catalog(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("w", ctypes.c_void_p), ("n", ctypes.c_int64)]


class cf_config(ctypes.Structure):
    _fields_ = [("periodic", ctypes.c_int), ("boxsize", ctypes.c_double * 3),
                ("dtype", ctypes.c_int), ("mode", ctypes.c_int), ("weighted", ctypes.c_int),
                ("want_ravg", ctypes.c_int), ("refine", ctypes.c_int * 3),
                ("flags", ctypes.c_uint32), ("stream", ctypes.c_void_p), ("autotune", ctypes.c_int),
                ("pair_chunk", ctypes.c_int), ("pair_pp", ctypes.c_int),
                ("shard_index", ctypes.c_int), ("shard_count", ctypes.c_int)]


class cf_result(ctypes.Structure):
    _fields_ = [("npairs", ctypes.POINTER(ctypes.c_uint64)), ("wsum", ctypes.POINTER(ctypes.c_double)),
                ("ravg", ctypes.POINTER(ctypes.c_double)), ("n_cellpairs", ctypes.c_uint64),
                ("n_evaluated", ctypes.c_uint64), ("n_rechecked", ctypes.c_uint64),
                ("n_band_violations", ctypes.c_uint64), ("kernel_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("n_kernels", ctypes.c_uint64),
                ("refine_used", ctypes.c_int * 3), ("chunk_used", ctypes.c_int),
                ("pp_used", ctypes.c_int), ("tuned", ctypes.c_int),
                ("table_linear", ctypes.c_int)]


class CfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    from . import build as _b
    return _b.LIB


def lib(build_if_stale: bool = True):
    """Load libcfgpu.so (compiling it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _b
            path = _b.build() if build_if_stale else _b.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"cfgpu CUDA library not found at {path}")
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            L.cf_countpairs_xi.argtypes = [ctypes.c_int, P(cf_catalog), P(cf_catalog),
                                           P(ctypes.c_double), ctypes.c_int, P(cf_config),
                                           P(cf_result)]
            L.cf_countpairs_xi.restype = ctypes.c_int
            L.cf_countpairs_rp_pi.argtypes = [ctypes.c_int, P(cf_catalog), P(cf_catalog),
                                              P(ctypes.c_double), ctypes.c_int, ctypes.c_double,
                                              ctypes.c_int, P(cf_config), P(cf_result)]
            L.cf_countpairs_rp_pi.restype = ctypes.c_int
            L.cf_last_error.restype = ctypes.c_char_p
            L.cf_version.restype = ctypes.c_char_p
            _lib = L
    return _lib


@dataclass
class Result:
    npairs: np.ndarray
    wsum: np.ndarray | None
    ravg: np.ndarray | None
    n_cellpairs: int
    n_evaluated: int
    n_rechecked: int
    n_band_violations: int
    kernel_ms: float
    total_ms: float
    n_kernels: int = 0
    refine_used: tuple = (0, 0, 0)
    chunk_used: int = 0
    pp_used: int = 0
    tuned: int = 0
    table_linear: int = 0


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


_TORCH_CODES = None  # torch dtype -> cf_dtype, filled on first use (torch imported lazily)


def _arr(a, name):
    """(pointer, dtype code, n, is_cuda, keepalive) of a 1-D contiguous array."""
    global _TORCH_CODES
    if _is_torch(a):
        if _TORCH_CODES is None:
            import torch
            _TORCH_CODES = {torch.float32: CF_FLOAT32, torch.float64: CF_FLOAT64}
        if a.dim() != 1 or not a.is_contiguous():
            raise ValueError(f"{name} must be a 1-D contiguous tensor")
        n = a.numel()
        return a.data_ptr() if n else None, _TORCH_CODES.get(a.dtype), n, a.is_cuda, a
    a = np.ascontiguousarray(a)
    if a.ndim != 1:
        raise ValueError(f"{name} must be 1-D")
    code = {np.dtype(np.float32): CF_FLOAT32, np.dtype(np.float64): CF_FLOAT64}.get(a.dtype)
    return a.ctypes.data if a.size else None, code, a.size, False, a


def _catalog(x, y, z, w, keep):
    ax, ay, az = _arr(x, "x"), _arr(y, "y"), _arr(z, "z")
    if not (ax[1] == ay[1] == az[1]) or ax[1] is None:
        raise ValueError("x, y, z must share one dtype, float32 or float64")
    if not (ax[2] == ay[2] == az[2]):
        raise ValueError("x, y, z must have the same length")
    keep += [ax[4], ay[4], az[4]]
    wp = None
    if w is not None:
        aw = _arr(w, "w")
        if aw[1] != CF_FLOAT64 or aw[2] != ax[2]:
            raise ValueError("weights must be float64 with one value per point")
        keep.append(aw[4])
        wp = aw[0]
    return cf_catalog(ax[0], ay[0], az[0], wp, ax[2]), ax[1], ax[3]


def _config(dtype, periodic, boxsize, mode, weighted, want_ravg, refine, flags, stream, cuda,
            tuning=None):
    c = cf_config()
    tuning = tuning or {}
    c.autotune = 1 if tuning.get("autotune") else 0
    c.pair_chunk = int(tuning.get("pair_chunk", 0))
    c.pair_pp = int(tuning.get("pair_pp", 0))
    shard = tuning.get("shard") or (0, 0)
    c.shard_index, c.shard_count = int(shard[0]), int(shard[1])
    c.periodic = 1 if periodic else 0
    if boxsize is None:
        boxsize = 0.0
    if isinstance(boxsize, (int, float)):
        c.boxsize[0] = c.boxsize[1] = c.boxsize[2] = float(boxsize)
    else:
        b = np.broadcast_to(np.asarray(boxsize, dtype=np.float64), (3,))
        c.boxsize[:] = [float(v) for v in b]
    c.dtype = dtype
    c.mode = {"fp64": CF_MODE_FP64, "fp32_recheck": CF_MODE_FP32_RECHECK}[mode]
    c.weighted = 1 if weighted else 0
    c.want_ravg = 1 if want_ravg else 0
    c.refine[0], c.refine[1], c.refine[2] = (int(v) for v in refine)
    c.flags = int(flags)
    if stream is None and cuda:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    c.stream = int(stream) if stream else None
    return c


def _run(fn, nslots, autocorr, x, y, z, w, x2, y2, z2, w2, extra, periodic, boxsize, mode,
         want_ravg, refine, flags, stream, tuning=None):
    L = lib()
    keep = []
    c1, dt, cuda = _catalog(x, y, z, w, keep)
    c2 = None
    if not autocorr:
        if x2 is None:
            raise ValueError("cross-correlation needs x2, y2, z2")
        c2, dt2, cuda2 = _catalog(x2, y2, z2, w2, keep)
        if dt2 != dt:
            raise ValueError("both catalogues must share one dtype")
        cuda = cuda or cuda2
    weighted = w is not None
    cfg = _config(dt, periodic, boxsize, mode, weighted, want_ravg, refine, flags, stream, cuda,
                  tuning)
    npairs = np.zeros(nslots, dtype=np.uint64)
    wsum = np.zeros(nslots) if weighted else None
    ravg = np.zeros(nslots) if want_ravg else None
    res = cf_result()
    res.npairs = npairs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    res.wsum = wsum.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if wsum is not None else None
    res.ravg = ravg.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if ravg is not None else None
    st = fn(L, int(bool(autocorr)), ctypes.byref(c1), ctypes.byref(c2) if c2 is not None else None,
            *extra, ctypes.byref(cfg), ctypes.byref(res))
    if st != CF_OK:
        raise CfError(st, L.cf_last_error().decode())
    return Result(npairs, wsum, ravg, int(res.n_cellpairs), int(res.n_evaluated),
                  int(res.n_rechecked), int(res.n_band_violations), float(res.kernel_ms),
                  float(res.total_ms), int(res.n_kernels), tuple(res.refine_used),
                  int(res.chunk_used), int(res.pp_used), int(res.tuned), int(res.table_linear))


def countpairs_xi(x, y, z, edges, *, w=None, x2=None, y2=None, z2=None, w2=None, autocorr=None,
                  periodic=True, boxsize=420.0, mode="fp32_recheck", want_ravg=False,
                  refine=(0, 0, 0), flags=0, stream=None, autotune=False, pair_chunk=0,
                  pair_pp=0, shard=None) -> Result:
    """DD(r) histogram through ``cf_countpairs_xi`` (see include/cf.h).

    shard=(k, n) counts only shard k of n (see cf_config.shard_index); the n
    shards' histograms sum to the full result."""
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    if autocorr is None:
        autocorr = x2 is None
    fn = lambda L, *a: L.cf_countpairs_xi(*a)  # noqa: E731
    extra = (edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(edges.size))
    return _run(fn, edges.size - 1, autocorr, x, y, z, w, x2, y2, z2, w2, extra, periodic, boxsize,
                mode, want_ravg, refine, flags, stream,
                dict(autotune=autotune, pair_chunk=pair_chunk, pair_pp=pair_pp, shard=shard))


def countpairs_rp_pi(x, y, z, rp_edges, pimax, npibins, *, w=None, x2=None, y2=None, z2=None,
                     w2=None, autocorr=None, periodic=True, boxsize=420.0, mode="fp32_recheck",
                     want_ravg=False, refine=(0, 0, 0), flags=0, stream=None,
                     autotune=False, shard=None) -> Result:
    """DD(rp, pi) histogram (rp-major, shape (nrp, npibins)) through ``cf_countpairs_rp_pi``."""
    rp_edges = np.ascontiguousarray(rp_edges, dtype=np.float64)
    if autocorr is None:
        autocorr = x2 is None
    fn = lambda L, *a: L.cf_countpairs_rp_pi(*a)  # noqa: E731
    extra = (rp_edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(rp_edges.size),
             ctypes.c_double(float(pimax)), int(npibins))
    r = _run(fn, (rp_edges.size - 1) * int(npibins), autocorr, x, y, z, w, x2, y2, z2, w2, extra,
             periodic, boxsize, mode, want_ravg, refine, flags, stream,
             dict(autotune=autotune, shard=shard))
    shp = (rp_edges.size - 1, int(npibins))
    r.npairs = r.npairs.reshape(shp)
    if r.wsum is not None:
        r.wsum = r.wsum.reshape(shp)
    if r.ravg is not None:
        r.ravg = r.ravg.reshape(shp)
    return r


def version() -> str:
    return lib().cf_version().decode()


def _tune_call(name, *args):
    L = lib()
    f = getattr(L, name)
    f.restype = ctypes.c_int
    st = f(*args)
    if st < 0:
        raise CfError(st, L.cf_last_error().decode())
    return st


def tune_save(path: str) -> None:
    """Write the autotuner cache to a JSON file (``cf_tune_save``)."""
    _tune_call("cf_tune_save", os.fsencode(path))


def tune_load(path: str) -> None:
    """Merge a JSON autotuner cache file into the cache (``cf_tune_load``)."""
    _tune_call("cf_tune_load", os.fsencode(path))


def tune_clear() -> None:
    _tune_call("cf_tune_clear")


def tune_count() -> int:
    return _tune_call("cf_tune_count")


class cf_bin_tables(ctypes.Structure):
    _fields_ = [("nthr", ctypes.c_int), ("lut_n", ctypes.c_int), ("lin", ctypes.c_int),
                ("lscale", ctypes.c_float), ("shift", ctypes.c_int), ("u0", ctypes.c_uint)]


CF_BIN_TABLE_MAX = 16384


def debug_bin_tables(edges, *, ncomp=3, coord_max, shift_max=0.0, rmax=None):
    """Float32 thresholds and bin table for these edges (``cf_debug_bin_tables``).

    Host only.  Returns (thr float32 [2 * nedges], table uint8 [lut_n], info
    dict with lin, lscale, shift, u0); see include/cf.h for their meaning.
    """
    L = lib()
    f = L.cf_debug_bin_tables
    P = ctypes.POINTER
    f.argtypes = [P(ctypes.c_double), ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                  ctypes.c_double, P(ctypes.c_float), P(ctypes.c_ubyte), P(cf_bin_tables)]
    f.restype = ctypes.c_int
    e = np.ascontiguousarray(edges, dtype=np.float64)
    rmax = float(e[-1]) if rmax is None else float(rmax)
    thr = np.zeros(max(2 * e.size, 1), dtype=np.float32)
    tab = np.zeros(CF_BIN_TABLE_MAX, dtype=np.uint8)
    info = cf_bin_tables()
    st = f(e.ctypes.data_as(P(ctypes.c_double)), int(e.size), int(ncomp), float(coord_max),
           float(shift_max), rmax, thr.ctypes.data_as(P(ctypes.c_float)),
           tab.ctypes.data_as(P(ctypes.c_ubyte)), ctypes.byref(info))
    if st < 0:
        raise CfError(st, L.cf_last_error().decode())
    return thr[:info.nthr].copy(), tab[:info.lut_n].copy(), {
        "lin": info.lin, "lscale": info.lscale, "shift": info.shift, "u0": info.u0}


def debug_pi_band(pimax, npibins, *, coord_max, shift_max=0.0):
    """(pscale, pband) of the float32 pi-bin decision (``cf_debug_pi_band``, host only)."""
    L = lib()
    f = L.cf_debug_pi_band
    P = ctypes.POINTER
    f.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                  P(ctypes.c_float), P(ctypes.c_float)]
    f.restype = ctypes.c_int
    ps, pb = ctypes.c_float(), ctypes.c_float()
    st = f(float(pimax), int(npibins), float(coord_max), float(shift_max), ctypes.byref(ps),
           ctypes.byref(pb))
    if st < 0:
        raise CfError(st, L.cf_last_error().decode())
    return np.float32(ps.value), np.float32(pb.value)


def countpairs_xi_noalloc(x, y, z, edges, *, x2=None, y2=None, z2=None, autocorr=None,
                          periodic=True, boxsize=420.0, mode="fp32_recheck", refine=(0, 0, 0),
                          flags=0, stream=None) -> Result:
    """DD(r) through ``cf_countpairs_xi_noalloc``: no device allocation per call.

    For callers that cannot allocate GPU memory while counting (see include/cf.h):
    inputs must be CUDA tensors, at most 131072 points per catalogue, unweighted.
    Calls on one device share the library's static scratch, so they must not
    overlap on the GPU.
    """
    L = lib()
    L.cf_countpairs_xi_noalloc.argtypes = L.cf_countpairs_xi.argtypes
    L.cf_countpairs_xi_noalloc.restype = ctypes.c_int
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    if autocorr is None:
        autocorr = x2 is None
    fn = lambda L, *a: L.cf_countpairs_xi_noalloc(*a)  # noqa: E731
    extra = (edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(edges.size))
    return _run(fn, edges.size - 1, autocorr, x, y, z, None, x2, y2, z2, None, extra, periodic,
                boxsize, mode, False, refine, flags, stream)


class cf_batch_stats(ctypes.Structure):
    _fields_ = [("n_jobs", ctypes.c_uint64), ("n_kernels", ctypes.c_uint64),
                ("pairs", ctypes.c_uint64), ("used_graph", ctypes.c_int), ("planned", ctypes.c_int),
                ("blocks", ctypes.c_int), ("kernel_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double)]


class Batch:
    """Many DD(r) / DD(rp, pi) jobs in one persistent launch (``cf_batch_*``).

    ``add_xi`` / ``add_rp_pi`` take the arguments of ``countpairs_xi`` /
    ``countpairs_rp_pi`` (CUDA tensors, unweighted) and return a ``Result``
    that ``run`` fills.  ``run(use_graph=True)`` captures the launch sequence
    into a CUDA graph on its first call and replays it afterwards.
    """

    def __init__(self):
        L = lib()
        self._L = L
        self._ptr = ctypes.c_void_p()
        L.cf_batch_create.argtypes = [ctypes.POINTER(ctypes.c_void_p)]
        L.cf_batch_create.restype = ctypes.c_int
        P = ctypes.POINTER
        L.cf_batch_add_xi.argtypes = [ctypes.c_void_p, ctypes.c_int, P(cf_catalog), P(cf_catalog),
                                      P(ctypes.c_double), ctypes.c_int, P(cf_config), P(cf_result)]
        L.cf_batch_add_xi.restype = ctypes.c_int
        L.cf_batch_add_rp_pi.argtypes = [ctypes.c_void_p, ctypes.c_int, P(cf_catalog),
                                         P(cf_catalog), P(ctypes.c_double), ctypes.c_int,
                                         ctypes.c_double, ctypes.c_int, P(cf_config), P(cf_result)]
        L.cf_batch_add_rp_pi.restype = ctypes.c_int
        L.cf_batch_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                   P(cf_batch_stats)]
        L.cf_batch_run.restype = ctypes.c_int
        L.cf_batch_destroy.argtypes = [ctypes.c_void_p]
        L.cf_batch_destroy.restype = ctypes.c_int
        st = L.cf_batch_create(ctypes.byref(self._ptr))
        if st != CF_OK:
            raise CfError(st, L.cf_last_error().decode())
        self._jobs = []  # (Result, cf_result, shape, keepalive)

    def _add(self, kind, x, y, z, edges, x2, y2, z2, autocorr, periodic, boxsize, mode, refine,
             flags, autotune, pimax=0.0, npibins=0):
        keep = []
        c1, dt, cuda = _catalog(x, y, z, None, keep)
        if autocorr is None:
            autocorr = x2 is None
        c2 = None
        if not autocorr:
            c2, dt2, _ = _catalog(x2, y2, z2, None, keep)
            if dt2 != dt:
                raise ValueError("both catalogues must share one dtype")
        cfg = _config(dt, periodic, boxsize, mode, False, False, refine, flags, None, False,
                      dict(autotune=autotune))
        edges = np.ascontiguousarray(edges, dtype=np.float64)
        nslots = (edges.size - 1) * (int(npibins) if kind == 1 else 1)
        npairs = np.zeros(nslots, dtype=np.uint64)
        res = cf_result()
        res.npairs = npairs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        eptr = edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c2p = ctypes.byref(c2) if c2 is not None else None
        if kind == 0:
            st = self._L.cf_batch_add_xi(self._ptr, int(bool(autocorr)), ctypes.byref(c1), c2p,
                                         eptr, int(edges.size), ctypes.byref(cfg),
                                         ctypes.byref(res))
        else:
            st = self._L.cf_batch_add_rp_pi(self._ptr, int(bool(autocorr)), ctypes.byref(c1), c2p,
                                            eptr, int(edges.size), ctypes.c_double(float(pimax)),
                                            int(npibins), ctypes.byref(cfg), ctypes.byref(res))
        if st != CF_OK:
            raise CfError(st, self._L.cf_last_error().decode())
        r = Result(npairs if kind == 0 else npairs.reshape(edges.size - 1, int(npibins)), None,
                   None, 0, 0, 0, 0, 0.0, 0.0)
        self._jobs.append((r, res, (c1, c2, cfg, edges, npairs, keep)))
        return r

    def add_xi(self, x, y, z, edges, *, x2=None, y2=None, z2=None, autocorr=None, periodic=True,
               boxsize=420.0, mode="fp32_recheck", refine=(0, 0, 0), flags=0,
               autotune=False) -> Result:
        return self._add(0, x, y, z, edges, x2, y2, z2, autocorr, periodic, boxsize, mode, refine,
                         flags, autotune)

    def add_rp_pi(self, x, y, z, rp_edges, pimax, npibins, *, x2=None, y2=None, z2=None,
                  autocorr=None, periodic=True, boxsize=420.0, mode="fp32_recheck",
                  refine=(0, 0, 0), flags=0, autotune=False) -> Result:
        return self._add(1, x, y, z, rp_edges, x2, y2, z2, autocorr, periodic, boxsize, mode,
                         refine, flags, autotune, pimax, npibins)

    def run(self, use_graph: bool = True, stream=None) -> dict:
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        stats = cf_batch_stats()
        st = self._L.cf_batch_run(self._ptr, ctypes.c_void_p(int(stream) if stream else None),
                                  int(bool(use_graph)), ctypes.byref(stats))
        if st != CF_OK:
            raise CfError(st, self._L.cf_last_error().decode())
        for r, res, _ in self._jobs:
            r.n_cellpairs = int(res.n_cellpairs)
            r.n_rechecked = int(res.n_rechecked)
            r.kernel_ms = float(res.kernel_ms)
            r.total_ms = float(res.total_ms)
            r.n_kernels = int(res.n_kernels)
            r.refine_used = tuple(res.refine_used)
            r.chunk_used = int(res.chunk_used)
            r.pp_used = int(res.pp_used)
            r.tuned = int(res.tuned)
        return {f: getattr(stats, f) for f, _ in cf_batch_stats._fields_}

    def close(self) -> None:
        if self._ptr:
            self._L.cf_batch_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
