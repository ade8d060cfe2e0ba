"""Seeded synthetic catalogues shaped like the paper's workloads.

This module only draws inputs: positions, weights and bin edges.  It holds
none of the pair-counting arithmetic, and both the CUDA path and the CPU
oracle consume what it returns.

Bit-exact reproducibility across machines (x86 build host, Arm GPU host, any
numpy version) is a design goal, because stored expected histograms are keyed
on the exact bits of a catalogue.  Therefore:

* random bits come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014) used as a counter-based
  generator, evaluated with numpy uint64 wrap-around arithmetic;
* floating point uses only IEEE-754 correctly rounded operations
  (+, -, *, /, sqrt, frexp/ldexp, comparisons).  The natural logarithm and
  exponential needed for Gaussian offsets, Poisson counts and log-spaced bin
  edges are evaluated here by argument reduction plus a truncated series, not
  by the platform's libm, whose last bit may differ between machines.

Workloads (the paper's catalogue is a 1.2M-galaxy periodic box of side 420,
Sec. 3; it is not available, so a Neyman-Scott process stands in for it):

* ``uniform_box``      -- i.i.d. uniform points in [0, L)^3;
* ``neyman_scott``     -- Poisson(mean) children per uniform parent, with
  isotropic Gaussian offsets of width sigma, wrapped into the periodic box;
* ``log_edges``        -- log-spaced bin edges from rmin to rmax.
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass

import numpy as np

_U64 = np.uint64
_GAMMA = _U64(0x9E3779B97F4A7C15)
_M1 = _U64(0xBF58476D1CE4E5B9)
_M2 = _U64(0x94D049BB133111EB)
_STREAM_MUL = _U64(0xD1B54A32D192ED03)
_TWO_M53 = 2.0 ** -53
_LN2 = float.fromhex("0x1.62e42fefa39efp-1")  # nearest double to ln 2


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied element-wise (uint64 in/out)."""
    z = z.copy()
    z ^= z >> _U64(30)
    z *= _M1
    z ^= z >> _U64(27)
    z *= _M2
    z ^= z >> _U64(31)
    return z


def random_u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """``n`` SplitMix64 outputs for (seed, stream), starting at counter ``offset``."""
    with np.errstate(over="ignore"):
        key = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=_U64)
        key ^= np.array([stream & 0xFFFFFFFFFFFFFFFF], dtype=_U64) * _STREAM_MUL
        base = _mix64(key)[0]
        ctr = np.arange(offset + 1, offset + n + 1, dtype=_U64)
        return _mix64(base + ctr * _GAMMA)


def uniform01(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits each (exact conversion)."""
    u = random_u64(seed, stream, n, offset) >> _U64(11)
    return u.astype(np.float64) * _TWO_M53


def _ln(x: np.ndarray) -> np.ndarray:
    """Natural log of positive finite doubles by frexp reduction + atanh series.

    ln(x) = e ln2 + 2 atanh(t), t = (m - 1)/(m + 1), m in [sqrt(1/2), sqrt(2)),
    so |t| < 0.1716 and the odd series converges to < 1e-17 in 14 terms.
    """
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    small = m < 0.7071067811865476
    m = np.where(small, m * 2.0, m)
    e = np.where(small, e - 1, e).astype(np.float64)
    t = (m - 1.0) / (m + 1.0)
    t2 = t * t
    acc = np.full_like(t, 1.0 / 29.0)
    for k in range(13, -1, -1):
        acc = acc * t2 + 1.0 / (2 * k + 1)
    return e * _LN2 + 2.0 * t * acc


def _exp(x: np.ndarray) -> np.ndarray:
    """exp of moderate doubles by ln2 reduction + Taylor series (|r| <= ln2/2)."""
    x = np.asarray(x, dtype=np.float64)
    k = np.floor(x / _LN2 + 0.5)
    r = x - k * _LN2
    acc = np.ones_like(r)
    for n in range(22, 0, -1):
        acc = acc * r / float(n) + 1.0
    return np.ldexp(acc, k.astype(np.int64))


def _wrap(v: np.ndarray, box: float) -> np.ndarray:
    """Map values within one period of [0, box) into [0, box)."""
    v = v.copy()
    for _ in range(4):
        hi = v >= box
        lo = v < 0.0
        if not (hi.any() or lo.any()):
            break
        v[hi] -= box
        v[lo] += box
    assert np.all((v >= 0.0) & (v < box))
    return v


def gaussian(seed: int, stream: int, n: int) -> np.ndarray:
    """``n`` standard normal deviates by Marsaglia's polar method."""
    out = np.empty(0, dtype=np.float64)
    offset = 0
    while out.size < n:
        need = n - out.size
        m = int((need // 2 + 1) * 1.35) + 64
        u = uniform01(seed, stream, 2 * m, offset) * 2.0 - 1.0
        offset += 2 * m
        a, b = u[0::2], u[1::2]
        s = a * a + b * b
        ok = (s > 0.0) & (s < 1.0)
        a, b, s = a[ok], b[ok], s[ok]
        f = np.sqrt(-2.0 * _ln(s) / s)
        pair = np.empty(2 * a.size, dtype=np.float64)
        pair[0::2] = a * f
        pair[1::2] = b * f
        out = np.concatenate([out, pair])
    return out[:n]


def poisson(seed: int, stream: int, n: int, mean: float) -> np.ndarray:
    """``n`` Poisson(mean) counts: arrivals of a unit-rate process in [0, mean]."""
    width = int(mean + 12.0 * np.sqrt(mean) + 40)
    u = uniform01(seed, stream, n * width).reshape(n, width)
    gaps = -_ln(1.0 - u)  # exponential(1) inter-arrival times; 1-u in (0, 1]
    arrival = np.cumsum(gaps, axis=1)
    counts = np.count_nonzero(arrival <= mean, axis=1)
    if np.any(counts == width):
        raise RuntimeError("poisson: truncation width exceeded")
    return counts.astype(np.int64)


@dataclass
class Catalog:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    w: np.ndarray | None
    box: float
    name: str

    @property
    def n(self) -> int:
        return int(self.x.size)

    def astype(self, dtype) -> "Catalog":
        """Cast positions (round to nearest); periodic coordinates that round up
        to the box side are mapped back to 0 so they stay in [0, box)."""
        dt = np.dtype(dtype)
        conv = []
        for v in (self.x, self.y, self.z):
            c = v.astype(dt)
            c[c >= dt.type(self.box)] = dt.type(0.0)
            conv.append(c)
        return Catalog(conv[0], conv[1], conv[2], self.w, self.box, f"{self.name}:{dt.name}")

    def digest(self) -> str:
        h = hashlib.sha256()
        for v in (self.x, self.y, self.z) + ((self.w,) if self.w is not None else ()):
            h.update(np.ascontiguousarray(v).tobytes())
        return h.hexdigest()[:16]

    def take(self, idx: np.ndarray) -> "Catalog":
        return Catalog(self.x[idx], self.y[idx], self.z[idx],
                       None if self.w is None else self.w[idx], self.box, self.name + ":take")


def uniform_box(n: int, box: float, seed: int) -> Catalog:
    """i.i.d. uniform points in [0, box)^3 (streams 0, 1, 2 for x, y, z)."""
    xyz = [_wrap(uniform01(seed, s, n) * box, box) for s in range(3)]
    return Catalog(xyz[0], xyz[1], xyz[2], None, float(box), f"uniform(n={n},L={box},seed={seed})")


def neyman_scott(n_parents: int, mean_children: float, sigma: float, box: float,
                 seed: int) -> Catalog:
    """Neyman-Scott cluster process in a periodic box.

    Parents uniform in [0, box)^3 (streams 0-2); children per parent
    Poisson(mean_children) (stream 3); child offsets N(0, sigma^2) per axis
    (streams 4-6); children wrapped into [0, box).  Children are listed
    parent by parent.
    """
    par = [_wrap(uniform01(seed, s, n_parents) * box, box) for s in range(3)]
    counts = poisson(seed, 3, n_parents, mean_children)
    owner = np.repeat(np.arange(n_parents), counts)
    n = owner.size
    xyz = []
    for ax in range(3):
        off = gaussian(seed, 4 + ax, n) * sigma
        xyz.append(_wrap(par[ax][owner] + off, box))
    return Catalog(xyz[0], xyz[1], xyz[2], None, float(box),
                   f"neyman_scott(np={n_parents},mu={mean_children},sigma={sigma},L={box},seed={seed})")


def uniform_weights(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Weights uniform in [lo, hi)."""
    return lo + uniform01(seed, 7, n) * (hi - lo)


def log_edges(rmin: float, rmax: float, nbins: int) -> np.ndarray:
    """``nbins + 1`` log-spaced edges with edges[0] = rmin and edges[-1] = rmax exactly."""
    a, b = _ln(np.array([rmin]))[0], _ln(np.array([rmax]))[0]
    k = np.arange(nbins + 1, dtype=np.float64)
    e = _exp(a + (b - a) * k / float(nbins))
    e[0], e[-1] = rmin, rmax
    assert np.all(np.diff(e) > 0)
    return e


def linear_edges(rmin: float, rmax: float, nbins: int) -> np.ndarray:
    k = np.arange(nbins + 1, dtype=np.float64)
    e = rmin + (rmax - rmin) * k / float(nbins)
    e[-1] = rmax
    return e


# Named workloads of the benchmark and the parity tests.
BOX = 420.0


def c1_uniform20k() -> Catalog:
    """20,000 uniform points, periodic box 420, seed 1."""
    return uniform_box(20_000, BOX, seed=1)


def c2_clustered() -> Catalog:
    """~1.2M Neyman-Scott points: 60,000 parents, Poisson(20) children, sigma 2, box 420, seed 2."""
    return neyman_scott(60_000, 20.0, 2.0, BOX, seed=2)


def c4_randoms(n: int = 12_000_000) -> Catalog:
    """12M uniform randoms in the box 420, seed 3."""
    return uniform_box(n, BOX, seed=3)


def batch_job(j: int, scale: float = 1.0) -> dict:
    """Job j of the 48-job batched workload (seed 1000 + j).

    N log-uniform in [5e4, 2e6] (times ``scale``); even j Neyman-Scott with
    N/20 parents (Poisson(20) children, sigma 2), odd j uniform; box side L
    log-uniform in [100, 1000]; Rmax = round(log-uniform [5, 40]) < L/2.
    Kind alternates in pairs of jobs: DD(r) with 20 log bins 0.1 -> Rmax, then
    DD(rp, pi) with 14 log rp bins 0.1 -> Rmax and pimax = Rmax in unit pi
    bins.  Mode alternates in blocks of four: float32 + re-check, then binary64.
    """
    seed = 1000 + j
    u = uniform01(seed, 20, 3)
    lg = lambda lo, hi, t: float(_exp(np.array([_ln(np.array([lo]))[0] + t * (  # noqa: E731
        _ln(np.array([hi]))[0] - _ln(np.array([lo]))[0])]))[0])
    n = max(2, int(round(lg(5e4, 2e6, u[0]) * scale)))
    box = lg(100.0, 1000.0, u[1])
    rmax = float(min(round(lg(5.0, 40.0, u[2])), int(box / 2.0) - 1))
    if j % 2 == 0:
        cat = neyman_scott(max(1, int(round(n / 20.0))), 20.0, 2.0, box, seed=seed)
    else:
        cat = uniform_box(n, box, seed=seed)
    kind = "xi" if (j // 2) % 2 == 0 else "rppi"
    mode = "fp32_recheck" if (j // 4) % 2 == 0 else "fp64"
    job = dict(j=j, kind=kind, mode=mode, cat=cat, box=box, rmax=rmax)
    if kind == "xi":
        job["edges"] = log_edges(0.1, rmax, 20)
    else:
        job["edges"] = log_edges(0.1, rmax, 14)
        job["pimax"] = rmax
        job["npibins"] = int(rmax)
    return job
