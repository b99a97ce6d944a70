"""Seeded synthetic inputs shared by the oracle-side and the CUDA-side tests.

This module holds random draws only -- none of the model's arithmetic (no
force law, no Roche geometry, no element sizing).  It implements SplitMix64
(Steele, Lea & Flood, OOPSLA 2014) as a counter-based generator: the n-th
output of stream (seed, s) is the variant-13 finaliser applied to
``seed ^ (s * 0xD1B54A32D192ED03) + (n + 1) * 0x9E3779B97F4A7C15`` (mod 2^64),
and uniform doubles take the top 53 bits.  Both the oracle and the library
implement the same published generator independently; the tests cross-check
all three.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_STREAM = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+n-1`` of SplitMix64 stream (seed, stream) as uint64."""
    with np.errstate(over="ignore"):
        s0 = np.uint64(int(seed) & 0xFFFFFFFFFFFFFFFF) ^ (
            np.uint64(int(stream) & 0xFFFFFFFFFFFFFFFF) * _STREAM)
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix(s0 + k * _GAMMA)


def u01(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (
        1.0 / 9007199254740992.0)


class Stream:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int, stream: int = 0):
        self.seed, self.stream, self.pos = int(seed), int(stream), 0

    def uniform(self, n: int) -> np.ndarray:
        out = u01(self.seed, self.stream, n, self.pos)
        self.pos += n
        return out

    def normal(self, n: int) -> np.ndarray:
        """Box-Muller pairs: r = sqrt(-2 ln(1-u1)), (r cos 2pi u2, r sin 2pi u2)."""
        npair = (n + 1) // 2
        u = self.uniform(2 * npair).reshape(npair, 2)
        r = np.sqrt(-2.0 * np.log(1.0 - u[:, 0]))
        z = np.stack([r * np.cos(2.0 * np.pi * u[:, 1]), r * np.sin(2.0 * np.pi * u[:, 1])], 1)
        return z.reshape(-1)[:n]

    def unit_ball(self, n: int) -> np.ndarray:
        """n points uniform in the unit ball by rejection from [-1,1]^3, in draw order."""
        pts = []
        while len(pts) < n:
            c = 2.0 * self.uniform(3) - 1.0
            if c @ c <= 1.0:
                pts.append(c)
        return np.array(pts, dtype=np.float64).reshape(n, 3)


def cloud(n: int, seed: int, *, radius: float = 1.0, center=(0.0, 0.0, 0.0),
          speed: float = 1.0, stream: int = 7) -> tuple[np.ndarray, np.ndarray]:
    """Random positions uniform in a ball and Gaussian velocities (n,3) each."""
    st = Stream(seed, stream)
    x = np.asarray(center, dtype=np.float64) + radius * st.unit_ball(n)
    v = speed * st.normal(3 * n).reshape(n, 3)
    return x, v


def uniform_between(lo: float, hi: float, n: int, seed: int, stream: int) -> np.ndarray:
    return lo + (hi - lo) * u01(seed, stream, n)


def log_uniform_int(lo: int, hi: int, n: int, seed: int, stream: int) -> np.ndarray:
    """Integers log-uniform in [lo, hi] (rounded)."""
    u = u01(seed, stream, n)
    return np.rint(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)


def sweep_systems(nsys: int = 256, seed: int = 0, nmin: int = 2048, nmax: int = 65536):
    """Parameter sweep of independent binaries: element count log-uniform in
    [nmin, nmax] (3/4 donor), q uniform in [0.1, 1], donor expansion rate
    uniform in [0.5, 2]e-5 r_L per step; one SplitMix64 stream per system."""
    n = log_uniform_int(nmin, nmax, nsys, seed, 21)
    q = uniform_between(0.1, 1.0, nsys, seed, 22)
    rate = uniform_between(0.5e-5, 2.0e-5, nsys, seed, 23)
    out = []
    for s in range(nsys):
        nd = int(round(0.75 * n[s]))
        out.append(dict(n_donor=nd, n_accretor=int(n[s]) - nd, q=float(q[s]), f_donor=0.9,
                        f_accretor=0.5, expand_rate=float(rate[s]), expand_steps=-1,
                        sigma_v=1e-3, seed=seed, stream=1000 + s))
    return out


def served_trace(nreq: int = 64, seed: int = 0, rate_hz: float = 20.0, nmin: int = 4096,
                 nmax: int = 262144, smin: int = 1000, smax: int = 20000, steps_div: int = 1):
    """Poisson arrivals (exponential gaps, mean 1/rate_hz), element count
    log-uniform in [nmin, nmax] (3/4 donor), steps uniform in [smin, smax]
    (divided by steps_div), q uniform in [0.1, 1], donor expansion rate
    uniform in [0.5, 2]e-5 r_L per step (the sweep's range)."""
    gaps = -np.log(1.0 - u01(seed, 31, nreq)) / rate_hz
    t = np.cumsum(gaps) - gaps[0]
    n = log_uniform_int(nmin, nmax, nreq, seed, 32)
    steps = smin + np.floor(u01(seed, 33, nreq) * (smax - smin + 1)).astype(np.int64)
    steps = np.maximum(1, steps // steps_div)
    q = uniform_between(0.1, 1.0, nreq, seed, 34)
    rate = uniform_between(0.5e-5, 2.0e-5, nreq, seed, 35)
    out = []
    for r in range(nreq):
        nd = int(round(0.75 * n[r]))
        out.append(dict(t_arrival=float(t[r]), nsteps=int(steps[r]),
                        desc=dict(n_donor=nd, n_accretor=int(n[r]) - nd, q=float(q[r]),
                                  f_donor=0.9, f_accretor=0.5, expand_rate=float(rate[r]),
                                  expand_steps=-1, sigma_v=1e-3, seed=seed,
                                  stream=5000 + r)))
    return out
