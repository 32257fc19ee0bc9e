"""Seeded synthetic inputs for Gaussian-boson-sampling probability workloads.

This module is shared by the tests, the benchmark and the oracle checks. It only
draws random numbers and lays them out; it holds none of the Hafnian or
probability arithmetic.

Interferometer: a Haar-random m x m unitary. The paper does not say how its
unitaries were drawn; the recipe used here is the standard one for sampling the
Haar measure: a complex Ginibre matrix (i.i.d. N(0,1/2) + i N(0,1/2) entries),
a QR factorisation, and a phase fix U = Q diag(R_ii / |R_ii|).

Output patterns: mode-index lists x = (x_1, ..., x_n), 0-based, sorted, where a
repeated index is a photon collision in that mode (the position-basis form of a
configuration s, Sec. 3.2 "Step 2: change of basis").
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "haar_unitary",
    "squeezing",
    "collision_free_patterns",
    "collision_patterns",
    "all_patterns",
    "pattern_to_counts",
    "poisson_arrivals",
    "serving_requests",
    "WORKLOADS",
    "workload",
]


def haar_unitary(m: int, seed: int) -> np.ndarray:
    """Haar-random m x m unitary (complex128) from a seeded Ginibre draw."""
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    ph = d / np.abs(d)
    return np.ascontiguousarray(q * ph[None, :])


def squeezing(m: int, kind: str, seed: int = 0, value: float = 0.5,
              lo: float = 0.6, hi: float = 1.0) -> np.ndarray:
    """Per-mode squeezing parameters r_i: identical ('const') or U[lo, hi]."""
    if kind == "const":
        return np.full(m, float(value))
    if kind == "uniform":
        rng = np.random.default_rng(seed)
        return rng.uniform(lo, hi, size=m)
    raise ValueError(kind)


def collision_free_patterns(m: int, n: int, count: int, seed: int) -> np.ndarray:
    """count patterns of n distinct modes drawn uniformly without replacement."""
    rng = np.random.default_rng(seed)
    out = np.empty((count, n), dtype=np.int32)
    for b in range(count):
        out[b] = np.sort(rng.choice(m, size=n, replace=False))
    return out


def collision_patterns(m: int, n_values, count: int, seed: int,
                       max_per_mode: int = 3) -> list:
    """count patterns with n drawn uniformly from n_values; n modes drawn
    uniformly with replacement, redrawn while any mode holds > max_per_mode."""
    rng = np.random.default_rng(seed)
    n_values = list(n_values)
    pats = []
    for _ in range(count):
        n = int(n_values[rng.integers(len(n_values))])
        while True:
            x = rng.integers(0, m, size=n)
            if n == 0 or np.bincount(x, minlength=m).max() <= max_per_mode:
                break
        pats.append(np.sort(x).astype(np.int32))
    return pats


def all_patterns(m: int, n: int) -> list:
    """Every configuration with n photons in m modes, as sorted index lists
    (the C(m+n-1, n) multisets), in lexicographic order."""
    out = []

    def rec(start, cur):
        if len(cur) == n:
            out.append(np.array(cur, dtype=np.int32))
            return
        for j in range(start, m):
            cur.append(j)
            rec(j, cur)
            cur.pop()

    rec(0, [])
    return out


def pattern_to_counts(x, m: int) -> np.ndarray:
    """Index list x -> occupation numbers s (length m)."""
    return np.bincount(np.asarray(x, dtype=np.int64), minlength=m)


def poisson_arrivals(rate_hz: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative seeded exponential gaps."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=count))


# The workloads the library is measured and checked on. Sizes follow the
# paper's setting of Haar-random interferometers with every mode squeezed
# (Sec. 2); the paper itself ran m = n^2 with identical r (Sec. 3.5).
WORKLOADS = {
    "tiny_m8": dict(m=8, seed=0, r=("const", 0.5)),
    "batched_m64_n16": dict(m=64, seed=1, r=("uniform", 0.6, 1.0), n=16, count=4096),
    "mixed_m144": dict(m=144, seed=2, r=("const", 0.88), n_values=tuple(range(8, 25, 2)),
                       count=2048, max_per_mode=3),
    "serving_m256": dict(m=256, seed=3, r=("const", 0.88), n_values=tuple(range(12, 27)),
                         rate_hz=2000.0),
    "large_m900": dict(m=900, seed=4, r=("const", 1.0), n28=64, n30=16),
    # photons bunched into few modes (a small interferometer, many photons):
    # the regime of the repeated-row route
    "bunched_m8": dict(m=8, seed=5, r=("const", 1.0), n=24, count=512),
}


def workload(name: str):
    """Return (U, r, patterns) for a named workload (patterns: list of int32 arrays)."""
    w = WORKLOADS[name]
    m, seed = w["m"], w["seed"]
    U = haar_unitary(m, seed)
    if w["r"][0] == "const":
        r = squeezing(m, "const", value=w["r"][1])
    else:
        r = squeezing(m, "uniform", seed=seed, lo=w["r"][1], hi=w["r"][2])
    if name == "tiny_m8":
        pats = [np.array(c, dtype=np.int32) for c in _combinations(m, 4)]
        pats += all_patterns(m, 2)
    elif name == "batched_m64_n16":
        pats = list(collision_free_patterns(m, w["n"], w["count"], seed + 100))
    elif name == "mixed_m144":
        pats = collision_patterns(m, w["n_values"], w["count"], seed + 100, w["max_per_mode"])
    elif name == "serving_m256":
        pats = []  # requests are drawn by the serving driver (serving_requests)
    elif name == "large_m900":
        pats = list(collision_free_patterns(m, 28, w["n28"], seed + 100))
        pats += list(collision_free_patterns(m, 30, w["n30"], seed + 200))
    elif name == "bunched_m8":
        rng = np.random.default_rng(seed + 100)
        pats = [np.sort(rng.choice(m, w["n"], replace=True)).astype(np.int32) for _ in range(w["count"])]
    else:
        raise KeyError(name)
    return U, r, pats


def serving_requests(count: int, seed: int = 3, rate_hz: float = None):
    """Request stream of the serving workload: (arrival_s, index list) pairs,
    n ~ Uniform{12..26}, collision-free, Poisson arrivals at 2000 req/s (or
    rate_hz; the same lists in the same order at every rate)."""
    w = WORKLOADS["serving_m256"]
    rng = np.random.default_rng(seed + 300)
    t = poisson_arrivals(rate_hz or w["rate_hz"], count, seed + 400)
    reqs = []
    for i in range(count):
        n = int(rng.integers(12, 27))
        x = np.sort(rng.choice(w["m"], size=n, replace=False)).astype(np.int32)
        reqs.append((float(t[i]), x))
    return reqs


def _combinations(m, k):
    import itertools
    return list(itertools.combinations(range(m), k))
