"""CPU reference oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package. It wraps ``oracle.c`` (plain C, double-double
arithmetic, OpenMP over patterns) through ctypes and shares no code with the
CUDA library.

What each function computes, and the passage it follows:

* ``build_B(U, r)``: B = U diag(tanh r) U^T (Sec. 2.3, W = U U^T, generalised to
  per-mode squeezing; reduces to tanh(r) W for identical r, which is Eq. ProOri's
  tanh^n factor since Haf is homogeneous of degree n/2).
* ``haf_pm(A)``: Hafnian by the perfect-matching sum (Eq. HafMatch), expanded
  along one index as in Appendix A.
* ``haf_subset(A)``: the 2^{n/2}-subset power-trace sum of Bjorklund, Gupt and
  Quesada (the O(n^3 2^{n/2}) method cited in Sec. 2.3), traces by repeated
  matrix products; also returns kappa = sum_S |f(X A_S)|.
* ``haf_subset_f64(A)``: the same sum in plain double precision.
* ``per_ryser(C)``: permanent by Ryser's formula.
* ``haf_repeated(B, reps)``: Hafnian of the matrix that repeats row and column j
  of B reps[j] times, as a sum over 0 <= nu_j <= reps[j] of
  prod_j (-1)^nu_j C(reps[j], nu_j) (x^T B x / 2)^{n/2}, x_j = reps[j] - 2 nu_j,
  divided by 2^n (n/2)! (the moment-extraction identity of Kan, 2008, "From
  moments of sum to moments of product", derived in the docstring below). Not
  in the paper: it is the collision path of the library (cost prod (reps+1)
  instead of 2^{n/2}). Plain Python, double-precision terms, exactly rounded
  sums (math.fsum); small cases only.
* ``prob(U, r, patterns)``: p(s) = |Haf(B_x)|^2 / (prod_j s_j! prod_i cosh r_i)
  (Eq. ProOri with per-mode r; W_x gather of Sec. 3.2).

Parity is pinned in ``tests/test_oracle_pins.py`` against closed forms, brute
force and textbook special cases; see that file for the list.
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-ffp-contract=off"]
    if platform.machine() in ("x86_64", "AMD64"):
        base.append("-mfma")  # hardware fma(); results are identical to libm's fma()
    tmp = _LIB + ".tmp.%d" % os.getpid()
    for extra in (["-fopenmp"], []):
        cmd = base + extra + ["-o", tmp, _SRC, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _LIB)
            return _LIB
    raise RuntimeError("oracle build failed: " + r.stderr)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lp = ctypes.POINTER(ctypes.c_long)
            lib.orc_build_B.argtypes = [ctypes.c_int, dp, dp, dp]
            lib.orc_haf_pm.argtypes = [ctypes.c_int, dp, dp]
            lib.orc_haf_subset.argtypes = [ctypes.c_int, dp, dp, dp]
            lib.orc_haf_subset_f64.argtypes = [ctypes.c_int, dp, dp]
            lib.orc_per_ryser.argtypes = [ctypes.c_int, dp, dp]
            lib.orc_prob.argtypes = [ctypes.c_int, dp, ip, ip, lp, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
            lib.orc_haf_batch_f64.argtypes = [dp, ip, lp, ctypes.c_int, dp]
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_set_num_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _cplx(A) -> np.ndarray:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.complex128))
    return A.view(np.float64).reshape(-1).copy() if A.size else np.zeros(2)


def _dd_complex(out4) -> complex:
    return complex(out4[0] + out4[1], out4[2] + out4[3])


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(t: int) -> None:
    """Threads of the oracle's parallel loops over patterns (timing only)."""
    _load().orc_set_num_threads(int(t))


def build_B_dd(U, t) -> np.ndarray:
    """B = U diag(t) U^T in double-double: array (m, m, 4) of re.hi, re.lo, im.hi, im.lo."""
    U = np.asarray(U, dtype=np.complex128)
    m = U.shape[0]
    u = _cplx(U)
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float64))
    out = np.zeros(m * m * 4)
    _load().orc_build_B(m, _dp(u), _dp(t), _dp(out))
    return out.reshape(m, m, 4)


def build_B(U, r) -> np.ndarray:
    """B = U diag(tanh r) U^T rounded to complex128."""
    Bdd = build_B_dd(U, np.tanh(np.asarray(r, dtype=np.float64)))
    return (Bdd[..., 0] + Bdd[..., 1]) + 1j * (Bdd[..., 2] + Bdd[..., 3])


def haf_pm(A) -> complex:
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0] if A.ndim == 2 else 0
    out = np.zeros(4)
    _load().orc_haf_pm(n, _dp(_cplx(A)), _dp(out))
    return _dd_complex(out)


def haf_subset(A, return_kappa: bool = False):
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0] if A.ndim == 2 else 0
    out = np.zeros(4)
    k = np.zeros(1)
    _load().orc_haf_subset(n, _dp(_cplx(A)), _dp(out), _dp(k))
    h = _dd_complex(out)
    return (h, float(k[0])) if return_kappa else h


def haf_subset_dd_parts(A) -> np.ndarray:
    """The dd result unrounded: (re.hi, re.lo, im.hi, im.lo)."""
    A = np.asarray(A, dtype=np.complex128)
    out = np.zeros(4)
    k = np.zeros(1)
    _load().orc_haf_subset(A.shape[0], _dp(_cplx(A)), _dp(out), _dp(k))
    return out


def haf_subset_f64(A) -> complex:
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0] if A.ndim == 2 else 0
    out = np.zeros(2)
    _load().orc_haf_subset_f64(n, _dp(_cplx(A)), _dp(out))
    return complex(out[0], out[1])


def haf_batch_f64(mats) -> np.ndarray:
    """FP64 subset sums of a list of square complex matrices (OpenMP over matrices)."""
    ns = np.array([m.shape[0] for m in mats], dtype=np.int32)
    offs = np.zeros(len(mats), dtype=np.int64)
    if len(mats) > 1:
        offs[1:] = np.cumsum(ns.astype(np.int64) ** 2)[:-1]
    flat = np.concatenate([_cplx(m) for m in mats]) if mats else np.zeros(2)
    out = np.zeros(2 * len(mats))
    _load().orc_haf_batch_f64(_dp(flat), ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                              offs.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), len(mats), _dp(out))
    return out[0::2] + 1j * out[1::2]


def per_ryser(C) -> complex:
    C = np.asarray(C, dtype=np.complex128)
    k = C.shape[0] if C.ndim == 2 else 0
    out = np.zeros(4)
    _load().orc_per_ryser(k, _dp(_cplx(C)), _dp(out))
    return _dd_complex(out)


def haf_repeated(B, reps):
    """Hafnian of B with row/column j repeated reps[j] times (n = sum reps).

    Derivation. With Q(z) = z^T A z / 2 for the n x n repeated matrix A, the
    coefficient of z_1 z_2 ... z_n in Q(z)^{n/2} / (n/2)! is Haf(A): each way of
    picking one entry A_ij z_i z_j (i != j) from each of the n/2 factors so that
    every variable appears once is a perfect matching, counted (n/2)! times over
    the factor order and once per orientation (the 1/2 of Q cancels the two
    orientations); diagonal entries give z_i^2 and never reach that monomial.
    For a homogeneous polynomial P of degree n, sum over s in {+1, -1}^n of
    (prod s_i) P(s) keeps exactly the monomials odd in every variable, i.e.
    2^n times the coefficient of z_1 ... z_n. At a sign vector, Q depends only on
    x_j = (sum of the signs of mode j's copies) = reps[j] - 2 nu_j, nu_j the
    number of minus signs among them, which C(reps[j], nu_j) sign vectors share,
    each with prod s_i = (-1)^nu_j.
    """
    B = np.asarray(B, dtype=np.complex128)
    reps = [int(v) for v in reps]
    n = sum(reps)
    if n % 2:
        return 0j
    h = n // 2
    re, im = [], []
    for nu in itertools.product(*[range(v + 1) for v in reps]):
        x = np.array([reps[j] - 2 * nu[j] for j in range(len(reps))], dtype=np.float64)
        w = 1
        for j, v in enumerate(reps):
            w *= (-1) ** nu[j] * math.comb(v, nu[j])
        t = w * (0.5 * (x @ B @ x)) ** h
        re.append(t.real)
        im.append(t.imag)
    scale = 2.0 ** n * math.factorial(h)
    return complex(math.fsum(re) / scale, math.fsum(im) / scale)


def log_norm(r) -> float:
    """sum_i log cosh r_i (the prod_i cosh r_i of Eq. ProOri, in log form)."""
    return float(np.sum(np.log(np.cosh(np.asarray(r, dtype=np.float64)))))


def prob(U, r, patterns, method: str = "subset", Bdd=None, zero_diag: bool = False) -> dict:
    """Output probabilities of index-list patterns (in any order, Appendix B).

    The subset sum pairs positions (2t, 2t+1) of each list as given; with
    zero_diag the diagonal of W_x is set to 0 first (no perfect matching uses
    it, Eq. HafMatch). Neither changes Haf or p; both change the individual
    subset terms and so kappa. Returns dict with arrays p, logp, haf
    (complex128, the dd value rounded), haf_dd (batch, 4) and kappa (sum_S |f|;
    subset method only)."""
    if Bdd is None:
        Bdd = build_B_dd(U, np.tanh(np.asarray(r, dtype=np.float64)))
    m = Bdd.shape[0]
    pats = [np.asarray(p, dtype=np.int32) for p in patterns]
    ns = np.array([len(p) for p in pats], dtype=np.int32)
    offs = np.zeros(len(pats), dtype=np.int64)
    if len(pats) > 1:
        offs[1:] = np.cumsum(ns.astype(np.int64))[:-1]
    idx = np.concatenate(pats).astype(np.int32) if len(pats) and ns.sum() else np.zeros(1, np.int32)
    B = np.ascontiguousarray(Bdd.reshape(-1))
    nb = len(pats)
    p = np.zeros(nb); lp = np.zeros(nb); hd = np.zeros(4 * nb); kap = np.zeros(nb)
    _load().orc_prob(m, _dp(B), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                     ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                     offs.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), nb, log_norm(r),
                     1 if method == "pm" else 0, 1 if zero_diag else 0, _dp(p), _dp(lp), _dp(hd),
                     _dp(kap))
    hd = hd.reshape(nb, 4)
    return dict(p=p, logp=lp, haf=(hd[:, 0] + hd[:, 1]) + 1j * (hd[:, 2] + hd[:, 3]),
                haf_dd=hd, kappa=kap)
