"""Python binding of the GB300 Gaussian-boson-sampling probability library.

Argument marshalling only: every function forwards to the C ABI declared in
``include/gbs.h`` (same names without the ``gbs_`` prefix), which runs every
step of the computation in the library's CUDA kernels. Device buffers are
torch tensors (or any object with ``data_ptr()``); host buffers may be numpy
arrays. There is no CPU fallback: importing this module on a machine where the
library cannot be built or loaded raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = [
    "FP64", "MIXED", "MAX_N", "GbsError", "lib", "build_kernel", "KernelMatrix",
    "hafnian_batch", "hafnian_batch_noalloc", "prob_batch", "autotune", "measure_fp64_peak", "Server", "serve_create", "pack_patterns",
    "pack_matrices", "last_error", "ERRORS", "photon_number_dist", "sample_bruteforce", "marginal_batch", "sample_chain",
    "sample_chain_batch", "sample", "sample_batch", "clear_plans",
]

FP64 = 0
MIXED = 1
MAX_N = 32
ERRORS = {0: "GBS_OK", -1: "GBS_EINVAL", -2: "GBS_ENOMEM", -3: "GBS_ERANGE", -4: "GBS_EAGAIN",
          -5: "GBS_ETIMEDOUT", -6: "GBS_ECUDA", -7: "GBS_ENOENT", -8: "GBS_ECANCELED"}

_lock = threading.Lock()
_lib = None


class GbsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class ServeStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("items", ctypes.c_int64), ("subsets", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("step_wall_s", ctypes.c_double),
                ("step_wall_max_s", ctypes.c_double), ("step_device_s", ctypes.c_double),
                ("step_device_max_s", ctypes.c_double), ("poll_gap_max_s", ctypes.c_double),
                ("launch_max_s", ctypes.c_double), ("update_max_s", ctypes.c_double),
                ("submit_max_s", ctypes.c_double), ("probed", ctypes.c_int64),
                ("cancelled", ctypes.c_int64), ("alloc_waits", ctypes.c_int64),
                ("arena_slots", ctypes.c_int64)]


class ServeOpts(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("mem_budget", ctypes.c_size_t),
                ("queue_capacity", ctypes.c_int), ("subsets_per_step", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("wait_timeout_s", ctypes.c_double),
                ("max_n", ctypes.c_int), ("fault_alloc_failures", ctypes.c_int)]


def lib():
    """Load (building first if needed) the in-tree libgbs.so."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            vp, dp, ip, i64p = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
            L.gbs_build_kernel.argtypes = [dp, dp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_void_p)]
            L.gbs_free_kernel.argtypes = [vp]
            L.gbs_kernel_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
            L.gbs_kernel_copy_B.argtypes = [vp, dp, vp]
            L.gbs_hafnian_batch.argtypes = [dp, ip, i64p, ctypes.c_int, ctypes.c_int, vp, dp, dp]
            L.gbs_hafnian_batch_noalloc.argtypes = [dp, ip, i64p, ctypes.c_int, ctypes.c_int, vp, dp, dp]
            L.gbs_prob_batch.argtypes = [vp, ip, ip, i64p, ctypes.c_int, ctypes.c_int, vp, dp, dp, dp, dp]
            L.gbs_photon_number_dist.argtypes = [vp, ctypes.c_int, vp, dp]
            L.gbs_sample_bruteforce.argtypes = [vp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, vp, ip, dp]
            L.gbs_marginal_batch.argtypes = [vp, ip, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, dp]
            L.gbs_sample_chain.argtypes = [vp, ctypes.c_int, dp, vp, ip]
            L.gbs_sample_chain_batch.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, vp, ip]
            L.gbs_sample.argtypes = [vp, ctypes.c_int, dp, vp, ctypes.POINTER(ctypes.c_int), ip]
            L.gbs_sample_batch.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, vp, ip, ip]
            L.gbs_autotune.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int)]
            L.gbs_measure_fp64_peak.argtypes = [vp, dp]
            L.gbs_set_timing_events.argtypes = [vp, vp]
            L.gbs_clear_plans.argtypes = []
            L.gbs_serve_create.argtypes = [vp, ctypes.POINTER(ServeOpts), ctypes.POINTER(ctypes.c_void_p)]
            L.gbs_serve_submit.argtypes = [vp, ip, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
            L.gbs_serve_poll.argtypes = [vp, ctypes.c_int64, dp, dp, dp]
            L.gbs_serve_cancel.argtypes = [vp, ctypes.c_int64]
            L.gbs_serve_wait_any.argtypes = [vp, ctypes.c_double, ctypes.c_int, vp, dp, dp, dp, ip,
                                             ctypes.POINTER(ctypes.c_int)]
            L.gbs_serve_destroy.argtypes = [vp]
            L.gbs_serve_stats.argtypes = [vp, ctypes.POINTER(ServeStats)]
            L.gbs_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def last_error() -> str:
    return lib().gbs_last_error().decode()


def _check(rc):
    if rc != 0:
        raise GbsError(rc, last_error())
    return rc


def _ptr(x):
    """Address (int, or None) of a torch tensor / numpy array / None; the
    c_void_p arguments take plain ints."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr() or None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy array must be C-contiguous")
        return x.ctypes.data or None
    raise TypeError("unsupported buffer type %r" % type(x))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream or None
    return int(stream) or None


def pack_patterns(patterns):
    """List of index lists -> (idx int32, n int32, offs int64) numpy arrays."""
    pats = [np.asarray(p, dtype=np.int32).reshape(-1) for p in patterns]
    n = np.array([len(p) for p in pats], dtype=np.int32)
    offs = np.zeros(len(pats), dtype=np.int64)
    if len(pats) > 1:
        offs[1:] = np.cumsum(n.astype(np.int64))[:-1]
    idx = np.concatenate(pats).astype(np.int32) if len(pats) and n.sum() else np.zeros(1, np.int32)
    return np.ascontiguousarray(idx), n, offs


def pack_matrices(mats):
    """List of square complex matrices -> (flat float64 interleaved, n, offs)."""
    ms = [np.ascontiguousarray(np.asarray(m, dtype=np.complex128)) for m in mats]
    n = np.array([m.shape[0] for m in ms], dtype=np.int32)
    offs = np.zeros(len(ms), dtype=np.int64)
    if len(ms) > 1:
        offs[1:] = np.cumsum(n.astype(np.int64) ** 2)[:-1]
    flat = np.concatenate([m.reshape(-1).view(np.float64) for m in ms]) if ms and n.sum() else np.zeros(2)
    return np.ascontiguousarray(flat), n, offs


class KernelMatrix:
    """Owner of a gbs_kernel handle (B = U diag(tanh r) U^T resident on the device)."""

    def __init__(self, handle, m):
        self.handle = handle
        self.m = m

    @property
    def log_norm(self) -> float:
        v = ctypes.c_double()
        _check(lib().gbs_kernel_info(self.handle, None, ctypes.byref(v)))
        return v.value

    def copy_B(self, dst, stream=None):
        _check(lib().gbs_kernel_copy_B(self.handle, _ptr(dst), _stream(stream)))
        return dst

    def free(self):
        if self.handle:
            _check(lib().gbs_free_kernel(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_kernel(U, r, stream=None) -> KernelMatrix:
    """U: m x m complex128 (torch tensor viewed as float64 pairs, or numpy); r: m doubles."""
    if isinstance(U, np.ndarray):
        U = np.ascontiguousarray(np.asarray(U, dtype=np.complex128)).view(np.float64)
        m = U.shape[0]
    else:
        m = U.shape[0]
    if isinstance(r, np.ndarray):
        r = np.ascontiguousarray(r, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(lib().gbs_build_kernel(_ptr(U), _ptr(r), int(m), _stream(stream), ctypes.byref(h)))
    return KernelMatrix(h, int(m))


def hafnian_batch(A, n, offs, precision=FP64, stream=None, haf_out=None, kappa_out=None):
    """Hafnians of packed matrices (see pack_matrices). n, offs: host arrays."""
    n = np.ascontiguousarray(n, dtype=np.int32)
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    _check(lib().gbs_hafnian_batch(_ptr(A), _ptr(n), _ptr(offs), len(n), int(precision),
                                   _stream(stream), _ptr(haf_out), _ptr(kappa_out)))
    return haf_out, kappa_out


def hafnian_batch_noalloc(A, n, offs, precision=FP64, stream=None, haf_out=None, kappa_out=None):
    """gbs_hafnian_batch_noalloc: same as hafnian_batch for callers that cannot
    allocate; A and the outputs must be device tensors. See include/gbs.h."""
    n = np.ascontiguousarray(n, dtype=np.int32)
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    _check(lib().gbs_hafnian_batch_noalloc(_ptr(A), _ptr(n), _ptr(offs), len(n), int(precision),
                                           _stream(stream), _ptr(haf_out), _ptr(kappa_out)))
    return haf_out, kappa_out


def prob_batch(kernel: KernelMatrix, idx, n, offs, precision=FP64, stream=None, p_out=None,
               logp_out=None, haf_out=None, err_out=None):
    """Output probabilities of packed index lists (see pack_patterns). n, offs: host arrays."""
    n = np.ascontiguousarray(n, dtype=np.int32)
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    _check(lib().gbs_prob_batch(kernel.handle, _ptr(idx), _ptr(n), _ptr(offs), len(n), int(precision),
                                _stream(stream), _ptr(p_out), _ptr(logp_out), _ptr(haf_out),
                                _ptr(err_out)))
    return p_out, logp_out, haf_out, err_out


def set_timing_events(start, stop):
    """Record torch.cuda.Event objects around each later subset-sum kernel (None, None = off)."""
    sp = ctypes.c_void_p(start.cuda_event) if start is not None else None
    tp = ctypes.c_void_p(stop.cuda_event) if stop is not None else None
    _check(lib().gbs_set_timing_events(sp, tp))


def clear_plans():
    """gbs_clear_plans: free the batch plans kept for repeated shapes."""
    _check(lib().gbs_clear_plans())


def photon_number_dist(kernel: KernelMatrix, n_max: int, stream=None) -> np.ndarray:
    """P_n for n = 0..n_max (gbs_photon_number_dist), as a host array."""
    out = np.zeros(n_max + 1)
    _check(lib().gbs_photon_number_dist(kernel.handle, int(n_max), _stream(stream), _ptr(out)))
    return out


def sample_bruteforce(kernel: KernelMatrix, n: int, uniforms, precision=FP64, stream=None):
    """Configurations with n photons drawn by gbs_sample_bruteforce from the given
    uniform numbers. Returns (patterns as a draws x n int32 array, total = P_n)."""
    u = np.ascontiguousarray(uniforms, dtype=np.float64)
    out = np.zeros((len(u), max(n, 1)), dtype=np.int32)
    tot = np.zeros(1)
    _check(lib().gbs_sample_bruteforce(kernel.handle, int(n), _ptr(u) if len(u) else None, len(u),
                                       int(precision), _stream(stream), _ptr(out), _ptr(tot)))
    return out[:, :n], float(tot[0])


def marginal_batch(kernel: KernelMatrix, prefixes, n: int, stream=None) -> np.ndarray:
    """q_n(x_1..x_k) for each row of `prefixes` (batch x k mode indices)."""
    x = np.ascontiguousarray(np.asarray(prefixes, dtype=np.int32).reshape(len(prefixes), -1))
    out = np.zeros(x.shape[0])
    _check(lib().gbs_marginal_batch(kernel.handle, _ptr(x) if x.size else None, int(x.shape[1]),
                                    int(x.shape[0]), int(n), _stream(stream), _ptr(out)))
    return out


def sample_chain(kernel: KernelMatrix, n: int, uniforms, stream=None) -> np.ndarray:
    """One position-basis sample x_1..x_n by Algorithm 1 (gbs_sample_chain)."""
    u = np.ascontiguousarray(uniforms, dtype=np.float64)
    x = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().gbs_sample_chain(kernel.handle, int(n), _ptr(u), _stream(stream), _ptr(x)))
    return x[:n]


def sample_chain_batch(kernel: KernelMatrix, n: int, uniforms, stream=None) -> np.ndarray:
    """Independent Algorithm 1 samples advanced together (gbs_sample_chain_batch).
    uniforms: (samples, n) numbers in [0, 1). Returns (samples, n) modes."""
    u = np.ascontiguousarray(uniforms, dtype=np.float64)
    S = u.shape[0] if u.ndim == 2 else 0
    if u.ndim != 2 or u.shape[1] != n:
        raise ValueError("uniforms must have shape (samples, n)")
    x = np.zeros((max(S, 1), max(n, 1)), dtype=np.int32)
    _check(lib().gbs_sample_chain_batch(kernel.handle, int(n), int(S), _ptr(u), _stream(stream), _ptr(x)))
    return x[:S, :n]


def sample(kernel: KernelMatrix, n_max: int, uniforms, stream=None) -> np.ndarray:
    """One complete sample (gbs_sample): n from P_n truncated at n_max, then
    Algorithm 1. uniforms: n_max + 1 numbers in [0, 1). Returns x_1..x_n."""
    u = np.ascontiguousarray(uniforms, dtype=np.float64)
    if u.size < n_max + 1:
        raise ValueError("need n_max + 1 uniform numbers")
    x = np.zeros(max(n_max, 1), dtype=np.int32)
    n = ctypes.c_int()
    _check(lib().gbs_sample(kernel.handle, int(n_max), _ptr(u), _stream(stream), ctypes.byref(n), _ptr(x)))
    return x[:n.value]


def sample_batch(kernel: KernelMatrix, n_max: int, uniforms, stream=None):
    """Complete samples at once (gbs_sample_batch). uniforms: (samples, n_max + 1)
    numbers in [0, 1). Returns a list of each sample's x_1..x_n."""
    u = np.ascontiguousarray(uniforms, dtype=np.float64)
    if u.ndim != 2 or u.shape[1] != n_max + 1:
        raise ValueError("uniforms must have shape (samples, n_max + 1)")
    S = u.shape[0]
    n = np.zeros(max(S, 1), dtype=np.int32)
    x = np.zeros((max(S, 1), max(n_max, 1)), dtype=np.int32)
    _check(lib().gbs_sample_batch(kernel.handle, int(n_max), int(S), _ptr(u), _stream(stream), _ptr(n), _ptr(x)))
    return [x[s, :n[s]].copy() for s in range(S)]


def measure_fp64_peak(stream=None) -> float:
    """gbs_measure_fp64_peak: the device's measured DFMA throughput, TFLOP/s."""
    v = ctypes.c_double()
    _check(lib().gbs_measure_fp64_peak(_stream(stream), ctypes.byref(v)))
    return v.value


def autotune(n, precision=FP64, stream=None) -> int:
    c = ctypes.c_int()
    _check(lib().gbs_autotune(int(n), int(precision), _stream(stream), ctypes.byref(c)))
    return c.value


class Server:
    """Continuous-batching server (gbs_serve_*)."""

    def __init__(self, kernel: KernelMatrix, max_slots=0, mem_budget=0, queue_capacity=0,
                 subsets_per_step=0, use_graphs=1, wait_timeout_s=0.0, max_n=0, fault_alloc_failures=0):
        self.kernel = kernel
        o = ServeOpts(max_slots, mem_budget, queue_capacity, subsets_per_step, use_graphs, wait_timeout_s,
                      max_n, fault_alloc_failures)
        h = ctypes.c_void_p()
        _check(lib().gbs_serve_create(kernel.handle, ctypes.byref(o), ctypes.byref(h)))
        self.handle = h

    def submit(self, x, precision=FP64) -> int:
        """Returns a ticket, or -1 when the queue is full (GBS_EAGAIN)."""
        x = np.ascontiguousarray(x, dtype=np.int32)
        t = ctypes.c_int64()
        rc = lib().gbs_serve_submit(self.handle, _ptr(x) if x.size else None, int(x.size),
                                    int(precision), ctypes.byref(t))
        if rc == -4:
            return -1
        _check(rc)
        return t.value

    def poll(self, ticket):
        """None while pending, else (p, haf complex, err_est)."""
        p = ctypes.c_double()
        hf = (ctypes.c_double * 2)()
        e = ctypes.c_double()
        rc = lib().gbs_serve_poll(self.handle, int(ticket), ctypes.byref(p), hf, ctypes.byref(e))
        if rc == 1:
            return None
        _check(rc)
        return p.value, complex(hf[0], hf[1]), e.value

    def wait_any(self, timeout_s=0.0, max_results=1024):
        """gbs_serve_wait_any: finished requests in any order, as numpy arrays
        (tickets, p, haf complex, err_est, rc); empty when none finished within
        timeout_s. A failed request has rc < 0 and NaN outputs."""
        if getattr(self, "_wa_cap", 0) < max_results:
            self._wa_cap = max_results
            self._wa = (np.zeros(max_results, np.int64), np.zeros(max_results), np.zeros(2 * max_results),
                        np.zeros(max_results), np.zeros(max_results, np.int32))
        t, p, hf, e, rc = self._wa
        cnt = ctypes.c_int()
        _check(lib().gbs_serve_wait_any(self.handle, float(timeout_s), int(max_results), _ptr(t), _ptr(p),
                                        _ptr(hf), _ptr(e), _ptr(rc), ctypes.byref(cnt)))
        k = cnt.value
        return t[:k].copy(), p[:k].copy(), hf[0:2 * k:2] + 1j * hf[1:2 * k:2], e[:k].copy(), rc[:k].copy()

    def cancel(self, ticket) -> int:
        """0: cancelled (its poll raises GBS_ECANCELED); 1: already finished."""
        rc = lib().gbs_serve_cancel(self.handle, int(ticket))
        if rc != 1:
            _check(rc)
        return rc

    def stats(self) -> dict:
        st = ServeStats()
        _check(lib().gbs_serve_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServeStats._fields_}

    def destroy(self):
        if self.handle:
            h, self.handle = self.handle, None  # freed even when destroy reports an error
            _check(lib().gbs_serve_destroy(h))

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def serve_create(kernel, **opts) -> Server:
    return Server(kernel, **opts)
