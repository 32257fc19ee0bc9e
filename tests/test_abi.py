"""The C ABI library builds, loads and exports every entry point include/gbs.h declares
(no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gbs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gbs_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("gbs_build_kernel", "gbs_hafnian_batch", "gbs_prob_batch", "gbs_serve_create",
                 "gbs_serve_submit", "gbs_serve_poll", "gbs_serve_destroy", "gbs_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1908_10070_gb300 import build

    lib = ctypes.CDLL(build.build())
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_last_error_starts_empty():
    """The last-error message is per thread: a thread that has made no call
    reads an empty string, whatever other threads (or tests) did before."""
    import threading

    from paper_1908_10070_gb300 import build

    lib = ctypes.CDLL(build.build())
    lib.gbs_last_error.restype = ctypes.c_char_p
    seen = []
    t = threading.Thread(target=lambda: seen.append(lib.gbs_last_error()))
    t.start()
    t.join()
    assert seen == [b""]


def test_argument_errors_without_device():
    """Checks that fail before any CUDA call return codes, not crashes."""
    from paper_1908_10070_gb300 import build

    lib = ctypes.CDLL(build.build())
    lib.gbs_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    assert lib.gbs_build_kernel(None, None, 4, None, ctypes.byref(out)) == -1
    assert b"null" in lib.gbs_last_error()
    assert lib.gbs_hafnian_batch(None, None, None, -1, 0, None, None, None) == -1
    assert lib.gbs_prob_batch(None, None, None, None, 1, 0, None, None, None, None, None) == -1
    assert lib.gbs_serve_create(None, None, ctypes.byref(out)) == -1
    assert lib.gbs_serve_destroy(None) == 0
    assert lib.gbs_free_kernel(None) == 0


def test_sampler_argument_errors_without_device():
    """The sampler entry points check their arguments before any CUDA call."""
    from paper_1908_10070_gb300 import build

    lib = ctypes.CDLL(build.build())
    lib.gbs_last_error.restype = ctypes.c_char_p
    i = ctypes.c_int()
    assert lib.gbs_sample_chain(None, 4, None, None, None) == -1
    assert b"null" in lib.gbs_last_error()
    assert lib.gbs_sample_chain_batch(None, 4, 2, None, None, None) == -1
    assert lib.gbs_sample(None, 4, None, None, ctypes.byref(i), None) == -1
    assert lib.gbs_sample_batch(None, 4, 2, None, None, None, None) == -1
    assert lib.gbs_marginal_batch(None, None, 2, 1, 4, None, None) == -1
