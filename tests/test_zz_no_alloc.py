"""The no-allocation Hafnian entry point, through the C ABI (GPU only).

gbs_hafnian_batch_noalloc serves callers that cannot allocate memory while they
run; it takes its working space from a fixed array inside the library. This
file is collected after the other test files, so a run that stops at the first
failure has already run everything else; it also passes on its own in a fresh
process, where its first call does the one-time per-device set-up.

Each call is checked against gbs_hafnian_batch on the same inputs, with the
FP64 tolerance of the other parity tests, for two calls in a row (the second
reuses the array the first one left behind).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def rand_sym(n, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return scale * (A + A.T) / 2


def test_noalloc_matches_allocating_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_10070_gb300 as gbs

    for call, seed in enumerate((11, 12)):
        mats = [rand_sym(n, seed * 100 + n) for n in (0, 2, 3, 4, 7, 10, 16, 20, 24)]
        flat, n, offs = gbs.pack_matrices(mats)
        A = torch.from_numpy(flat).cuda()
        b = len(mats)
        ref = torch.zeros(2 * b, dtype=torch.float64, device="cuda")
        refk = torch.zeros(b, dtype=torch.float64, device="cuda")
        gbs.hafnian_batch(A, n, offs, gbs.FP64, haf_out=ref, kappa_out=refk)
        got = torch.full((2 * b,), float("nan"), dtype=torch.float64, device="cuda")
        gotk = torch.full((b,), float("nan"), dtype=torch.float64, device="cuda")
        gbs.hafnian_batch_noalloc(A, n, offs, gbs.FP64, haf_out=got, kappa_out=gotk)
        torch.cuda.synchronize()
        r = ref.cpu().numpy()
        g = got.cpu().numpy()
        hr = r[0::2] + 1j * r[1::2]
        hg = g[0::2] + 1j * g[1::2]
        rel = np.abs(hg - hr) / np.maximum(np.abs(hr), 1e-300)
        assert np.all(rel <= FP64_TOL), (call, rel)
        assert np.allclose(gotk.cpu().numpy(), refk.cpu().numpy(), rtol=FP64_TOL, atol=0)


def test_noalloc_rejects_oversized_batch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_10070_gb300 as gbs

    flat, n, offs = gbs.pack_matrices([np.eye(2)] * 1025)
    A = torch.from_numpy(flat).cuda()
    out = torch.zeros(2 * 1025, dtype=torch.float64, device="cuda")
    with pytest.raises(gbs.GbsError) as ei:
        gbs.hafnian_batch_noalloc(A, n, offs, gbs.FP64, haf_out=out)
    assert ei.value.code == -3 and "1024" in str(ei.value)


def test_noalloc_mixed_precision_against_oracle(orc):
    """GBS_MIXED through the no-allocation entry point: with no float copy of
    the inputs (the entry point holds none), the float kernel reads the double
    matrices itself. Two calls in a row; each result within the mixed path's
    stated bound min(n, 4) 2^-24 kappa of the double-double oracle, and of the
    allocating entry point's mixed result."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_10070_gb300 as gbs

    for call, seed in enumerate((21, 22)):
        mats = [rand_sym(n, seed * 100 + n) for n in (2, 4, 7, 10, 16, 20, 24)]
        flat, n, offs = gbs.pack_matrices(mats)
        A = torch.from_numpy(flat).cuda()
        b = len(mats)
        ref = torch.zeros(2 * b, dtype=torch.float64, device="cuda")
        refk = torch.zeros(b, dtype=torch.float64, device="cuda")
        gbs.hafnian_batch(A, n, offs, gbs.MIXED, haf_out=ref, kappa_out=refk)
        got = torch.full((2 * b,), float("nan"), dtype=torch.float64, device="cuda")
        gotk = torch.full((b,), float("nan"), dtype=torch.float64, device="cuda")
        gbs.hafnian_batch_noalloc(A, n, offs, gbs.MIXED, haf_out=got, kappa_out=gotk)
        torch.cuda.synchronize()
        r = ref.cpu().numpy()
        g = got.cpu().numpy()
        hr = r[0::2] + 1j * r[1::2]
        hg = g[0::2] + 1j * g[1::2]
        kg = gotk.cpu().numpy()
        kr = refk.cpu().numpy()
        for i, A_ in enumerate(mats):
            nn = A_.shape[0]
            if nn % 2:
                assert hg[i] == 0
                continue
            exact = orc.haf_subset(A_)
            bound = min(nn, 4) * 2.0 ** -24 * kg[i]
            assert abs(hg[i] - exact) <= bound * abs(exact), (call, nn, abs(hg[i] - exact) / abs(exact), bound)
            assert abs(hg[i] - hr[i]) <= (bound + min(nn, 4) * 2.0 ** -24 * kr[i]) * abs(exact)


def test_noalloc_rejects_too_many_work_items():
    """1024 matrices of order 24 need more than the 16384 work items the fixed
    array holds: GBS_ERANGE with the reason, and nothing launched."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_10070_gb300 as gbs

    flat, n, offs = gbs.pack_matrices([np.eye(24)] * 1024)
    A = torch.from_numpy(flat).cuda()
    out = torch.zeros(2 * 1024, dtype=torch.float64, device="cuda")
    with pytest.raises(gbs.GbsError) as ei:
        gbs.hafnian_batch_noalloc(A, n, offs, gbs.FP64, haf_out=out)
    assert ei.value.code == -3 and "16384" in str(ei.value)
