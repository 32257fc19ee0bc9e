"""Kept batch plans (gbs_prob_batch / gbs_hafnian_batch with a repeated shape).

A call whose n[], offs[], m, precision and launch shape match an earlier call
reuses that call's plan block (work items, descriptors, ordering-probe tables)
from device memory. The plan never depends on the index lists or matrices, so
a call through a kept plan must give the same bits as the same call planned
afresh (after gbs_clear_plans), for new inputs of the same shape, from host or
device inputs, on other streams, and after other shapes have evicted it.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gbs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_10070_gb300 as g

    g.lib()
    return g


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def kernel(gbs, m, seed, r=0.8):
    U = W.haar_unitary(m, seed)
    return gbs.build_kernel(dev(np.ascontiguousarray(U).view(np.float64)), dev(np.full(m, r)))


def probs(gbs, K, idx, n, offs, precision, host=False, stream=None):
    b = len(n)
    if host:
        hf = np.zeros(2 * b)
        er = np.zeros(b)
        gbs.prob_batch(K, idx, n, offs, precision, haf_out=hf, err_out=er, stream=stream)
        return hf, er
    hf = torch.zeros(2 * b, dtype=torch.float64, device="cuda")
    er = torch.zeros(b, dtype=torch.float64, device="cuda")
    gbs.prob_batch(K, dev(idx), n, offs, precision, haf_out=hf, err_out=er, stream=stream)
    torch.cuda.synchronize()
    return hf.cpu().numpy(), er.cpu().numpy()


def fresh(gbs, fn):
    gbs.clear_plans()
    return fn()


def mixed_batch(m, seed, count=96):
    """Orders 2..32 with repeated modes in some lists (both routes)."""
    rng = np.random.default_rng(seed)
    pats = []
    for i in range(count):
        n = 2 * (1 + i % 16)
        if i % 7 == 3:
            pats.append(np.sort(rng.integers(0, 3, size=n)).astype(np.int32))  # bunched
        else:
            pats.append(rng.integers(0, m, size=n).astype(np.int32))
    return pats


@pytest.mark.parametrize("precision", [0, 1])
def test_kept_plan_gives_fresh_bits_for_new_inputs(gbs, precision):
    m = 40
    K = kernel(gbs, m, 17)
    shape = None
    for seed in (1, 2, 3):
        idx, n, offs = gbs.pack_patterns(mixed_batch(m, seed))
        if shape is None:
            shape = (n.copy(), offs.copy())
        assert np.array_equal(n, shape[0]) and np.array_equal(offs, shape[1])
        kept = probs(gbs, K, idx, n, offs, precision)  # plan of seed 1, kept
        ref = fresh(gbs, lambda: probs(gbs, K, idx, n, offs, precision))
        assert np.array_equal(kept[0], ref[0]) and np.array_equal(kept[1], ref[1]), seed
        host = probs(gbs, K, idx, n, offs, precision, host=True)
        assert np.array_equal(host[0], ref[0]) and np.array_equal(host[1], ref[1]), seed


def test_kept_plan_with_ordering_probe(gbs):
    """n = 28 and 30: the probe's choice is made per call (in the call's own
    scratch); a kept plan with other matrices still probes them afresh."""
    m = 96
    K = kernel(gbs, m, 5, r=0.7)
    rng = np.random.default_rng(8)
    for rep in range(3):
        pats = [rng.permutation(m)[:28].astype(np.int32), rng.permutation(m)[:30].astype(np.int32),
                rng.permutation(m)[:16].astype(np.int32)]
        idx, n, offs = gbs.pack_patterns(pats)
        kept = probs(gbs, K, idx, n, offs, 0)
        ref = fresh(gbs, lambda: probs(gbs, K, idx, n, offs, 0))
        assert np.array_equal(kept[0], ref[0]), rep


def test_kept_plan_on_other_streams(gbs):
    """Calls of one shape alternate between two streams; each reads the plan
    uploaded by the first (ordered after its upload by an event)."""
    m = 48
    K = kernel(gbs, m, 21)
    gbs.clear_plans()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    batches = [gbs.pack_patterns(mixed_batch(m, 40 + i, count=64)) for i in range(4)]
    for i, (idx, n, offs) in enumerate(batches):
        st = s1 if i % 2 == 0 else s2
        hf = torch.zeros(2 * len(n), dtype=torch.float64, device="cuda")
        with torch.cuda.stream(st):
            d_idx = dev(idx)
            gbs.prob_batch(K, d_idx, n, offs, 0, haf_out=hf, stream=st)
        outs.append((st, hf, d_idx))
    torch.cuda.synchronize()
    for (idx, n, offs), (_, hf, _) in zip(batches, outs):
        ref = fresh(gbs, lambda: probs(gbs, K, idx, n, offs, 0))
        assert np.array_equal(hf.cpu().numpy(), ref[0])


def test_kept_plans_evicted_and_rebuilt(gbs):
    """More shapes than the library keeps: the oldest are evicted (freed after
    the device is idle) and planned again when they return, same bits."""
    m = 32
    K = kernel(gbs, m, 3)
    gbs.clear_plans()
    rng = np.random.default_rng(2)
    shapes = []
    for s in range(12):
        pats = [rng.integers(0, m, size=2 * (1 + (s + j) % 12)).astype(np.int32) for j in range(s + 1)]
        shapes.append(gbs.pack_patterns(pats))
    first = [probs(gbs, K, *sh, 0)[0] for sh in shapes]
    again = [probs(gbs, K, *sh, 0)[0] for sh in shapes]
    for a, b in zip(first, again):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_kept_plan_hafnian_batch(gbs, precision):
    """Explicit matrices of one shape, new values each call, host and device."""
    rng = np.random.default_rng(12)
    sizes = [4, 10, 16, 22, 8, 16]
    for rep in range(3):
        mats = []
        for v in sizes:
            A = rng.standard_normal((v, v)) + 1j * rng.standard_normal((v, v))
            mats.append((A + A.T) / 2)
        flat, n, offs = gbs.pack_matrices(mats)
        out = torch.zeros(2 * len(n), dtype=torch.float64, device="cuda")
        gbs.hafnian_batch(dev(flat), n, offs, precision, haf_out=out)
        torch.cuda.synchronize()
        kept = out.cpu().numpy()
        gbs.clear_plans()
        host = np.zeros(2 * len(n))
        gbs.hafnian_batch(flat, n, offs, precision, haf_out=host)
        assert np.array_equal(kept, host), rep


def test_kept_plan_still_checks_host_lists(gbs):
    """A host index list is range-checked on every call, also when the call's
    shape has a kept plan (GBS_ERANGE, nothing launched); the next valid call
    of that shape still gives the fresh plan's bits."""
    m = 24
    K = kernel(gbs, m, 4)
    idx, n, offs = gbs.pack_patterns(mixed_batch(m, 9, count=40))
    good = probs(gbs, K, idx, n, offs, 0, host=True)  # plans and keeps the shape
    bad = idx.copy()
    bad[int(offs[7])] = m  # one index past the last mode
    with pytest.raises(gbs.GbsError) as ei:
        probs(gbs, K, bad, n, offs, 0, host=True)
    assert ei.value.code == -3
    again = probs(gbs, K, idx, n, offs, 0, host=True)
    assert np.array_equal(good[0], again[0]) and np.array_equal(good[1], again[1])
    gbs.clear_plans()
    gbs.clear_plans()  # nothing kept: still fine
