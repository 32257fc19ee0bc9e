"""CUDA path vs the CPU oracle, through the C ABI (GPU only).

FP64 path: relative error of Haf and p within 1e-10 of the double-double oracle.
Mixed path: relative error within its stated per-result bound err_est (reported
by the library: n * 2^-24 * kappa), checked against the oracle.
"""
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def gbs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_10070_gb300 as g

    g.lib()
    return g


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_haf(gbs, mats, precision):
    flat, n, offs = gbs.pack_matrices(mats)
    A = dev(flat)
    out = torch.zeros(2 * len(mats), dtype=torch.float64, device="cuda")
    kap = torch.zeros(len(mats), dtype=torch.float64, device="cuda")
    gbs.hafnian_batch(A, n, offs, precision, haf_out=out, kappa_out=kap)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    return o[0::2] + 1j * o[1::2], kap.cpu().numpy()


def run_prob(gbs, K, pats, precision, host=False):
    idx, n, offs = gbs.pack_patterns(pats)
    b = len(pats)
    if host:
        p = np.zeros(b); lp = np.zeros(b); hf = np.zeros(2 * b); er = np.zeros(b)
        gbs.prob_batch(K, idx, n, offs, precision, p_out=p, logp_out=lp, haf_out=hf, err_out=er)
        return p, lp, hf[0::2] + 1j * hf[1::2], er
    p = torch.zeros(b, dtype=torch.float64, device="cuda")
    lp = torch.zeros_like(p)
    hf = torch.zeros(2 * b, dtype=torch.float64, device="cuda")
    er = torch.zeros_like(p)
    gbs.prob_batch(K, dev(idx), n, offs, precision, p_out=p, logp_out=lp, haf_out=hf, err_out=er)
    torch.cuda.synchronize()
    h = hf.cpu().numpy()
    return p.cpu().numpy(), lp.cpu().numpy(), h[0::2] + 1j * h[1::2], er.cpu().numpy()


def kernel_for(gbs, U, r):
    Ud = dev(np.ascontiguousarray(U).view(np.float64))
    return gbs.build_kernel(Ud, dev(r))


def rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def rand_sym(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return scale * (A + A.T) / 2


# --- kernel matrix ------------------------------------------------------------

@pytest.mark.parametrize("m,seed", [(8, 0), (64, 1), (145, 2)])
def test_build_kernel_matches_oracle(gbs, orc, m, seed):
    U = W.haar_unitary(m, seed)
    r = W.squeezing(m, "uniform", seed=seed)
    K = kernel_for(gbs, U, r)
    B = torch.zeros(2 * m * m, dtype=torch.float64, device="cuda")
    K.copy_B(B)
    torch.cuda.synchronize()
    Bg = B.cpu().numpy().view(np.complex128).reshape(m, m)
    Bo = orc.build_B(U, r)
    assert np.abs(Bg - Bo).max() <= 1e-15 * max(1.0, math.sqrt(m))
    assert np.array_equal(Bg, Bg.T)
    assert abs(K.log_norm - orc.log_norm(r)) <= 1e-13 * abs(orc.log_norm(r))


def test_build_kernel_host_inputs(gbs, orc):
    m = 20
    U = W.haar_unitary(m, 7)
    r = W.squeezing(m, "const", value=0.7)
    K = gbs.build_kernel(U, r)  # numpy (host) inputs
    B = np.zeros(2 * m * m)
    K.copy_B(B)
    assert np.abs(B.view(np.complex128).reshape(m, m) - orc.build_B(U, r)).max() <= 1e-15 * 5


# --- Hafnians -----------------------------------------------------------------

@pytest.mark.parametrize("precision", [0, 1])
def test_hafnian_random_all_sizes(gbs, orc, precision):
    """n = 0..24 (odd included), several per size: tiles of every lane-group shape."""
    mats = [rand_sym(n, 1000 + 7 * n + k, scale=0.3) for n in range(0, 25) for k in range(3)]
    got, kap = run_haf(gbs, mats, precision)
    for A, g, kp in zip(mats, got, kap):
        n = A.shape[0]
        # the library reads no diagonal entry, and its subset sum pairs source
        # positions (t, t + n/2); kappa depends on that pairing, the Hafnian not
        order = [(p >> 1) + (n // 2 if p & 1 else 0) for p in range(n)]
        A0 = A[np.ix_(order, order)].copy()
        np.fill_diagonal(A0, 0)
        ref, K = orc.haf_subset(A0, return_kappa=True)
        if n % 2:
            assert g == 0
            continue
        if precision == 0:
            assert rel(g, ref) <= FP64_TOL, (n, g, ref)
        else:
            bound = max(n, 1) * 2.0 ** -24 * kp
            assert rel(g, ref) <= bound, (n, rel(g, ref), bound)
        if n >= 2:
            # kappa reported with |z|_1: between the modulus-based value and sqrt(2) times it
            kap_ref = K / abs(ref)
            assert kap_ref * (1 - 1e-6) <= kp <= math.sqrt(2) * kap_ref * (1 + 1e-6) + 1e-12


def test_hafnian_all_ones(gbs):
    """Haf(J_2k) = (2k-1)!!: FP64 path within its kappa * u bound."""
    mats = [np.ones((2 * k, 2 * k)) for k in range(0, 9)]
    got, kap = run_haf(gbs, mats, 0)
    for k, (g, kp) in enumerate(zip(got, kap)):
        expect = math.prod(range(2 * k - 1, 0, -2)) if k else 1
        assert abs(g - expect) <= 4 * max(2 * k, 1) * 2.0 ** -53 * kp * expect
        if k <= 6:
            assert rel(g, expect) <= 1e-11


def test_hafnian_bipartite_permanent(gbs, orc):
    """Haf([[0, C], [C^T, 0]]) = Per(C) (Ryser)."""
    rng = np.random.default_rng(5)
    mats, pers = [], []
    for k in (1, 2, 3, 5, 8, 11):
        C = (rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))) * 0.5
        Z = np.zeros((2 * k, 2 * k), complex)
        Z[:k, k:] = C
        Z[k:, :k] = C.T
        mats.append(Z)
        pers.append(orc.per_ryser(C))
    got, _ = run_haf(gbs, mats, 0)
    for g, p in zip(got, pers):
        assert rel(g, p) <= FP64_TOL


def test_hafnian_diagonal_ignored_and_permutation(gbs, orc):
    A = rand_sym(14, 3, 0.4)
    B = A.copy()
    np.fill_diagonal(B, 5.0 + 1j)
    perm = np.random.default_rng(9).permutation(14)
    C = A[np.ix_(perm, perm)]
    got, _ = run_haf(gbs, [A, B, C], 0)
    ref = orc.haf_subset(A)
    assert got[0] == got[1]  # the diagonal is never read
    for g in got:
        assert rel(g, ref) <= FP64_TOL


def test_hafnian_host_buffers(gbs, orc):
    mats = [rand_sym(n, 50 + n, 0.3) for n in (4, 10, 16)]
    flat, n, offs = gbs.pack_matrices(mats)
    out = np.zeros(2 * len(mats))
    kap = np.zeros(len(mats))
    gbs.hafnian_batch(flat, n, offs, 0, haf_out=out, kappa_out=kap)
    for A, g in zip(mats, out[0::2] + 1j * out[1::2]):
        assert rel(g, orc.haf_subset(A)) <= FP64_TOL


@pytest.mark.parametrize("precision", [0, 1])
def test_hafnian_max_size_n32(gbs, orc, precision):
    """n = 32 (GBS_MAX_N), two pins the oracle can afford at that size:
    Haf(A (+) B) = Haf(A) Haf(B) for a block-diagonal matrix of two n = 16
    blocks, and Haf([[0, C], [C^T, 0]]) = Per(C) for a 16 x 16 C (Ryser)."""
    rng = np.random.default_rng(32)
    A1, A2 = rand_sym(16, 321, 0.4), rand_sym(16, 322, 0.4)
    D = np.zeros((32, 32), complex)
    D[:16, :16], D[16:, 16:] = A1, A2
    perm = rng.permutation(32)  # hide the block structure from the pairing
    D = D[np.ix_(perm, perm)]
    C = (rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))) * 0.35
    Z = np.zeros((32, 32), complex)
    Z[:16, 16:], Z[16:, :16] = C, C.T
    got, kap = run_haf(gbs, [D, Z], precision)
    ref = [orc.haf_subset(A1) * orc.haf_subset(A2), orc.per_ryser(C)]
    for g, k, r_ in zip(got, kap, ref):
        if precision == 0:
            assert rel(g, r_) <= FP64_TOL, rel(g, r_)
        else:
            assert rel(g, r_) <= 32 * 2.0 ** -24 * k


def test_hafnian_ragged_batch_every_order(gbs, orc):
    """A ragged batch mixing every n in 0..26 (odd included), in shuffled order."""
    rng = np.random.default_rng(77)
    sizes = list(range(0, 27)) * 2
    rng.shuffle(sizes)
    mats = [rand_sym(n, 500 + i, 0.3) for i, n in enumerate(sizes)]
    got, _ = run_haf(gbs, mats, 0)
    for A, g in zip(mats, got):
        n = A.shape[0]
        if n % 2:
            assert g == 0
        elif n <= 22:
            assert rel(g, orc.haf_subset(A)) <= FP64_TOL


# --- probabilities ---------------------------------------------------------------

def test_prob_tiny_exhaustive(gbs, orc):
    """m = 8, r = 0.5: all 70 collision-free 4-photon and all 36 2-photon patterns,
    against the perfect-matching oracle."""
    U, r, pats = W.workload("tiny_m8")
    K = kernel_for(gbs, U, r)
    ref = orc.prob(U, r, pats, method="pm")
    for prec in (0, 1):
        p, lp, hf, er = run_prob(gbs, K, pats, prec)
        if prec == 0:
            assert np.all(rel(hf, ref["haf"]) <= FP64_TOL)
            assert np.all(rel(p, ref["p"]) <= FP64_TOL)
            assert np.all(np.abs(lp - ref["logp"]) <= FP64_TOL * np.abs(ref["logp"]))
        else:
            assert np.all(rel(hf, ref["haf"]) <= er)


def test_prob_host_and_device_buffers_agree(gbs):
    U, r, pats = W.workload("tiny_m8")
    K = kernel_for(gbs, U, r)
    a = run_prob(gbs, K, pats, 0, host=False)
    b = run_prob(gbs, K, pats, 0, host=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_prob_pair_sum_budget_overflow(gbs, orc):
    """A batch whose pair sums exceed their 2 GiB budget: 32768 collision-free
    n = 16 patterns need about 2.3 GB, so the first matrices form R_2 from their
    pair sums and the last ones by the product, in the same launch. Matrices
    from both ends are checked against the oracle."""
    m = 64
    U = W.haar_unitary(m, 1)
    r = W.squeezing(m, "uniform", seed=1)
    rng = np.random.default_rng(77)
    pats = [np.sort(rng.choice(m, 16, replace=False)).astype(np.int32) for _ in range(32768)]
    K = kernel_for(gbs, U, r)
    p, lp, hf, er = run_prob(gbs, K, pats, 0)
    sample = list(range(0, 12)) + list(range(32768 - 12, 32768))
    ref = orc.prob(U, r, [pats[i] for i in sample])
    assert np.all(rel(hf[sample], ref["haf"]) <= FP64_TOL), rel(hf[sample], ref["haf"])
    assert np.all(np.isfinite(p)) and np.all(p > 0)


def test_prob_batched_n16_sampled(gbs, orc):
    """The benchmark's workload and launch (M = 64, 4096 patterns, n = 16): the
    whole batch runs on the GPU; 48 patterns spread over it are checked."""
    U, r, pats = W.workload("batched_m64_n16")
    K = kernel_for(gbs, U, r)
    p, lp, hf, er = run_prob(gbs, K, pats, 0)
    sample = list(range(0, 4096, 4096 // 48))[:48] + [4095]
    ref = orc.prob(U, r, [pats[i] for i in sample])
    assert np.all(rel(hf[sample], ref["haf"]) <= FP64_TOL)
    assert np.all(rel(p[sample], ref["p"]) <= FP64_TOL)
    assert np.all(np.isfinite(p)) and np.all(p > 0)


def test_prob_mixed_collisions(gbs, orc):
    """M = 144, n in {8..24}, up to 3 photons per mode: FP64 within 1e-10, mixed
    within its own err_est, on a sample of the 2048-pattern batch."""
    U, r, pats = W.workload("mixed_m144")
    K = kernel_for(gbs, U, r)
    p64, _, h64, e64 = run_prob(gbs, K, pats, 0)
    p32, _, h32, e32 = run_prob(gbs, K, pats, 1)
    sample = list(range(0, 2048, 2048 // 40))
    ref = orc.prob(U, r, [pats[i] for i in sample])
    assert np.all(rel(h64[sample], ref["haf"]) <= FP64_TOL)
    assert np.all(rel(h32[sample], ref["haf"]) <= e32[sample])
    assert np.all(np.isfinite(e64)) and np.all(e64 >= 0)


@pytest.mark.slow
def test_prob_large_n28_n30_sampled(gbs, orc):
    """M = 900, r = 1: the 80-pattern batch (64 at n = 28, 16 at n = 30) in one
    launch; one n = 28 and one n = 30 result against the oracle."""
    U, r, pats = W.workload("large_m900")
    K = kernel_for(gbs, U, r)
    p, lp, hf, er = run_prob(gbs, K, pats, 0)
    sample = [0, 64]
    ref = orc.prob(U, r, [pats[i] for i in sample])
    assert np.all(rel(hf[sample], ref["haf"]) <= FP64_TOL), (rel(hf[sample], ref["haf"]), er[sample])
    assert np.all(np.isfinite(lp))


def test_prob_large_all_patterns_golden(gbs):
    """All 80 large instances (M = 900, r = 1, n = 28 and 30) against stored
    double-double oracle values (tests/golden/large_m900_oracle.json, written
    by tests/golden/make_large_golden.py from the oracle alone)."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "large_m900_oracle.json")))
    U, r, pats = W.workload("large_m900")
    assert [list(map(int, x)) for x in pats] == [q["x"] for q in g["patterns"]]
    K = kernel_for(gbs, U, r)
    B = torch.zeros(2 * 900 * 900, dtype=torch.float64, device="cuda")
    K.copy_B(B)
    Bc = B.cpu().numpy().view(np.complex128)
    # the box's Haar draw must match the one the values were computed from
    assert abs(np.abs(Bc).sum() - g["B_checksum"][0]) <= 1e-9 * g["B_checksum"][0]
    p, lp, hf, er = run_prob(gbs, K, pats, 0)
    ref = np.array([complex(q["haf_dd"][0] + q["haf_dd"][1], q["haf_dd"][2] + q["haf_dd"][3])
                    for q in g["patterns"]])
    err = rel(hf, ref)
    nn = np.array([len(x) for x in pats])
    for n_ in (28, 30):  # shown with -s
        e_ = err[nn == n_]
        print("n=%d: %d patterns, max rel. error %.2e, median %.2e, largest estimate %.2e, within estimate: %s"
              % (n_, e_.size, e_.max(), np.median(e_), er[nn == n_].max(), bool(np.all(e_ <= er[nn == n_]))))
    assert np.all(err <= FP64_TOL), (err.max(), int(np.argmax(err)))
    assert np.all(np.abs(lp - np.array([q["logp"] for q in g["patterns"]])) <= 1e-9)


def test_prob_heavy_collisions(gbs, orc):
    """Patterns with many photons in few modes (up to 8 in one mode), n <= 16."""
    m = 12
    U = W.haar_unitary(m, 61)
    r = W.squeezing(m, "uniform", seed=61)
    K = kernel_for(gbs, U, r)
    pats = [np.array([3] * 8 + [5] * 8), np.array([0] * 6 + [1] * 6 + [2, 2, 7, 7]),
            np.array([4] * 4 + [9] * 4 + [11] * 2), np.array([1] * 10 + [2] * 2 + [6] * 2),
            np.array([0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3])]
    p, lp, hf, er = run_prob(gbs, K, pats, 0)
    ref = orc.prob(U, r, pats, method="pm")
    assert np.all(rel(hf, ref["haf"]) <= FP64_TOL), rel(hf, ref["haf"])
    assert np.all(rel(p, ref["p"]) <= FP64_TOL)


def bunched_patterns(m, n_values, per_n, seed):
    """Multisets of n modes drawn with replacement from m: many photons per mode."""
    rng = np.random.default_rng(seed)
    return [np.sort(rng.choice(m, n, replace=True)).astype(np.int32) for n in n_values for _ in range(per_n)]


def test_prob_repeated_row_route(gbs, orc):
    """Host index lists with many repeated modes take the repeated-row route
    (terms of the moment-extraction identity) when it is cheaper than the
    subset sum; device index lists and explicit matrices take the subset sum.
    All three agree with the double-double oracle within 1e-10."""
    m = 8
    U = W.haar_unitary(m, 5)
    r = np.full(m, 1.0)
    K = kernel_for(gbs, U, r)
    pats = bunched_patterns(m, (8, 12, 16, 20), 3, 71) + bunched_patterns(m, (24, 28), 1, 72)
    ref = orc.prob(U, r, pats)
    p_h, lp_h, hf_h, er_h = run_prob(gbs, K, pats, 0, host=True)
    p_d, lp_d, hf_d, er_d = run_prob(gbs, K, pats, 0)
    assert np.all(rel(hf_h, ref["haf"]) <= FP64_TOL), rel(hf_h, ref["haf"])
    assert np.all(rel(p_h, ref["p"]) <= FP64_TOL)
    assert np.all(rel(hf_d, ref["haf"]) <= FP64_TOL), rel(hf_d, ref["haf"])
    assert np.all(np.abs(lp_h - lp_d) <= 1e-9)
    B = torch.zeros(2 * m * m, dtype=torch.float64, device="cuda")
    K.copy_B(B)
    Bc = B.cpu().numpy().view(np.complex128).reshape(m, m)
    flat, n, offs = gbs.pack_matrices([Bc[np.ix_(x, x)] for x in pats])
    hm = np.zeros(2 * len(pats))
    gbs.hafnian_batch(flat, n, offs, gbs.FP64, haf_out=hm)
    assert np.all(rel(hm[0::2] + 1j * hm[1::2], ref["haf"]) <= FP64_TOL)


def test_repeated_row_route_extreme_bunching(gbs, orc):
    """32 photons in 2 modes (289 terms): the repeated-row route against the
    oracle's repeated-row formula, and much faster than the subset sum that a
    device index list takes for the same pattern (2^16 subsets of order <= 32)."""
    import time

    m = 6
    U = W.haar_unitary(m, 8)
    r = np.full(m, 0.9)
    K = kernel_for(gbs, U, r)
    x = np.array([1] * 16 + [4] * 16, np.int32)
    Bdd = orc.build_B_dd(U, np.tanh(r))
    B = (Bdd[..., 0] + Bdd[..., 1]) + 1j * (Bdd[..., 2] + Bdd[..., 3])
    ref = orc.haf_repeated(B[np.ix_([1, 4], [1, 4])], [16, 16])
    _, _, hf_h, _ = run_prob(gbs, K, [x], 0, host=True)
    _, _, hf_d, _ = run_prob(gbs, K, [x], 0)
    assert rel(hf_h, np.array([ref]))[0] <= FP64_TOL, (hf_h, ref)
    assert rel(hf_d, np.array([ref]))[0] <= FP64_TOL, (hf_d, ref)

    def best(host, reps=3):
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            run_prob(gbs, K, [x], 0, host=host)
            ts.append(time.perf_counter() - t0)
        return min(ts)

    assert best(True) * 3 < best(False)


def test_prob_mixed_bound_large_golden(gbs):
    """The mixed path's stated per-result bound holds on the n = 28, 30 instances."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "large_m900_oracle.json")))
    U, r, pats = W.workload("large_m900")
    K = kernel_for(gbs, U, r)
    sel = [0, 1, 2, 64, 65]
    p, lp, hf, er = run_prob(gbs, K, [pats[i] for i in sel], 1)
    ref = np.array([complex(g["patterns"][i]["haf_dd"][0] + g["patterns"][i]["haf_dd"][1],
                            g["patterns"][i]["haf_dd"][2] + g["patterns"][i]["haf_dd"][3]) for i in sel])
    assert np.all(rel(hf, ref) <= er), (rel(hf, ref), er)


# --- edge cases -------------------------------------------------------------------

def test_edge_cases(gbs, orc):
    m = 10
    U = W.haar_unitary(m, 11)
    r = W.squeezing(m, "uniform", seed=11)
    K = kernel_for(gbs, U, r)
    pats = [np.array([], np.int32), np.array([3], np.int32), np.array([2, 2]), np.array([0, 9]),
            np.array([5, 5, 5, 5, 5, 5]), np.array([1, 2, 3]), np.array([9, 0, 4, 4])]
    p, lp, hf, er = run_prob(gbs, K, pats, 0)
    ref = orc.prob(U, r, pats)
    L = orc.log_norm(r)
    assert abs(p[0] - math.exp(-L)) <= 1e-14 * math.exp(-L) and hf[0] == 1
    assert p[1] == 0 and hf[1] == 0 and lp[1] == -np.inf
    assert p[5] == 0 and hf[5] == 0
    for i in (2, 3, 4, 6):
        assert rel(hf[i], ref["haf"][i]) <= FP64_TOL
        assert rel(p[i], ref["p"][i]) <= FP64_TOL
    # empty batch
    gbs.prob_batch(K, dev(np.zeros(1, np.int32)), np.zeros(0, np.int32), np.zeros(0, np.int64), 0)


def test_errors(gbs):
    m = 6
    U = W.haar_unitary(m, 1)
    K = gbs.build_kernel(U, np.full(m, 0.5))
    idx, n, offs = gbs.pack_patterns([np.array([0, 7])])
    with pytest.raises(gbs.GbsError) as ei:
        gbs.prob_batch(K, idx, n, offs, 0, p_out=np.zeros(1))
    assert ei.value.code == -3
    idx, n, offs = gbs.pack_patterns([np.zeros(34, np.int32)])
    with pytest.raises(gbs.GbsError) as ei:
        gbs.prob_batch(K, idx, n, offs, 0, p_out=np.zeros(1))
    assert ei.value.code == -3
    with pytest.raises(gbs.GbsError) as ei:
        gbs.prob_batch(K, idx, n, offs, 7, p_out=np.zeros(1))
    assert ei.value.code == -1
    # device index list with an out-of-range entry: NaN result, no fault
    idx, n, offs = gbs.pack_patterns([np.array([0, 1]), np.array([0, 99]), np.array([2, 3])])
    p = torch.zeros(3, dtype=torch.float64, device="cuda")
    gbs.prob_batch(K, dev(idx), n, offs, 0, p_out=p)
    pc = p.cpu().numpy()
    assert np.isfinite(pc[0]) and np.isnan(pc[1]) and np.isfinite(pc[2])


def test_determinism_and_order_independence(gbs):
    U, r, pats = W.workload("mixed_m144")
    pats = pats[:300]
    K = kernel_for(gbs, U, r)
    a = run_prob(gbs, K, pats, 0)
    b = run_prob(gbs, K, pats, 0)
    assert np.array_equal(a[2], b[2])
    perm = np.random.default_rng(0).permutation(len(pats))
    c = run_prob(gbs, K, [pats[i] for i in perm], 0)
    assert np.array_equal(c[2], a[2][perm])


def test_pairing_choice_lowers_cancellation(gbs):
    """For n >= 26 the batched path runs the subset sum in the candidate ordering
    of rows and columns whose sampled sum |f| is smallest. The Hafnian is the
    same in every ordering; the cancellation ratio kappa = sum |f| / |Haf| falls
    (the no-alloc entry point keeps the given ordering), and both results agree
    with the stored oracle values."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "large_m900_oracle.json")))
    U, r, pats = W.workload("large_m900")
    pats = pats[:16]
    K = kernel_for(gbs, U, r)
    B = torch.zeros(2 * 900 * 900, dtype=torch.float64, device="cuda")
    K.copy_B(B)
    Bc = B.cpu().numpy().view(np.complex128).reshape(900, 900)
    flat, n, offs = gbs.pack_matrices([Bc[np.ix_(x, x)] for x in pats])
    A = dev(flat)
    b = len(pats)
    h1 = torch.zeros(2 * b, dtype=torch.float64, device="cuda")
    k1 = torch.zeros(b, dtype=torch.float64, device="cuda")
    gbs.hafnian_batch(A, n, offs, gbs.FP64, haf_out=h1, kappa_out=k1)
    h0 = torch.zeros(2 * b, dtype=torch.float64, device="cuda")
    k0 = torch.zeros(b, dtype=torch.float64, device="cuda")
    for c in range(0, b, 2):
        out = torch.zeros(4, dtype=torch.float64, device="cuda")
        ko = torch.zeros(2, dtype=torch.float64, device="cuda")
        gbs.hafnian_batch_noalloc(A, n[c:c + 2], offs[c:c + 2], gbs.FP64, haf_out=out, kappa_out=ko)
        h0[2 * c:2 * c + 4] = out
        k0[c:c + 2] = ko
    ref = np.array([complex(q["haf_dd"][0] + q["haf_dd"][1], q["haf_dd"][2] + q["haf_dd"][3])
                    for q in g["patterns"][:16]])
    for h in (h1, h0):
        a = h.cpu().numpy()
        assert np.all(rel(a[0::2] + 1j * a[1::2], ref) <= FP64_TOL)
    ratio = k1.cpu().numpy() / k0.cpu().numpy()
    assert np.all(np.isfinite(ratio))
    assert np.exp(np.mean(np.log(ratio))) < 0.8, ratio


def test_repeated_row_route_largest_orders(gbs, orc):
    """n = 30 and 32 through the repeated-row route: all photons in one mode
    (Haf = B_vv^16 (31)!!, the closed form of J_32 scaled) and photons spread
    over 5 to 6 modes (the oracle's repeated-row formula); each result is also
    within its own error estimate."""
    m = 6
    U = W.haar_unitary(m, 9)
    r = np.full(m, 0.6)
    K = kernel_for(gbs, U, r)
    Bdd = orc.build_B_dd(U, np.tanh(r))
    B = (Bdd[..., 0] + Bdd[..., 1]) + 1j * (Bdd[..., 2] + Bdd[..., 3])
    one = np.full(32, 3, np.int32)
    _, _, hf, er = run_prob(gbs, K, [one], 0, host=True)
    ref = B[3, 3] ** 16 * math.prod(range(31, 0, -2))
    # the 33 alternating terms cancel strongly here (measured 3.6e-11)
    err = abs(hf[0] - ref) / abs(ref)
    assert err <= FP64_TOL and err <= er[0], (hf[0], ref, er[0])
    pats = [np.array([0] * 7 + [1] * 5 + [2] * 6 + [4] * 6 + [5] * 6, np.int32),
            np.array([0] * 4 + [1] * 6 + [2] * 6 + [3] * 6 + [4] * 4 + [5] * 6, np.int32)]
    _, _, hf, er = run_prob(gbs, K, pats, 0, host=True)
    for x, h, e in zip(pats, hf, er):
        modes, reps = np.unique(x, return_counts=True)
        ref = orc.haf_repeated(B[np.ix_(modes, modes)], reps)
        assert abs(h - ref) <= FP64_TOL * abs(ref) and abs(h - ref) <= e * abs(ref), (reps, h, ref, e)


@pytest.mark.parametrize("precision", [0, 1])
def test_whole_matrix_items_match_per_size_items(gbs, precision):
    """In a large batch most matrices of an order are one whole-matrix work item
    (all subset sizes staged and reduced together); a single-pattern call runs
    per-size items. Both give the same Hafnian: within 1e-11 (FP64) or within
    the stated bound (mixed)."""
    U, r, pats = W.workload("batched_m64_n16")
    K = kernel_for(gbs, U, r)
    _, _, hb, eb = run_prob(gbs, K, pats, precision)
    for i in (0, 1, 777, 2048, 3000):
        _, _, hs, es = run_prob(gbs, K, [pats[i]], precision)
        tol = 1e-11 if precision == 0 else max(eb[i], es[0])
        assert rel(hb[i:i + 1], hs)[0] <= tol, (i, hb[i], hs[0], tol)
