"""CUDA path vs the CPU oracle, through the C ABI (GPU only).

FP64 path: relative error of Haf and p within 1e-10 of the double-double oracle.
Mixed path: relative error within its stated per-result bound err_est (reported
by the library: min(n, 4) * 2^-24 * kappa), checked against the oracle.
"""
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def mixed_c(n):
    """The mixed path's stated bound is c u kappa with u = 2^-24, c = min(n, 4)
    (fitted on the oracle; include/gbs.h)."""
    return np.minimum(np.maximum(np.asarray(n), 1), 4)


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


def golden(name):
    """Stored double-double oracle values (tests/golden/make_golden.py)."""
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        g = json.load(f)
    g["haf"] = np.array(g["haf_re"]) + 1j * np.array(g["haf_im"])
    g["logp"] = np.array(g["logp"])
    g["kappa"] = np.array(g["kappa"])
    return g


def check_draw(U, g):
    """The Haar draw on this machine is byte for byte the one the stored values
    were computed from (the draw comes from a LAPACK QR, whose last bits differ
    between platforms; tests/golden/make_golden.py writes the values on the
    platform that runs these tests)."""
    import hashlib

    h = hashlib.sha256(np.ascontiguousarray(U, dtype=np.complex128).tobytes()).hexdigest()
    assert h == g["U_sha256"], "Haar draw differs from the stored values' draw: regenerate tests/golden"


def check_B(K, g):
    """The box's Haar draw and kernel matrix are the ones the values came from."""
    m = g["m"]
    B = torch.zeros(2 * m * m, dtype=torch.float64, device="cuda")
    K.copy_B(B)
    Bc = B.cpu().numpy().view(np.complex128)
    assert abs(np.abs(Bc).sum() - g["B_checksum"][0]) <= 1e-9 * g["B_checksum"][0]
    return Bc.reshape(m, m)


def kappa_pin(kp, kref, slack=0.0):
    """The library reports kappa with |z|_1 = |re| + |im| per term, the oracle
    with the modulus: the ratio lies in [1, sqrt(2)] (up to the slack of the
    path's own rounding of the terms)."""
    return (kref * (1 - 1e-6 - slack) <= kp) & (kp <= math.sqrt(2) * kref * (1 + 1e-6 + slack))


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
    # entries correctly rounded up to the last bit of tanh r_k (each side
    # rounds it once; sum_k |U_ik| |U_jk| <= 1, so that moves an entry by at
    # most ~1e-16) and the final rounding
    d = np.abs(Bg - Bo)
    assert np.all(d.real <= 2 * np.spacing(np.abs(Bo.real)) + 2.3e-16), d.real.max()
    assert np.all(d.imag <= 2 * np.spacing(np.abs(Bo.imag)) + 2.3e-16), d.imag.max()
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
            bound = mixed_c(n) * 2.0 ** -24 * kp
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
            assert rel(g, r_) <= mixed_c(32) * 2.0 ** -24 * k


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


def golden_batch_check(gbs, name):
    """A whole workload batch in both precisions, as the benchmark launches it
    (device index lists), against stored oracle values for every pattern:
    FP64 within 1e-10 and within its own error estimate; the mixed path within
    its stated bound, whose kappa is first pinned to the oracle's kappa of the
    same pairing (the library pairs positions (t, t + n/2) and zeroes the
    diagonal below n = 26, as the stored kappa does)."""
    U, r, pats = W.workload(name)
    g = golden(name + "_oracle.json")
    check_draw(U, g)
    assert [list(map(int, x)) for x in pats] == g["x"]
    K = kernel_for(gbs, U, r)
    check_B(K, g)
    nn = np.array([len(x) for x in pats])
    p64, lp64, h64, e64 = run_prob(gbs, K, pats, 0)
    err = rel(h64, g["haf"])
    assert np.all(err <= FP64_TOL), (err.max(), int(np.argmax(err)))
    assert np.all(err <= e64), int(np.argmax(err / e64))
    assert np.all(np.abs(lp64 - g["logp"]) <= FP64_TOL * np.abs(g["logp"]))
    assert np.all(rel(p64, np.exp(g["logp"])) <= FP64_TOL)
    # FP64 kappa (subset route; no pattern here is bunched enough for the
    # repeated-row route) against the oracle's
    k64 = e64 / (nn * 2.0 ** -53)
    assert np.all(kappa_pin(k64, g["kappa"])), np.min(k64 / g["kappa"])
    p32, _, h32, e32 = run_prob(gbs, K, pats, 1)
    k32 = e32 / (mixed_c(nn) * 2.0 ** -24)
    assert np.all(kappa_pin(k32, g["kappa"], slack=1e-3)), (np.min(k32 / g["kappa"]), np.max(k32 / g["kappa"]))
    err32 = rel(h32, g["haf"])
    assert np.all(err32 <= e32), (err32 / e32).max()
    return err, err32, e32


def test_prob_batched_n16_all_patterns_golden(gbs):
    """The benchmark's workload and launch (M = 64, 4096 patterns, n = 16): every
    result against the stored oracle values."""
    golden_batch_check(gbs, "batched_m64_n16")


def test_prob_mixed_collisions(gbs):
    """M = 144, n in {8..24}, up to 3 photons per mode (collisions, Eq.
    W_s_example): all 2048 results against the stored oracle values."""
    golden_batch_check(gbs, "mixed_m144")


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
    check_draw(U, g)
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
    assert np.all(err <= er), (err / er).max()
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
    """Index lists with many repeated modes take the repeated-row route (terms
    of the moment-extraction identity) when it is cheaper than the subset sum:
    chosen on the host for host lists and on the device for device lists, with
    bit-identical results; explicit matrices take the subset sum. All agree
    with the double-double oracle within 1e-10."""
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
    # the same route on both sides (the planner's item split of subset-sum
    # patterns may differ, which changes only the rounding)
    assert np.all(rel(hf_d, hf_h) <= 1e-12) and np.all(np.abs(er_d - er_h) <= 1e-6 * er_h)
    assert np.all(np.abs(lp_h - lp_d) <= 1e-9)
    B = torch.zeros(2 * m * m, dtype=torch.float64, device="cuda")
    K.copy_B(B)
    Bc = B.cpu().numpy().view(np.complex128).reshape(m, m)
    flat, n, offs = gbs.pack_matrices([Bc[np.ix_(x, x)] for x in pats])
    hm = np.zeros(2 * len(pats))
    gbs.hafnian_batch(flat, n, offs, gbs.FP64, haf_out=hm)
    assert np.all(rel(hm[0::2] + 1j * hm[1::2], ref["haf"]) <= FP64_TOL)


def test_repeated_row_route_extreme_bunching(gbs, orc):
    """32 photons in 2 modes (289 terms): the repeated-row route, from a host
    or a device index list, against the oracle's repeated-row formula, and much
    faster than the subset sum that the explicit matrix takes (2^16 subsets of
    order <= 32)."""
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

    Bg = torch.zeros(2 * m * m, dtype=torch.float64, device="cuda")
    K.copy_B(Bg)
    Bc = Bg.cpu().numpy().view(np.complex128).reshape(m, m)
    flat, n, offs = gbs.pack_matrices([Bc[np.ix_(x, x)]])
    Ad = dev(flat)
    hm = torch.zeros(2, dtype=torch.float64, device="cuda")

    def best(fn, reps=3):
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return min(ts)

    t_rep = best(lambda: run_prob(gbs, K, [x], 0))
    t_sub = best(lambda: gbs.hafnian_batch(Ad, n, offs, gbs.FP64, haf_out=hm))
    assert t_rep * 3 < t_sub, (t_rep, t_sub)


def test_prob_mixed_bound_large_golden(gbs):
    """The mixed path's stated per-result bound holds on the n = 28, 30 instances.
    The kappa behind it is pinned first: the no-allocation entry point keeps
    the default pairing (positions t and t + n/2), for which the oracle's kappa
    is stored (tests/golden/large_m900_default_order.json), in both precisions;
    the batched call then runs the mixed path in its chosen ordering."""
    U, r, pats = W.workload("large_m900")
    K = kernel_for(gbs, U, r)
    gd = golden("large_m900_default_order.json")
    check_draw(U, gd)
    Bc = check_B(K, gd)
    sel = gd["pattern_index"]
    xs = [pats[i] for i in sel]
    assert [list(map(int, x)) for x in xs] == gd["x"]
    nn = np.array([len(x) for x in xs])
    for prec, slack in ((0, 0.0), (1, 1e-3)):
        hc = np.zeros(len(xs), complex)
        kc = np.zeros(len(xs))
        for q, x in enumerate(xs):  # one matrix per call: within the entry point's item limit
            flat, n, offs = gbs.pack_matrices([Bc[np.ix_(x, x)]])
            h = torch.zeros(2, dtype=torch.float64, device="cuda")
            k = torch.zeros(1, dtype=torch.float64, device="cuda")
            gbs.hafnian_batch_noalloc(dev(flat), n, offs, prec, haf_out=h, kappa_out=k)
            torch.cuda.synchronize()
            hh = h.cpu().numpy()
            hc[q] = complex(hh[0], hh[1])
            kc[q] = k.cpu().numpy()[0]
        assert np.all(kappa_pin(kc, gd["kappa"], slack)), (prec, kc / gd["kappa"])
        bound = (nn * 2.0 ** -53 if prec == 0 else mixed_c(nn) * 2.0 ** -24) * kc
        assert np.all(rel(hc, gd["haf"]) <= bound), (prec, rel(hc, gd["haf"]) / bound)
    g = golden_large()
    sel = [0, 1, 2, 64, 65]
    p, lp, hf, er = run_prob(gbs, K, [pats[i] for i in sel], 1)
    assert np.all(rel(hf, g[sel]) <= er), (rel(hf, g[sel]), er)


def golden_large():
    """Hafnians of the 80 large instances (tests/golden/large_m900_oracle.json)."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "large_m900_oracle.json")))
    return np.array([complex(q["haf_dd"][0] + q["haf_dd"][1], q["haf_dd"][2] + q["haf_dd"][3])
                     for q in g["patterns"]])


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


def test_prob_bunched_batch_device_index_list(gbs, orc):
    """The bunched workload (M = 8, r = 1, 512 patterns of n = 24 drawn with
    replacement, the collision case of Eq. W_s_example) as one batch from a
    device index list: the route choice on the device sends these patterns to
    the repeated-row sum, bit-identical to the host list's route; the patterns
    with the largest error estimates and a spread of others are within 1e-10
    of the double-double oracle and within their estimates."""
    U, r, pats = W.workload("bunched_m8")
    K = kernel_for(gbs, U, r)
    p_d, lp_d, hf_d, er_d = run_prob(gbs, K, pats, 0)
    p_h, lp_h, hf_h, er_h = run_prob(gbs, K, pats, 0, host=True)
    assert np.array_equal(hf_d, hf_h) and np.array_equal(er_d, er_h)
    assert np.array_equal(p_d, p_h)
    worst = list(np.argsort(er_d)[-6:])
    sample = sorted(set(worst + list(range(0, 512, 128))))
    ref = orc.prob(U, r, [pats[i] for i in sample])
    err = rel(hf_d[sample], ref["haf"])
    assert np.all(err <= FP64_TOL), (err, er_d[sample])
    assert np.all(err <= er_d[sample]), (err, er_d[sample])
    assert np.all(rel(p_d[sample], ref["p"]) <= FP64_TOL)


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


@pytest.mark.parametrize("n_", [16, 28])
def test_autotune_shape_fits_and_agrees(gbs, n_):
    """gbs_autotune times its candidate launch shapes for one photon number and
    keeps the fastest: a batch then runs in the tuned shape (so it fits) and
    gives the same Hafnians as before tuning within 1e-10, both within 1e-10
    of the stored oracle values."""
    if n_ == 16:
        U, r, pats = W.workload("batched_m64_n16")
        ref = golden("batched_m64_n16_oracle.json")["haf"]
        sel = list(range(0, 4096, 16))
    else:
        U, r, pats = W.workload("large_m900")
        ref = golden_large()
        sel = list(range(8))
    K = kernel_for(gbs, U, r)
    xs = [pats[i] for i in sel]
    _, _, before, _ = run_prob(gbs, K, xs, 0)
    chosen = gbs.autotune(n_, gbs.FP64)
    assert chosen in (1, 2, 4, 8, 16)
    _, _, after, er = run_prob(gbs, K, xs, 0)
    assert np.all(rel(after, before) <= FP64_TOL)
    assert np.all(rel(after, ref[sel]) <= FP64_TOL) and np.all(rel(before, ref[sel]) <= FP64_TOL)
    assert np.all(rel(after, ref[sel]) <= er)


def test_float_probe_picks_the_fp64_probes_ordering(gbs):
    """At n >= 26 gbs_prob_batch ranks the 16 candidate orderings with the
    float kernel over the kernel's float copy of B, gbs_hafnian_batch with the
    FP64 kernel over the explicit matrices B_x. Both read the same entries and
    then run the same FP64 subset sum, so where they choose the same ordering
    they give the same Hafnian and the same cancellation ratio kappa: checked
    on n = 28 and n = 30 instances of the large batch (the gbs_autotune runs
    at n = 28 cover the probe under an explicit launch shape)."""
    U, r, pats = W.workload("large_m900")
    m = U.shape[0]
    K = kernel_for(gbs, U, r)
    sel = [0, 1, 2, 3, 64, 65]
    xs = [pats[i] for i in sel]
    _, _, hp, ep = run_prob(gbs, K, xs, 0)
    Bg = torch.zeros(2 * m * m, dtype=torch.float64, device="cuda")
    K.copy_B(Bg)
    torch.cuda.synchronize()
    B = Bg.cpu().numpy().view(np.complex128).reshape(m, m)
    hh, kh = run_haf(gbs, [B[np.ix_(x, x)] for x in xs], 0)
    n = np.array([len(x) for x in xs], dtype=float)
    kp = ep / (n * 2.0 ** -53)  # err_est = n u kappa
    assert np.all(np.abs(kp / kh - 1.0) <= 1e-12), (kp, kh)
    assert np.all(rel(hp, hh) <= 1e-14), (hp, hh)
