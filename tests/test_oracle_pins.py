"""Pins for the CPU oracle: it is checked against facts fixed by the paper and by
mathematics, never against itself or the CUDA path.

Each test names what it pins. Together they are chosen so that a plausible slip
in the oracle (a dropped pair swap X, a wrong sign (-1)^{h-|S|}, a 1/k instead of
1/(2k), a transposed U, a missing s_j!, a wrong cosh normalisation) fails one.
"""
import itertools
import math
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dfact(k):  # (k)!! for odd k, 1 for k <= 0
    return math.prod(range(k, 0, -2)) if k > 0 else 1


def rand_sym(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return (A + A.T) / 2


# --- Hafnian tiers -----------------------------------------------------------

@pytest.mark.parametrize("k", range(0, 9))
def test_haf_all_ones_double_factorial(orc, k):
    """Haf(J_2k) = (2k-1)!!, the number of perfect matchings (Eq. HafMatch)."""
    J = np.ones((2 * k, 2 * k))
    assert orc.haf_pm(J) == dfact(2 * k - 1)
    assert orc.haf_subset(J) == dfact(2 * k - 1)


@pytest.mark.parametrize("k", [9, 10])
def test_haf_all_ones_subset_large(orc, k):
    """(2k-1)!! through the subset sum at n = 18, 20 (kappa ~1e6: dd is needed)."""
    J = np.ones((2 * k, 2 * k))
    assert orc.haf_subset(J) == dfact(2 * k - 1)


def test_haf_odd_and_empty(orc):
    """Odd n has no perfect matching (Haf = 0); the empty matrix has Haf = 1."""
    assert orc.haf_pm(np.ones((3, 3))) == 0
    assert orc.haf_subset(np.ones((5, 5))) == 0
    assert orc.haf_pm(np.zeros((0, 0))) == 1
    assert orc.haf_subset(np.zeros((0, 0))) == 1


def test_haf_n4_paper_expansion(orc):
    """The n = 4 expansion printed in Sec. 2.3, read from the golden fixture."""
    lines = [l.split() for l in open(os.path.join(GOLDEN, "ws_example.txt")) if not l.startswith("#")]
    matchings = [l for l in lines if l[0] == "matchings"][0][1:]
    V = rand_sym(4, 1)
    expect = 0
    for mt in matchings:
        term = 1
        for pair in mt.split(","):
            a, b = (int(v) - 1 for v in pair.split("-"))
            term *= V[a, b]
        expect += term
    assert abs(orc.haf_pm(V) - expect) < 1e-14 * abs(expect)
    assert abs(orc.haf_subset(V) - expect) < 1e-14 * abs(expect)


@pytest.mark.parametrize("n", [2, 4, 6, 8, 10, 12, 14])
def test_subset_equals_matchings_dd(orc, n):
    """The two independent Hafnian tiers agree to dd accuracy (~1e-20)."""
    A = rand_sym(n, 100 + n)
    a = orc.haf_pm(A)
    b = orc.haf_subset(A)
    assert abs(a - b) <= 1e-20 * abs(a) + 1e-300


def test_subset_equals_matchings_n16(orc):
    A = rand_sym(16, 7)
    a = orc.haf_pm(A)
    b = orc.haf_subset(A)
    assert abs(a - b) <= 1e-20 * abs(a)


def test_haf_bipartite_equals_permanent(orc):
    """Haf([[0, C], [C^T, 0]]) = Per(C) (textbook), Per by Ryser (O3)."""
    rng = np.random.default_rng(3)
    for k in (1, 2, 3, 5, 7):
        C = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
        Z = np.zeros((2 * k, 2 * k), complex)
        Z[:k, k:] = C
        Z[k:, :k] = C.T
        per = orc.per_ryser(C)
        assert abs(orc.haf_pm(Z) - per) <= 1e-13 * abs(per)
        assert abs(orc.haf_subset(Z) - per) <= 1e-13 * abs(per)


def test_ryser_pins(orc):
    """Ryser against the permutation sum (k <= 6), Per(J_k) = k!, Per(I) = 1."""
    rng = np.random.default_rng(4)
    for k in range(1, 7):
        C = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
        bf = sum(np.prod([C[i, s[i]] for i in range(k)]) for s in itertools.permutations(range(k)))
        assert abs(orc.per_ryser(C) - bf) <= 1e-13 * abs(bf)
        assert orc.per_ryser(np.ones((k, k))) == math.factorial(k)
        assert orc.per_ryser(np.eye(k)) == 1


def test_haf_permutation_invariance_and_homogeneity(orc):
    """Haf(P A P^T) = Haf(A) (Sec. 2.3, Appendix B); Haf(cA) = c^{n/2} Haf(A)."""
    n = 12
    A = rand_sym(n, 11)
    h = orc.haf_subset(A)
    perm = np.random.default_rng(12).permutation(n)
    assert abs(orc.haf_subset(A[np.ix_(perm, perm)]) - h) <= 1e-24 * abs(h) * 1e4
    c = 0.7 - 0.4j
    assert abs(orc.haf_subset(c * A) - c ** (n // 2) * h) <= 1e-13 * abs(h)


def test_haf_diagonal_independent(orc):
    """No perfect matching uses V(i, i) (Eq. HafMatch): the diagonal is irrelevant."""
    A = rand_sym(10, 5)
    B = A.copy()
    np.fill_diagonal(B, np.arange(10) * (1 + 2j))
    assert abs(orc.haf_subset(A) - orc.haf_subset(B)) <= 1e-20 * abs(orc.haf_subset(A))


def test_haf_laplace_expansion(orc):
    """Haf(V) = sum_u V(n,u) Haf(V without rows/cols n,u) (Appendix A)."""
    n = 10
    V = rand_sym(n, 21)
    total = 0
    for u in range(n - 1):
        keep = [i for i in range(n - 1) if i != u]
        total += V[n - 1, u] * orc.haf_subset(V[np.ix_(keep, keep)])
    h = orc.haf_subset(V)
    assert abs(total - h) <= 1e-13 * abs(h)


def test_f64_twin_error_within_kappa_bound(orc):
    """The double-precision twin stays within a small multiple of kappa*u."""
    for n, seed in ((8, 1), (12, 2), (16, 3)):
        A = rand_sym(n, seed)
        h, K = orc.haf_subset(A, return_kappa=True)
        f = orc.haf_subset_f64(A)
        assert abs(f - h) <= 4 * n * K * 2.0 ** -53


# --- kernel matrix and probabilities -----------------------------------------

def test_build_B_definition(orc):
    """B = U diag(tanh r) U^T is symmetric; with t = 1 it is unitary (Sec. 2.3)."""
    U = W.haar_unitary(12, 5)
    r = W.squeezing(12, "uniform", seed=5)
    B = orc.build_B(U, r)
    ref = np.einsum("ik,k,jk->ij", U, np.tanh(r), U)
    assert np.abs(B - ref).max() < 1e-14
    assert np.abs(B - B.T).max() < 1e-15
    Wm = orc.build_B_dd(U, np.ones(12))
    Wc = Wm[..., 0] + 1j * Wm[..., 2]
    assert np.abs(Wc @ Wc.conj().T - np.eye(12)).max() < 1e-13


def test_prob_two_photons(orc):
    """n = 2: p(1_i 1_j) = |B_ij|^2 / prod cosh r; p(2_j) = |B_jj|^2 / (2! prod cosh r)."""
    m = 6
    U = W.haar_unitary(m, 9)
    r = W.squeezing(m, "uniform", seed=9)
    B = orc.build_B(U, r)
    L = np.sum(np.log(np.cosh(r)))
    pats = [np.array([1, 4]), np.array([3, 3])]
    out = orc.prob(U, r, pats)
    assert abs(out["p"][0] - abs(B[1, 4]) ** 2 * np.exp(-L)) < 1e-14 * out["p"][0]
    assert abs(out["p"][1] - abs(B[3, 3]) ** 2 * np.exp(-L) / 2) < 1e-14 * out["p"][1]


def test_single_mode_collision(orc):
    """n photons in one mode: B_x = b J_n, Haf = b^{n/2} (n-1)!!."""
    m = 5
    U = W.haar_unitary(m, 2)
    r = W.squeezing(m, "const", value=0.8)
    B = orc.build_B(U, r)
    for n in (2, 4, 6, 8):
        out = orc.prob(U, r, [np.full(n, 2, dtype=np.int32)])
        expect = B[2, 2] ** (n // 2) * dfact(n - 1)
        assert abs(out["haf"][0] - expect) <= 1e-13 * abs(expect)
        lp = 2 * np.log(abs(expect)) - math.lgamma(n + 1) - np.sum(np.log(np.cosh(r)))
        assert abs(out["logp"][0] - lp) < 1e-12


def smss_c2(s, r):
    """|c_s(r)|^2 of a single-mode squeezed state (Sec. 2.1), 0 for odd s."""
    if s % 2:
        return 0.0
    return (1 / np.cosh(r)) * (np.tanh(r) / 2) ** s * math.factorial(s) / math.factorial(s // 2) ** 2


def test_identity_network_product_state(orc):
    """U = I (and a permutation): p(s) = prod_j |c_{s_j}(r_j)|^2 (Sec. 2.1)."""
    m = 5
    r = W.squeezing(m, "uniform", seed=1, lo=0.3, hi=1.1)
    for U, rr in ((np.eye(m), r), (np.eye(m)[[2, 0, 4, 1, 3]], r)):
        # output mode i of U receives input mode perm^{-1}(i): r seen at output i
        r_out = np.array([rr[np.argmax(np.abs(U[i]))] for i in range(m)])
        for pat in ([0, 0], [1, 1, 3, 3], [2, 2, 2, 2], [0, 0, 1, 1, 4, 4], [0, 1], [1, 1, 2]):
            x = np.array(pat, dtype=np.int32)
            s = W.pattern_to_counts(x, m)
            expect = np.prod([smss_c2(int(s[j]), r_out[j]) for j in range(m)])
            got = orc.prob(U, rr, [x])["p"][0]
            assert abs(got - expect) <= 1e-14 * max(expect, 1e-300) + (1e-300 if expect == 0 else 0)


def neg_binomial(m, n, r):
    """P_n = C((m+n)/2 - 1, n/2) tanh^n r / cosh^m r (Eq. Eqdistribution)."""
    return math.comb((m + n) // 2 - 1, n // 2) * np.tanh(r) ** n / np.cosh(r) ** m


def per_mode_Pn(r, n):
    """[z^n] prod_i sech r_i (1 - tanh^2 r_i z^2)^{-1/2}: P_n for unequal r."""
    series = np.zeros(n + 1)
    series[0] = 1.0
    for ri in r:
        t2 = np.tanh(ri) ** 2
        f = np.zeros(n + 1)
        for k in range(0, n // 2 + 1):  # (1 - a z^2)^{-1/2} = sum C(2k,k)/4^k a^k z^{2k}
            f[2 * k] = math.comb(2 * k, k) / 4 ** k * t2 ** k
        series = np.convolve(series, f)[: n + 1] / np.cosh(ri)
    return series[n]


@pytest.mark.parametrize("n", [0, 2, 4, 6])
def test_total_probability_negative_binomial(orc, n):
    """sum_{|s| = n} p(s) = P_n, identical r (Eq. Eqdistribution), m = 8."""
    m = 8
    U = W.haar_unitary(m, 0)
    r = W.squeezing(m, "const", value=0.5)
    pats = W.all_patterns(m, n)
    tot = orc.prob(U, r, pats, method="pm")["p"].sum()
    assert abs(tot - neg_binomial(m, n, 0.5)) <= 1e-12 * neg_binomial(m, n, 0.5)


def test_total_probability_per_mode_r(orc):
    """The same sum with unequal r_i against the product generating function."""
    m, n = 6, 6
    U = W.haar_unitary(m, 3)
    r = W.squeezing(m, "uniform", seed=3)
    pats = W.all_patterns(m, n)
    tot = orc.prob(U, r, pats)["p"].sum()
    ref = per_mode_Pn(r, n)
    assert abs(tot - ref) <= 1e-12 * ref


@pytest.mark.parametrize("m,n", [(4, 4), (3, 6), (5, 2)])
def test_position_basis_normalisation(orc, m, n):
    """sum_{x in [m]^n} |Haf(W_x)|^2 = f_n = n! C((m+n)/2 - 1, n/2), W = U U^T
    (Appendix A). Summed over configurations s with multiplicity n!/prod s_j!."""
    U = W.haar_unitary(m, 40 + m)
    Wdd = orc.build_B_dd(U, np.ones(m))
    pats = W.all_patterns(m, n)
    out = orc.prob(U, np.zeros(m), pats, Bdd=Wdd)  # r = 0: no cosh factor
    total = math.factorial(n) * out["p"].sum()  # p = |Haf|^2 / prod s_j!
    f_n = 1  # recurrence f_n = (n-1)(m+n-2) f_{n-2}, f_0 = 1 (Eq. Eqf)
    for k in range(2, n + 1, 2):
        f_n *= (k - 1) * (m + k - 2)
    # closed form n! C((m+n)/2 - 1, n/2), a generalised binomial when m is odd
    a = (m + n) / 2 - 1
    closed = math.factorial(n) * math.exp(math.lgamma(a + 1) - math.lgamma(n // 2 + 1) - math.lgamma(a - n // 2 + 1))
    assert abs(closed - f_n) <= 1e-12 * f_n
    assert abs(total - f_n) <= 1e-12 * f_n


def test_ws_example_paper(orc):
    """Sec. 2.3's W_s example: s = (1,1,0,2,0,0) selects rows/cols (1,2,4,4) of W;
    its Hafnian by the n = 4 expansion equals the oracle's for x = (0,1,3,3)."""
    lines = {l.split()[0]: l.split()[1:] for l in open(os.path.join(GOLDEN, "ws_example.txt"))
             if not l.startswith("#") and l.strip()}
    s = np.array([int(v) for v in lines["s"]])
    rows = [int(v) - 1 for v in lines["rows"]]
    x = np.repeat(np.arange(len(s)), s).astype(np.int32)
    assert list(x) == rows
    m = len(s)
    U = W.haar_unitary(m, 17)
    Wdd = orc.build_B_dd(U, np.ones(m))
    Wc = (Wdd[..., 0] + Wdd[..., 1]) + 1j * (Wdd[..., 2] + Wdd[..., 3])
    Ws = Wc[np.ix_(rows, rows)]
    expect = Ws[0, 1] * Ws[2, 3] + Ws[0, 2] * Ws[1, 3] + Ws[0, 3] * Ws[1, 2]
    out = orc.prob(U, np.zeros(m), [x], Bdd=Wdd)
    assert abs(out["haf"][0] - expect) <= 1e-14 * abs(expect)
    assert abs(out["p"][0] - abs(expect) ** 2 / 2) <= 1e-13 * out["p"][0]


def test_prob_methods_agree_tiny_workload(orc):
    """Tiny workload (m = 8, 4- and 2-photon patterns): subset sum vs matchings."""
    U, r, pats = W.workload("tiny_m8")
    a = orc.prob(U, r, pats, method="subset")
    b = orc.prob(U, r, pats, method="pm")
    assert np.all(np.abs(a["haf"] - b["haf"]) <= 1e-15 * np.abs(b["haf"]) + 1e-300)
    assert np.all(np.abs(a["p"] - b["p"]) <= 1e-14 * b["p"])


# --- repeated-row Hafnian (collision path; Kan's moment identity) ---------------

def expand(B, reps):
    idx = np.repeat(np.arange(len(reps)), reps)
    return np.asarray(B)[np.ix_(idx, idx)]


@pytest.mark.parametrize("seed", range(6))
def test_haf_repeated_brute_force(orc, seed):
    """haf_repeated equals the perfect-matching sum of the explicitly repeated
    matrix (brute force, Eq. HafMatch) for random complex symmetric B and
    random multiplicities with n <= 10."""
    rng = np.random.default_rng(100 + seed)
    mp = int(rng.integers(1, 5))
    reps = [int(v) for v in rng.integers(0, 4, size=mp)]
    if sum(reps) % 2:
        reps[0] += 1
    if sum(reps) > 10:
        reps = [min(v, 2) for v in reps]
        if sum(reps) % 2:
            reps[0] += 1
    B = rand_sym(mp, 200 + seed)
    ref = orc.haf_pm(expand(B, reps))
    got = orc.haf_repeated(B, reps)
    assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (reps, got, ref)


@pytest.mark.parametrize("k", range(1, 7))
def test_haf_repeated_single_mode(orc, k):
    """One mode repeated 2k times: the repeated matrix is b J_2k, so
    Haf = b^k (2k-1)!!."""
    b = 0.7 - 0.4j
    got = orc.haf_repeated(np.array([[b]]), [2 * k])
    ref = b ** k * dfact(2 * k - 1)
    assert abs(got - ref) <= 1e-13 * abs(ref)


def test_haf_repeated_collision_free_and_edges(orc):
    """All multiplicities 1: the plain Hafnian (double-double subset sum); odd n
    gives 0; a mode with multiplicity 0 is the same as leaving it out."""
    B = rand_sym(8, 31)
    ref = orc.haf_subset(B)
    assert abs(orc.haf_repeated(B, [1] * 8) - ref) <= 1e-12 * abs(ref)
    assert orc.haf_repeated(B[:3, :3], [1, 1, 1]) == 0
    B4 = rand_sym(4, 32)
    a = orc.haf_repeated(B4, [2, 0, 1, 1])
    b = orc.haf_repeated(B4[np.ix_([0, 2, 3], [0, 2, 3])], [2, 1, 1])
    assert abs(a - b) <= 1e-14 * abs(b)


def test_prob_order_and_diagonal_free(orc):
    """p(s) is a function of the configuration s alone: any order of the index
    list x gives the same Haf(W_x) (Appendix B) and the same prod_j s_j!; and no
    perfect matching uses a diagonal entry (Eq. HafMatch), so zeroing the
    diagonal of W_x leaves Haf and p unchanged, while the subset sum's terms
    (and so kappa) change. Checked against the perfect-matching oracle on
    patterns with collisions."""
    m = 7
    U = W.haar_unitary(m, 41)
    r = W.squeezing(m, "uniform", seed=41)
    rng = np.random.default_rng(41)
    pats = [np.sort(rng.choice(m, n, replace=True)).astype(np.int32) for n in (4, 6, 8, 10) for _ in range(2)]
    ref = orc.prob(U, r, pats, method="pm")
    shuffled = [rng.permutation(x).astype(np.int32) for x in pats]
    for zd in (False, True):
        out = orc.prob(U, r, shuffled, zero_diag=zd)
        assert np.all(np.abs(out["haf"] - ref["haf"]) <= 1e-15 * np.abs(ref["haf"]))
        assert np.all(np.abs(out["p"] - ref["p"]) <= 1e-14 * ref["p"])
        assert np.all(np.abs(out["logp"] - ref["logp"]) <= 1e-12 * np.abs(ref["logp"]))
    k0 = orc.prob(U, r, pats)["kappa"]
    k1 = orc.prob(U, r, pats, zero_diag=True)["kappa"]
    assert np.all(k0 > 0) and np.all(k1 > 0) and not np.allclose(k0, k1)


def _theorem1_position_sets(Wm, x, n, orc, part=0, weight_modes=None):
    """Theorem 1 in the order the library sums it (over position sets rho =
    [k] minus A, multiset weights prod alpha_v! C(m_v, alpha_v), only the sizes
    inside the theorem's ranges), from the oracle's perfect-matching Hafnians.
    part 1 / 2 keeps only the sets rho with / without position k - 1;
    weight_modes (default x) gives the modes the weights count."""
    k, m = len(x), Wm.shape[0]
    wx = x if weight_modes is None else weight_modes

    def haf(pos):
        if not pos:
            return 1.0
        if len(pos) % 2:
            return 0.0
        sel = [x[i] for i in pos]
        return orc.haf_pm(Wm[np.ix_(sel, sel)])

    def lgb(a, b):
        return math.lgamma(a + 1) - math.lgamma(b + 1) - math.lgamma(a - b + 1)

    def in_range(mu, ja, jb):
        lo = max(0, 2 * k - n)
        return ja >= lo and jb >= lo and max(0, 3 * k - ja - jb - n) <= mu <= k - max(ja, jb)

    def F(mu, ja, jb):  # F(k, mu, ja, jb) / f_n
        if not in_range(mu, ja, jb):
            return 0.0
        return math.exp(math.lgamma(n - k + 1) + lgb(0.5 * (n - k + mu + m) - 1, k - 0.5 * (ja + jb) + 0.5 * m - 1)
                        - math.lgamma(n + 1) - lgb(0.5 * (m + n) - 1, 0.5 * n))

    mult = {}
    for v in wx:
        mult[v] = mult.get(v, 0) + 1
    q = 0.0
    for c in range(0, k + 1, 2):
        mu = k - c
        need = [ja for ja in range(0, c + 1, 2) if any(in_range(mu, ja, jb) for jb in range(0, c + 1, 2))]
        for rho in itertools.combinations(range(k), c):
            if (part == 1 and k - 1 not in rho) or (part == 2 and k - 1 in rho):
                continue
            G = {ja: sum(haf(list(s)) * haf([i for i in rho if i not in s]) for s in itertools.combinations(rho, ja))
                 for ja in need}
            form = sum(F(mu, a, b) * (G[a] * np.conj(G[b])).real for a in need for b in need)
            w = 1.0
            for v, mv in mult.items():
                al = mv - sum(1 for i in rho if wx[i] == v)
                w *= math.factorial(al) * math.comb(mv, al)
            q += w * form
    return q


@pytest.mark.parametrize("m,n", [(4, 4), (3, 6), (5, 6)])
def test_theorem1_position_set_sum_equals_definition(orc, m, n):
    """The reading of Theorem 1 the library computes (the sum over position sets
    with multiset weights, terms outside the theorem's ranges never formed)
    equals the brute-force marginal of Eq. marginal_definition, sum over the
    completions of |Haf(W_x)|^2 / f_n, for prefixes with and without repeated
    modes and every prefix length."""
    U = W.haar_unitary(m, 808 + m + n)
    Wm = U @ U.T
    a = (m + n) / 2 - 1
    f_n = math.factorial(n) * math.exp(math.lgamma(a + 1) - math.lgamma(n / 2 + 1) - math.lgamma(a - n / 2 + 1))
    rng = np.random.default_rng(m * 10 + n)
    for k in range(0, n + 1):
        for trial in range(2):
            x = [1] * k if trial == 0 else [int(v) for v in rng.integers(0, m, size=k)]
            brute = 0.0
            for comp in itertools.product(range(m), repeat=n - k):
                y = x + list(comp)
                brute += abs(orc.haf_pm(Wm[np.ix_(y, y)])) ** 2
            brute /= f_n
            got = _theorem1_position_sets(Wm, x, n, orc)
            assert abs(got - brute) <= 1e-11 * abs(brute) + 1e-300, (m, n, x, got, brute)


def test_theorem1_split_by_the_new_position(orc):
    """The chain sampler's split of step k: for a candidate mode l after the
    prefix x, q(x, l) = (the sets rho that hold position k - 1, weighted by
    (x, l)) + (1 + multiplicity of l in x) * (the sets without it, weighted by
    x and a mode of its own at k - 1), since (a+1)! C(m+1, a+1) = (m+1) a! C(m, a)."""
    m, n = 4, 6
    U = W.haar_unitary(m, 909)
    Wm = U @ U.T
    for x in ([2, 0], [1, 1, 3], [0, 0, 0, 2], [3]):
        k = len(x) + 1
        s0 = _theorem1_position_sets(Wm, x + [0], n, orc, part=2, weight_modes=x + [-1])
        for l in range(m):
            full = _theorem1_position_sets(Wm, x + [l], n, orc)
            s1 = _theorem1_position_sets(Wm, x + [l], n, orc, part=1)
            split = s1 + (1 + x.count(l)) * s0
            assert abs(split - full) <= 1e-12 * abs(full) + 1e-300, (x, l, split, full, k)
