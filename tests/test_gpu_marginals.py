"""Theorem 1 marginals and the chain-rule sampler (Sec. 3.3-3.4, Algorithm 1)
on the GPU, against the plain definition q_n(x_1..x_k) = sum over completions
of |Haf(W_x)|^2 / f_n computed by the oracle."""
import itertools
import math

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


def f_n(m, n):
    a = (m + n) / 2 - 1
    return math.factorial(n) * math.exp(math.lgamma(a + 1) - math.lgamma(n / 2 + 1) - math.lgamma(a - n / 2 + 1))


def brute_marginals(orc, U, prefixes, n):
    """sum over x_{k+1..n} of |Haf(W_x)|^2 / f_n, W = U U^T (oracle, double-double)."""
    m = U.shape[0]
    Wdd = orc.build_B_dd(U, np.ones(m))
    out = []
    for x in prefixes:
        comps = [np.array(list(x) + list(c), dtype=np.int32) for c in itertools.product(range(m), repeat=n - len(x))]
        h = orc.prob(U, np.zeros(m), comps, method="pm", Bdd=Wdd)["haf"]
        out.append(np.sum(np.abs(h) ** 2) / f_n(m, n))
    return np.array(out)


@pytest.mark.parametrize("m,n,r", [(4, 4, 0.7), (6, 4, 0.5), (4, 6, 0.9), (5, 4, 0.6)])
def test_marginals_vs_definition(gbs, orc, m, n, r):
    U = W.haar_unitary(m, 50 + m + n)
    K = gbs.build_kernel(U, np.full(m, r))
    rng = np.random.default_rng(m * 7 + n)
    for k in range(0, n + 1):
        prefixes = [rng.integers(0, m, size=k) for _ in range(3)]
        if k >= 2:
            prefixes.append(np.full(k, 1))  # all photons in one mode
        got = gbs.marginal_batch(K, np.array(prefixes).reshape(len(prefixes), k), n)
        ref = brute_marginals(orc, U, prefixes, n)
        assert np.all(np.abs(got - ref) <= 1e-10 * np.abs(ref) + 1e-300), (k, got, ref)


def test_marginal_limits_and_consistency(gbs, orc):
    """k = 0 gives 1; k = n gives q_n(x) = |Haf(W_x)|^2 / f_n (Eq. EqDisE); summing
    over the last position recovers the shorter prefix (Eq. marginal_definition)."""
    m, n = 12, 6
    U = W.haar_unitary(m, 12)
    K = gbs.build_kernel(U, np.full(m, 0.8814))
    assert abs(gbs.marginal_batch(K, np.zeros((1, 0), np.int32), n)[0] - 1.0) <= 1e-12
    x = np.array([[3, 7, 7, 0, 11, 2]], np.int32)
    Wm = U @ U.T
    ref = abs(orc.haf_pm(Wm[np.ix_(x[0], x[0])])) ** 2 / f_n(m, n)
    assert abs(gbs.marginal_batch(K, x, n)[0] - ref) <= 1e-10 * ref
    for pre in ([5], [5, 9], [5, 9, 9], [4, 1, 8, 10]):
        whole = gbs.marginal_batch(K, np.array([pre], np.int32), n)[0]
        ext = gbs.marginal_batch(K, np.array([pre + [l] for l in range(m)], np.int32), n)
        assert abs(ext.sum() - whole) <= 1e-11 * whole, (pre, ext.sum(), whole)


def test_marginals_reject_unequal_squeezing(gbs):
    K = gbs.build_kernel(W.haar_unitary(6, 1), np.linspace(0.3, 0.8, 6))
    with pytest.raises(gbs.GbsError) as ei:
        gbs.marginal_batch(K, np.array([[1, 2]], np.int32), 4)
    assert ei.value.code == -1


def test_chain_sampler_distribution(gbs, orc):
    """Algorithm 1 samples follow p_n(s) = N_p q_n(x) (Sec. 3.2): the configuration
    frequencies of 1500 chain samples against the oracle's p_n(s)."""
    m, n = 5, 4
    U = W.haar_unitary(m, 77)
    K = gbs.build_kernel(U, np.full(m, 0.6))
    rng = np.random.default_rng(4)
    draws = 1500
    counts = {}
    for _ in range(draws):
        x = gbs.sample_chain(K, n, rng.random(n))
        key = tuple(sorted(int(v) for v in x))
        counts[key] = counts.get(key, 0) + 1
    configs = W.all_patterns(m, n)
    Wdd = orc.build_B_dd(U, np.ones(m))
    h = orc.prob(U, np.zeros(m), configs, method="pm", Bdd=Wdd)["haf"]
    pn = []
    for c, hv in zip(configs, h):
        s = W.pattern_to_counts(c, m)
        Np = math.factorial(n) / np.prod([math.factorial(int(v)) for v in s])
        pn.append(Np * abs(hv) ** 2 / f_n(m, n))
    pn = np.array(pn)
    assert abs(pn.sum() - 1.0) < 1e-10  # the p_n(s) form a distribution
    freq = np.array([counts.get(tuple(int(v) for v in c), 0) for c in configs]) / draws
    tv = 0.5 * np.abs(freq - pn).sum()
    expected = 0.5 * np.sqrt(2 / (np.pi * draws)) * np.sum(np.sqrt(pn * (1 - pn)))
    assert tv <= 1.5 * expected, (tv, expected)


def test_end_to_end_sample(gbs):
    """gbs_sample (Sec. 3, Steps 1-3): the photon number of every draw is the
    inverse-CDF pick of P_n restricted to n <= n_max (Eq. Eqdistribution), the
    photons are then placed by Algorithm 1, the same uniforms give the same
    sample, and the frequencies of n follow the truncated P_n."""
    m, r, n_max = 5, 0.6, 4
    U = W.haar_unitary(m, 91)
    K = gbs.build_kernel(U, np.full(m, r))
    P = gbs.photon_number_dist(K, n_max)
    Pe = np.array([P[v] if v % 2 == 0 else 0.0 for v in range(n_max + 1)])
    cum = np.cumsum(Pe)
    rng = np.random.default_rng(11)
    draws = 600
    counts = np.zeros(n_max + 1)
    for _ in range(draws):
        u = rng.random(n_max + 1)
        x = gbs.sample(K, n_max, u)
        n = len(x)
        assert n == int(np.searchsorted(cum, u[0] * cum[-1], side="right"))
        assert n % 2 == 0 and np.all((x >= 0) & (x < m))
        if n:
            assert np.array_equal(x, gbs.sample_chain(K, n, u[1:n + 1]))
        counts[n] += 1
    pt = Pe / Pe.sum()
    tv = 0.5 * np.abs(counts / draws - pt).sum()
    expected = 0.5 * np.sqrt(2 / (np.pi * draws)) * np.sum(np.sqrt(pt * (1 - pt)))
    assert tv <= 2.0 * expected, (tv, expected, counts, pt)
    u = np.full(n_max + 1, 0.3)
    assert np.array_equal(gbs.sample(K, n_max, u), gbs.sample(K, n_max, u))
    assert len(gbs.sample(K, n_max, np.zeros(n_max + 1))) == 0  # u_0 = 0 picks n = 0 (P_0 > 0)
    with pytest.raises(gbs.GbsError) as ei:
        gbs.sample(gbs.build_kernel(U, np.linspace(0.3, 0.8, m)), n_max, u)
    assert ei.value.code == -1


def test_chain_sampler_cache_matches_plain_chain(gbs):
    """The chain sampler keeps the sampled prefix's sub-Hafnians across steps
    (the exponential-space variant, Appendix D) and computes only the new
    ones; its samples equal a plain chain whose every step recomputes all
    conditional weights with gbs_marginal_batch (inverse CDF in mode order)."""
    m, n = 7, 8
    U = W.haar_unitary(m, 123)
    K = gbs.build_kernel(U, np.full(m, 0.7))
    rng = np.random.default_rng(5)
    for _ in range(12):
        u = rng.random(n)
        got = gbs.sample_chain(K, n, u)
        x = []
        for k in range(1, n + 1):
            pre = np.array([x + [l] for l in range(m)], np.int32)
            w = np.maximum(gbs.marginal_batch(K, pre, n), 0.0)
            c = np.cumsum(w)
            x.append(int(min(np.searchsorted(c, u[k - 1] * c[-1], side="right"), m - 1)))
        assert list(got) == x, (list(got), x)


def brute_marginals_subset(orc, U, prefixes, n):
    """The plain definition with the oracle's double-double subset sum (pinned
    against perfect matchings) for the longer lists."""
    m = U.shape[0]
    Wdd = orc.build_B_dd(U, np.ones(m))
    out = []
    for x in prefixes:
        comps = [np.array(list(x) + list(c), dtype=np.int32) for c in itertools.product(range(m), repeat=n - len(x))]
        h = orc.prob(U, np.zeros(m), comps, Bdd=Wdd)["haf"]
        out.append(np.sum(np.abs(h) ** 2) / f_n(m, n))
    return np.array(out)


@pytest.mark.parametrize("m,n,ks", [(3, 14, (12, 13, 14)), (14, 14, (12, 13)), (4, 16, (13, 14)), (2, 20, (18, 19, 20))])
def test_marginals_long_prefixes_vs_definition(gbs, orc, m, n, ks):
    """Prefixes of 12 to 20 photons (beyond the nested sums' reach): with many
    repeated modes (m = 2..4, where the multiset weights w(rho) carry the sum) and
    without any (m = 14, one prefix of distinct modes), against the brute-force
    marginal of Eq. marginal_definition."""
    U = W.haar_unitary(m, 300 + m + n)
    K = gbs.build_kernel(U, np.full(m, 0.75))
    rng = np.random.default_rng(m * 31 + n)
    for k in ks:
        if m >= k:
            prefixes = [rng.permutation(m)[:k] for _ in range(2)]
        else:
            prefixes = [rng.integers(0, m, size=k) for _ in range(3)]
        got = gbs.marginal_batch(K, np.array(prefixes).reshape(len(prefixes), k), n)
        ref = brute_marginals_subset(orc, U, prefixes, n)
        assert np.all(np.abs(got - ref) <= 1e-10 * np.abs(ref) + 1e-300), (k, got, ref)


def test_chain_sampler_n12_matches_plain_chain(gbs):
    """A 12-photon chain sample (Algorithm 1) with the Appendix D cache equals
    the chain that recomputes every conditional weight with gbs_marginal_batch."""
    m, n = 9, 12
    U = W.haar_unitary(m, 321)
    K = gbs.build_kernel(U, np.full(m, 0.8))
    rng = np.random.default_rng(6)
    for _ in range(3):
        u = rng.random(n)
        got = gbs.sample_chain(K, n, u)
        x = []
        for k in range(1, n + 1):
            pre = np.array([x + [l] for l in range(m)], np.int32)
            w = np.maximum(gbs.marginal_batch(K, pre, n), 0.0)
            c = np.cumsum(w)
            x.append(int(min(np.searchsorted(c, u[k - 1] * c[-1], side="right"), m - 1)))
        assert list(got) == x, (list(got), x)


@pytest.mark.parametrize("m,n,seed", [(40, 16, 11), (24, 20, 12)])
def test_chain_sampler_long_matches_plain_chain(gbs, m, n, seed):
    """16- and 20-photon chain samples (the paper's 18-20 photon regime, with
    collisions at m = 24): the cached chain, whose new sub-Hafnians come from
    the row expansion, picks the same modes as the chain that recomputes every
    conditional weight with gbs_marginal_batch (batched subset sums)."""
    U = W.haar_unitary(m, 900 + seed)
    K = gbs.build_kernel(U, np.full(m, 0.8814))
    rng = np.random.default_rng(seed)
    for _ in range(2):
        u = rng.random(n)
        got = gbs.sample_chain(K, n, u)
        x = []
        for k in range(1, n + 1):
            pre = np.array([x + [l] for l in range(m)], np.int32)
            w = np.maximum(gbs.marginal_batch(K, pre, n), 0.0)
            c = np.cumsum(w)
            x.append(int(min(np.searchsorted(c, u[k - 1] * c[-1], side="right"), m - 1)))
        assert list(got) == x, (list(got), x)


@pytest.mark.parametrize("m,n,count", [(30, 12, 8), (6, 12, 6), (40, 16, 3), (40, 16, 64)])
def test_chain_batch_equals_single_samples(gbs, m, n, count):
    """Samples advanced together (one launch sequence for all of them) equal
    the same samples drawn one at a time, with and without collisions. At 64
    samples of 16 photons the middle steps are heavy enough that the sum over
    the sets without the new photon is formed once per sample and shared by
    its candidates; one at a time it is formed per candidate."""
    U = W.haar_unitary(m, 700 + m + n)
    K = gbs.build_kernel(U, np.full(m, 0.7))
    u = np.random.default_rng(m + n).random((count, n))
    got = gbs.sample_chain_batch(K, n, u)
    assert got.shape == (count, n)
    for s in range(count):
        assert list(got[s]) == list(gbs.sample_chain(K, n, u[s])), s
    assert gbs.sample_chain_batch(K, n, np.zeros((0, n))).shape == (0, n)


def test_chain_batch_distribution(gbs, orc):
    """40,000 batched Algorithm 1 samples at m = 6, n = 6 (all 462
    configurations, collisions included) follow the oracle's p_n(s): total
    variation within 1.5 times its expectation under exact sampling."""
    m, n = 6, 6
    U = W.haar_unitary(m, 606)
    K = gbs.build_kernel(U, np.full(m, 0.7))
    draws = 40000
    x = gbs.sample_chain_batch(K, n, np.random.default_rng(66).random((draws, n)))
    counts = {}
    for row in x:
        key = tuple(sorted(int(v) for v in row))
        counts[key] = counts.get(key, 0) + 1
    configs = W.all_patterns(m, n)
    Wdd = orc.build_B_dd(U, np.ones(m))
    h = orc.prob(U, np.zeros(m), configs, method="pm", Bdd=Wdd)["haf"]
    pn = []
    for c, hv in zip(configs, h):
        s = W.pattern_to_counts(c, m)
        Np = math.factorial(n) / np.prod([math.factorial(int(v)) for v in s])
        pn.append(Np * abs(hv) ** 2 / f_n(m, n))
    pn = np.array(pn)
    assert len(configs) == 462 and abs(pn.sum() - 1.0) < 1e-10
    assert sum(counts.values()) == draws and set(counts) <= {tuple(int(v) for v in c) for c in configs}
    freq = np.array([counts.get(tuple(int(v) for v in c), 0) for c in configs]) / draws
    tv = 0.5 * np.abs(freq - pn).sum()
    expected = 0.5 * np.sqrt(2 / (np.pi * draws)) * np.sum(np.sqrt(pn * (1 - pn)))
    assert tv <= 1.5 * expected, (tv, expected)


def test_sample_batch_equals_single_samples(gbs):
    """gbs_sample_batch: each row equals gbs_sample with the same uniforms
    (photon number from the truncated P_n, then the chain of that n, samples of
    one n advanced together); empty batches and n = 0 rows work."""
    m, r, n_max = 9, 0.9, 8
    K = gbs.build_kernel(W.haar_unitary(m, 92), np.full(m, r))
    u = np.random.default_rng(12).random((60, n_max + 1))
    u[3, 0] = 0.0  # n = 0
    got = gbs.sample_batch(K, n_max, u)
    assert len(got) == 60 and len(got[3]) == 0
    assert len({len(x) for x in got}) >= 3  # several photon numbers in one batch
    for s in range(60):
        assert np.array_equal(got[s], gbs.sample(K, n_max, u[s])), s
    assert gbs.sample_batch(K, n_max, np.zeros((0, n_max + 1))) == []


@pytest.mark.parametrize("m", [1, 2])
def test_chain_sampler_one_and_two_modes(gbs, m):
    """Every photon in one of one or two modes: the repeated-mode weights carry
    the whole sum. One mode gives x = 0...0; two modes equal the plain chain."""
    n = 10
    U = W.haar_unitary(m, 5 + m)
    K = gbs.build_kernel(U, np.full(m, 0.8))
    u = np.random.default_rng(m).random((4, n))
    got = gbs.sample_chain_batch(K, n, u)
    if m == 1:
        assert np.all(got == 0)
        return
    for s in range(4):
        x = []
        for k in range(1, n + 1):
            pre = np.array([x + [l] for l in range(m)], np.int32)
            w = np.maximum(gbs.marginal_batch(K, pre, n), 0.0)
            c = np.cumsum(w)
            x.append(int(min(np.searchsorted(c, u[s, k - 1] * c[-1], side="right"), m - 1)))
        assert list(got[s]) == x, (list(got[s]), x)


def test_marginal_batch_beyond_grid_extent(gbs):
    """70,000 prefixes (more than one launch's 65,535): every one equals the
    same prefix in a small batch, so the chunks and their counters are right."""
    m, n = 12, 6
    K = gbs.build_kernel(W.haar_unitary(m, 71), np.full(m, 0.7))
    rng = np.random.default_rng(70)
    base = rng.integers(0, m, size=(64, 2)).astype(np.int32)
    ref = gbs.marginal_batch(K, base, n)
    big = np.tile(base, (70000 // 64 + 1, 1))[:70000]
    got = gbs.marginal_batch(K, big, n)
    assert np.array_equal(got, ref[np.arange(70000) % 64])


def test_chain_batch_across_sample_groups(gbs):
    """300 samples of 20 photons span two groups (256 caches of 2^20 entries
    fit in one): samples on both sides of the boundary equal single draws."""
    m, n = 22, 20
    K = gbs.build_kernel(W.haar_unitary(m, 72), np.full(m, 0.8))
    u = np.random.default_rng(72).random((300, n))
    got = gbs.sample_chain_batch(K, n, u)
    for s in (0, 1, 255, 256, 257, 299):
        assert list(got[s]) == list(gbs.sample_chain(K, n, u[s])), s


def test_chain_sampler_many_modes(gbs):
    """m = 2000 modes, 6 photons: the draw's 32 lanes each scan 63 modes and a
    step has 2000 candidates; samples equal the chain recomputed with
    gbs_marginal_batch."""
    m, n = 2000, 6
    K = gbs.build_kernel(W.haar_unitary(m, 2000), np.full(m, 0.6))
    u = np.random.default_rng(2000).random((3, n))
    got = gbs.sample_chain_batch(K, n, u)
    for s in range(3):
        x = []
        for k in range(1, n + 1):
            pre = np.array([x + [l] for l in range(m)], np.int32)
            w = np.maximum(gbs.marginal_batch(K, pre, n), 0.0)
            c = np.cumsum(w)
            x.append(int(min(np.searchsorted(c, u[s, k - 1] * c[-1], side="right"), m - 1)))
        assert list(got[s]) == x, (list(got[s]), x)
