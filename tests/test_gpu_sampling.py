"""Sampling rows on the GPU: photon-number distribution (Sec. 3.1, Eq.
Eqdistribution) and the brute-force configuration sampler (Appendix I)."""
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


def neg_binomial(m, n, r):
    """P_n = C((m+n)/2 - 1, n/2) tanh^n r / cosh^m r (generalised binomial), 0 for odd n."""
    if n % 2:
        return 0.0
    a = (m + n) / 2 - 1
    lc = math.lgamma(a + 1) - math.lgamma(n // 2 + 1) - math.lgamma(a - n // 2 + 1)
    return math.exp(lc + n * math.log(math.tanh(r)) - m * math.log(math.cosh(r)))


def per_mode_Pn(r, n_max):
    """[z^n] prod_i sech r_i (1 - tanh^2 r_i z^2)^{-1/2}, n = 0..n_max."""
    series = np.zeros(n_max + 1)
    series[0] = 1.0
    for ri in r:
        t2 = np.tanh(ri) ** 2
        f = np.zeros(n_max + 1)
        for k in range(0, n_max // 2 + 1):
            f[2 * k] = math.comb(2 * k, k) / 4 ** k * t2 ** k
        series = np.convolve(series, f)[: n_max + 1] / np.cosh(ri)
    return series


@pytest.mark.parametrize("r", [0.3423, 0.8814])
def test_photon_number_identical_r(gbs, r):
    """The paper's Fig. DisPhotons setting: m = 36 squeezed modes."""
    m = 36
    K = gbs.build_kernel(W.haar_unitary(m, 3), np.full(m, r))
    P = gbs.photon_number_dist(K, 80)
    for n in range(81):
        ref = neg_binomial(m, n, r)
        assert abs(P[n] - ref) <= 1e-12 * max(ref, 1e-300) + (1e-300 if ref == 0 else 0), (n, P[n], ref)
    # the truncated distribution carries (almost) all the probability
    assert abs(P.sum() - 1.0) < (1e-6 if r < 0.5 else 2e-2)


def test_photon_number_per_mode_r(gbs):
    m = 24
    r = W.squeezing(m, "uniform", seed=8, lo=0.2, hi=1.1)
    K = gbs.build_kernel(W.haar_unitary(m, 8), r)
    P = gbs.photon_number_dist(K, 60)
    ref = per_mode_Pn(r, 60)
    assert np.all(np.abs(P - ref) <= 1e-12 * ref + 1e-300)


@pytest.mark.parametrize("m,n,rk", [(16, 2, "c"), (16, 4, "c"), (16, 6, "c"), (10, 6, "u"), (6, 8, "u")])
def test_bruteforce_total_is_Pn(gbs, m, n, rk):
    """Sum of p over every n-photon configuration = P_n (Sec. 2.2)."""
    r = np.full(m, 0.5) if rk == "c" else W.squeezing(m, "uniform", seed=m + n)
    K = gbs.build_kernel(W.haar_unitary(m, 20 + m), r)
    _, total = gbs.sample_bruteforce(K, n, np.zeros(0))
    ref = neg_binomial(m, n, 0.5) if rk == "c" else per_mode_Pn(r, n)[n]
    assert abs(total - ref) <= 1e-11 * ref, (total, ref)


def colex_multisets(m, n):
    """All n-element multisets of {0..m-1} in colex order of c_j = x_j + j."""
    combs = list(itertools.combinations(range(m + n - 1), n))
    combs.sort(key=lambda c: tuple(reversed(c)))
    return [np.array([c[j] - j for j in range(n)], dtype=np.int32) for c in combs]


def test_bruteforce_sampler_paper_check(gbs, orc):
    """Sec. 3.5's check at n = 4, m = 16 with 400,000 draws: every draw is the
    inverse-CDF pick of the oracle's probabilities (same colex order), and the
    empirical frequencies agree with p_n(s) = p(s) / P_n."""
    m, n = 16, 4
    U = W.haar_unitary(m, 16)
    r = np.full(m, 0.5)
    K = gbs.build_kernel(U, r)
    rng = np.random.default_rng(2019)
    u = rng.random(400000)
    pats, total = gbs.sample_bruteforce(K, n, u)
    configs = colex_multisets(m, n)
    ref = orc.prob(U, r, configs, method="pm")["p"]
    cum = np.cumsum(ref)
    assert abs(total - cum[-1]) <= 1e-12 * cum[-1]
    pick = np.searchsorted(cum, u * cum[-1], side="right")
    pick = np.minimum(pick, len(configs) - 1)
    lookup = {tuple(c): i for i, c in enumerate(configs)}
    got = np.array([lookup[tuple(p)] for p in pats])
    exact = np.mean(got == pick)
    assert exact >= 0.9999 and np.all(np.abs(got - pick) <= 1), exact
    freq = np.bincount(got, minlength=len(configs)) / len(u)
    tv = 0.5 * np.abs(freq - ref / cum[-1]).sum()
    expected = 0.5 * np.sqrt(2 / (np.pi * len(u))) * np.sum(np.sqrt(ref / cum[-1] * (1 - ref / cum[-1])))
    assert tv <= 1.3 * expected, (tv, expected)
