"""Pins for the split deviates: hypergeometric (Sec. 3: the number of samples
left of a split) and binomial (Sec. 4.6: the same split with replacement).

- exact pmfs from integer binomial coefficients (chi-square over many
  independent node streams), for both the inversion and the
  ratio-of-uniforms branch and every parameter reduction;
- the inversion branch returns the exact quantile of its uniform;
- the table-mountain hat really dominates the scaled pmf (the condition
  under which ratio-of-uniforms is exact), checked exhaustively on a grid;
- closed-form mean and variance at the sizes of the large runs.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

D1 = 2 * math.sqrt(2 / math.e)
D2 = 3 - 2 * math.sqrt(3 / math.e)


def hg_pmf(n, K, S):
    tot = math.comb(S, n)
    return [Fraction(math.comb(K, k) * math.comb(S - K, n - k), tot) for k in range(0, min(n, K) + 1)]


def bin_pmf(c, K, S):
    p = Fraction(K, S)
    return [math.comb(c, k) * p**k * (1 - p) ** (c - k) for k in range(c + 1)]


def chisq_p(samples, pmf):
    """Chi-square p-value of integer samples against an exact pmf, merging
    cells so that every expected count is at least 5."""
    m = len(samples)
    obs = np.bincount(np.asarray(samples), minlength=len(pmf))[: len(pmf)]
    assert obs.sum() == m, "sample outside the support"
    exp = np.array([float(p) * m for p in pmf])
    o_cells, e_cells, o_acc, e_acc = [], [], 0, 0.0
    for o, e in zip(obs, exp):
        o_acc += o
        e_acc += e
        if e_acc >= 5:
            o_cells.append(o_acc)
            e_cells.append(e_acc)
            o_acc, e_acc = 0, 0.0
    if e_acc > 0:
        if e_cells:
            o_cells[-1] += o_acc
            e_cells[-1] += e_acc
        else:
            o_cells.append(o_acc)
            e_cells.append(e_acc)
    e_cells = np.array(e_cells) * (m / np.sum(e_cells))
    if len(e_cells) < 2:
        return 1.0
    return stats.chisquare(o_cells, e_cells).pvalue


HG_CASES = [
    # (n, K, S): inversion (mean < 16) and ratio-of-uniforms, with every
    # combination of the K > S/2 and n > S/2 reductions.
    (10, 20, 50), (30, 7, 100), (70, 30, 100), (80, 90, 100), (3, 1, 4), (1, 1, 2),
    (40, 60, 100), (100, 100, 300), (500, 400, 1000), (200, 700, 1000), (900, 700, 1000),
    (62, 31, 124), (31, 31, 62),
]


@pytest.mark.parametrize("n,K,S", HG_CASES)
def test_hg_exact_pmf(oracle, n, K, S):
    m = 12000
    xs = [oracle.hg(2024, node, n, K, S) for node in range(1, m + 1)]
    assert chisq_p(xs, hg_pmf(n, K, S)) > 1e-4


BIN_CASES = [(10, 5, 10), (31, 15, 31), (50, 25, 51), (200, 100, 200), (1000, 333, 1000), (77, 38, 77), (5, 1, 3)]


@pytest.mark.parametrize("c,K,S", BIN_CASES)
def test_bin_exact_pmf(oracle, c, K, S):
    m = 12000
    xs = [oracle.binom(77, node, c, K, S) for node in range(1, m + 1)]
    assert chisq_p(xs, bin_pmf(c, K, S)) > 1e-4


def test_hg_fast_paths(oracle):
    assert oracle.hg(1, 1, 0, 5, 10) == 0
    assert oracle.hg(1, 1, 5, 0, 10) == 0
    assert oracle.hg(1, 1, 4, 10, 10) == 4
    assert oracle.hg(1, 1, 10, 4, 10) == 4
    assert oracle.binom(1, 1, 0, 5, 10) == 0
    assert oracle.binom(1, 1, 9, 0, 1) == 0


@pytest.mark.parametrize("n,K,S", [(10, 20, 50), (12, 30, 64), (5, 400, 1000)])
def test_hg_inversion_is_exact_quantile(oracle, n, K, S):
    """No reduction applies (n, K <= S/2, mean < 16): the deviate is the
    smallest k with u < F(k), u = V(value 0 of the node's stream), unless u
    sits within rounding of a boundary of the exact cdf."""
    pmf = hg_pmf(n, K, S)
    cdf = np.cumsum([float(p) for p in pmf])
    exact_cdf = []
    acc = Fraction(0)
    for p in pmf:
        acc += p
        exact_cdf.append(acc)
    for node in range(1, 800):
        u = Fraction(oracle.v_closed(oracle.value(9, 1, node, 0)))
        want = next(k for k, F in enumerate(exact_cdf) if u < F)
        got = oracle.hg(9, node, n, K, S)
        if got != want:
            assert min(abs(float(u) - c) for c in cdf) < 1e-12, (node, got, want)


def _hat_ok(logf, support, mu, var):
    """Ratio-of-uniforms with the table-mountain hat is exact iff for every k
    max(|k - alpha|, |k + 1 - alpha|) * sqrt(f(k)/f(M)) <= h/2 and f <= f(M)."""
    alpha = mu + 0.5
    h = D1 * math.sqrt(var + 0.5) + D2
    lmax = max(logf)
    worst = 0.0
    for k in support:
        g = math.exp(logf[k] - lmax)
        dist = max(abs(k - alpha), abs(k + 1 - alpha))
        worst = max(worst, dist * math.sqrt(g) / (h / 2))
    return worst


def test_hg_hat_dominates(oracle):
    """Exhaustive over a grid of (a, b, S) in the ratio-of-uniforms branch."""
    worst = 0
    for S in list(range(34, 130, 3)) + [200, 517, 1000, 4099]:
        for a in sorted({16, 20, 33, S // 4, S // 3, S // 2}):
            for b in sorted({a, S // 3, S // 2}):
                if not (1 <= a <= b <= S // 2):
                    continue
                mu = a * b / S
                if mu < 16:
                    continue
                var = mu * ((S - a) / S) * ((S - b) / (S - 1))
                logf = [math.lgamma(a + 1) - math.lgamma(k + 1) - math.lgamma(a - k + 1)
                        + math.lgamma(S - a + 1) - math.lgamma(b - k + 1) - math.lgamma(S - a - b + k + 1)
                        if b - k >= 0 else -math.inf for k in range(a + 1)]
                M = (a + 1) * (b + 1) // (S + 2)
                assert logf[M] >= max(logf) - 1e-9, (a, b, S)
                worst = max(worst, _hat_ok(logf, range(a + 1), mu, var))
    assert worst <= 1.0, worst


def test_bin_hat_dominates(oracle):
    worst = 0
    for c in list(range(32, 400, 7)) + [1000, 4096, 7630]:
        for K, S in [(1, 2), (5, 11), (50, 101), (333, 1000), (2, 5)]:
            p = K / S
            mu = c * p
            if mu < 16:
                continue
            logf = [math.lgamma(c + 1) - math.lgamma(k + 1) - math.lgamma(c - k + 1)
                    + k * math.log(p) + (c - k) * math.log1p(-p) for k in range(c + 1)]
            M = (c + 1) * K // S
            assert abs(logf[M] - max(logf)) < 1e-9, (c, K, S)
            worst = max(worst, _hat_ok(logf, range(c + 1), mu, mu * (1 - p)))
    assert worst <= 1.0, worst


@pytest.mark.parametrize("n,K,S", [(10**9, 2**49, 2**50), (7630, 2**32, 2**33), (10**6, 500000000, 10**9),
                                   (3, 2**61, 2**62)])
def test_hg_moments_large(oracle, n, K, S):
    """Mean nK/S and variance nK(S-K)(S-n)/(S^2(S-1)) at the tree's sizes."""
    m = 6000
    xs = np.array([oracle.hg(31, node, n, K, S) for node in range(1, m + 1)], dtype=float)
    mean = n * K / S
    var = n * (K / S) * ((S - K) / S) * ((S - n) / (S - 1))
    z = (xs.mean() - mean) / math.sqrt(var / m)
    assert abs(z) < 5, z
    if var > 1:
        ratio = xs.var(ddof=1) / var
        assert abs(ratio - 1) < 5 * math.sqrt(2 / (m - 1)), ratio


@pytest.mark.parametrize("c,K,S", [(10**9, 2**39, 2**40), (7630, 2**21, 2**22), (10**9, 3, 7)])
def test_bin_moments_large(oracle, c, K, S):
    m = 6000
    xs = np.array([oracle.binom(32, node, c, K, S) for node in range(1, m + 1)], dtype=float)
    p = K / S
    z = (xs.mean() - c * p) / math.sqrt(c * p * (1 - p) / m)
    assert abs(z) < 5, z
    ratio = xs.var(ddof=1) / (c * p * (1 - p))
    assert abs(ratio - 1) < 5 * math.sqrt(2 / (m - 1)), ratio


def _window_ratio(logf, lo, hi, alpha, h, lmode):
    step = max(1, (hi - lo) // 20000)
    worst = 0.0
    for k in range(lo, hi + 1, step):
        g = math.exp(logf(k) - lmode)
        worst = max(worst, max(abs(k - alpha), abs(k + 1 - alpha)) * math.sqrt(g) / (h / 2))
    return worst


@pytest.mark.parametrize("c,p", [(3000, 0.5), (10**5, 0.5), (10**7, 0.5), (10**6, 0.1), (10**6, 0.01)])
def test_bin_hat_dominates_large(c, p):
    """Away from the centre the scaled pmf decays like a normal density whose
    envelope the hat matches asymptotically; the ratio stays below 1 (its
    maximum lies within 8 standard deviations of the centre)."""
    mu, var = c * p, c * p * (1 - p)
    alpha, h, sig = mu + 0.5, D1 * math.sqrt(var + 0.5) + D2, math.sqrt(var)
    M = int((c + 1) * p)
    logf = lambda k: (-math.lgamma(k + 1) - math.lgamma(c - k + 1) + k * math.log(p) + (c - k) * math.log1p(-p))
    lo, hi = max(0, int(alpha - 8 * sig) - 2), min(c, int(alpha + 8 * sig) + 2)
    assert _window_ratio(logf, lo, hi, alpha, h, max(logf(M), logf(min(c, M + 1)))) <= 1.0


@pytest.mark.parametrize("n,K,S", [(7630, 2**32, 2**33), (10**5, 5 * 10**5, 10**6), (10**6, 2**29, 2**30)])
def test_hg_hat_dominates_large(n, K, S):
    a, b = min(n, K), max(n, K)
    mu = a * b / S
    var = mu * ((S - a) / S) * ((S - b) / (S - 1))
    alpha, h, sig = mu + 0.5, D1 * math.sqrt(var + 0.5) + D2, math.sqrt(var)
    M = (a + 1) * (b + 1) // (S + 2)
    logf = lambda k: (-math.lgamma(k + 1) - math.lgamma(a - k + 1) - math.lgamma(b - k + 1)
                      - math.lgamma(S - a - b + k + 1))
    lo, hi = max(0, int(alpha - 8 * sig) - 2), min(a, int(alpha + 8 * sig) + 2)
    assert _window_ratio(logf, lo, hi, alpha, h, logf(M)) <= 1.0


@pytest.mark.parametrize("n,K,S", [(32, 32, 64), (16, 63, 64), (40, 40, 100), (17, 1000, 1063)])
def test_hg_exact_pmf_low_variance_rou(oracle, n, K, S):
    """The ratio-of-uniforms branch at its smallest variances (mean just
    above 16), where the hat's additive constant matters most; many draws."""
    m = 60000
    xs = [oracle.hg(4242, node, n, K, S) for node in range(1, m + 1)]
    assert chisq_p(xs, hg_pmf(n, K, S)) > 1e-4


@pytest.mark.parametrize("c,K,S", [(32, 1, 2), (33, 16, 33), (160, 1, 10)])
def test_bin_exact_pmf_low_variance_rou(oracle, c, K, S):
    m = 60000
    xs = [oracle.binom(4343, node, c, K, S) for node in range(1, m + 1)]
    assert chisq_p(xs, bin_pmf(c, K, S)) > 1e-4


def _first_trial_checks(oracle, seed, logf, mu, var, M, top, draw, nodes):
    """For each node, redo the first ratio-of-uniforms trial in exact
    arithmetic: X = alpha + h (V - 0.5) / U with h from the hat's definition,
    accept iff 2 ln U <= ln f(k) - ln f(M).  Where it clearly accepts, the
    oracle must return k = floor(X).  Returns the number of checked nodes."""
    import mpmath
    alpha = mu + 0.5
    h = D1 * math.sqrt(var + 0.5) + D2
    checked = 0
    for node in nodes:
        U = oracle.u_open(oracle.value(seed, 1, node, 0))
        V = oracle.v_closed(oracle.value(seed, 1, node, 1))
        X = alpha + h * (V - 0.5) / U
        if X < 0 or X >= top + 1 or abs(X - round(X)) < 1e-9:
            continue
        k = int(math.floor(X))
        T = logf(k) - logf(M)
        lhs = 2 * mpmath.log(mpmath.mpf(U))
        if lhs < T - mpmath.mpf(1e-9):
            assert draw(node) == k, (node, k)
            checked += 1
    return checked


@pytest.mark.parametrize("n,K,S", [(32, 32, 64), (100, 100, 300), (7630, 2**32, 2**33), (10**6, 2**29, 2**30)])
def test_hg_rou_first_trial_exact(oracle, n, K, S):
    import mpmath
    a, b = min(n, K), max(n, K)
    mu = a * b / S
    var = mu * ((S - a) / S) * ((S - b) / (S - 1))
    M = (a + 1) * (b + 1) // (S + 2)
    lg = lambda x: mpmath.loggamma(mpmath.mpf(x) + 1)
    logf = lambda k: -lg(k) - lg(a - k) - lg(b - k) - lg(S - a - b + k)
    nodes = range(1, 1500)
    got = _first_trial_checks(oracle, 77, logf, mu, var, M, a, lambda v: oracle.hg(77, v, n, K, S), nodes)
    assert got > len(nodes) // 3


@pytest.mark.parametrize("c,K,S", [(32, 1, 2), (1000, 333, 1000), (10**9, 2**39, 2**40)])
def test_bin_rou_first_trial_exact(oracle, c, K, S):
    import mpmath
    p = mpmath.mpf(K) / S
    mu = c * (K / S)
    var = mu * (1 - K / S)
    M = (c + 1) * K // S
    lg = lambda x: mpmath.loggamma(mpmath.mpf(x) + 1)
    logf = lambda k: -lg(k) - lg(c - k) + k * mpmath.log(p) + (c - k) * mpmath.log(1 - p)
    nodes = range(1, 1500)
    got = _first_trial_checks(oracle, 78, logf, mu, var, M, c, lambda v: oracle.binom(78, v, c, K, S), nodes)
    assert got > len(nodes) // 3
