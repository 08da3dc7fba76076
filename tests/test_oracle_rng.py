"""Pins of the oracle's random-number and JIT-connectivity routines (Appendix C).

What pins what:
* Philox4x32-10 block       -> published known-answer vectors (tests/golden).
* SplitMix64 output         -> published known answers (tests/golden).
* gap range K               -> closed form: p = 2/(K+1) must give back K.
* gap distribution U[1,K]   -> range, mean (K+1)/2, chi-square uniformity.
* realised probability      -> mean row length n_post * 2/(K+1).
* column coverage           -> exact renewal density of the gap process (first
                               target at U_0 - 1), column by column.
* weight streams            -> uniform range/moments, normal moments + KS test.
* per-row reproducibility   -> a row does not depend on which other rows fire.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as orc
from paper_2311_05106_gb300 import workloads as wl


def test_philox_known_answers(golden):
    for row in golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = orc.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_splitmix64_known_answers(golden):
    for row in golden("splitmix64_kat.txt"):
        assert orc.splitmix64(int(row[0]), int(row[1])) == int(row[2], 16)


def test_projection_seeds_distinct():
    s = 2024
    assert orc.projection_seed(s, 0) == orc.splitmix64(s, 0)
    assert orc.projection_seed(s, 1) == orc.splitmix64(s, 1)
    assert orc.projection_seed(s, 0) != orc.projection_seed(s, 1)


@pytest.mark.parametrize("K", [1, 2, 3, 19, 99, 199, 999, 1999, 9999, 99999])
def test_jit_K_inverts_expectation(K):
    # E[U[1,K]] = (K+1)/2 = 1/p  <=>  p = 2/(K+1)
    assert orc.jit_K(2.0 / (K + 1)) == K


@pytest.mark.parametrize("N", [4000, 40000, 400000, 4000000])
def test_jit_K_scaled_network(N):
    # p = 80/N  ->  2/p - 1 = N/40 - 1 exactly
    assert orc.jit_K(80.0 / N) == N // 40 - 1


def test_jit_K_floor_and_ceil_agree_when_integral_and_clamp():
    assert orc.jit_K(1.0) == 1          # 2/p - 1 = 1
    assert orc.jit_K(1.5) == 1          # 2/p - 1 = 1/3 -> ceil 1
    assert orc.jit_K(0.3) == math.ceil(2 / 0.3 - 1)


def _gaps_of_row(seed, K, row, n_post):
    cols, _ = orc.jit_row(seed, K, row, n_post)
    return np.diff(np.concatenate([[-1], cols.astype(np.int64)]))


def test_gap_distribution_uniform():
    K = 99
    gaps = np.concatenate([_gaps_of_row(123, K, r, 200000) for r in range(20)])
    assert gaps.min() >= 1 and gaps.max() <= K
    n = len(gaps)
    mean_sd = math.sqrt((K * K - 1) / 12.0 / n)
    assert abs(gaps.mean() - (K + 1) / 2) < 5 * mean_sd
    hist = np.bincount(gaps, minlength=K + 1)[1:]
    chi2, pval = stats.chisquare(hist)
    assert pval > 1e-4


@pytest.mark.parametrize("p", [0.02, 0.1, 0.001])
def test_realised_connection_probability(p):
    K = orc.jit_K(p)
    n_post = 20000
    rows = 400 if p >= 0.01 else 2000
    lens = orc.jit_row_lengths(77, K, rows, n_post)
    p_real = 2.0 / (K + 1)
    mean = lens.mean() / n_post
    # each row length ~ n_post / E[gap]; the between-row sd is below sqrt(n_post p)
    sd = math.sqrt(n_post * p_real) / n_post / math.sqrt(rows)
    assert abs(mean - p_real) < 6 * sd + 1.0 / n_post


def _renewal_density(K, n_post):
    """P(column q is a target) for targets q_0 = U_0 - 1, q_{k+1} = q_k + U_{k+1},
    U ~ U[1, K]: u(q) = P(U_0 = q + 1) + sum_g P(U = g) u(q - g)."""
    u = np.zeros(n_post)
    for q in range(n_post):
        acc = (1.0 / K) if q + 1 <= K else 0.0
        lo = max(0, q - K)
        acc += u[lo:q].sum() / K
        u[q] = acc
    return u


def test_targets_follow_renewal_density():
    """Columns are hit with the exact density of the gap process: about half of p
    at column 0, converging to 2/(K+1) after a few K (the generator is an
    approximation of Bernoulli(p), Appendix C)."""
    K = orc.jit_K(0.05)
    n_post = 400
    rows = 4000
    counts = np.zeros(n_post, np.int64)
    for r in range(rows):
        c, _ = orc.jit_row(5, K, r, n_post)
        assert np.all(np.diff(c) >= 1)          # strictly increasing: no duplicate synapse
        assert c.min(initial=0) >= 0 and c.max(initial=0) < n_post
        counts += np.bincount(c, minlength=n_post)
    u = _renewal_density(K, n_post)
    assert abs(u[-1] - 2.0 / (K + 1)) < 1e-3
    expect = rows * u
    # each column's count is a sum of independent Bernoulli rows
    z = (counts - expect) / np.sqrt(expect * (1 - u))
    assert np.abs(z).max() < 5.0
    chi2 = float((z ** 2).sum())
    assert stats.chi2.sf(chi2, n_post) > 1e-4
    # a first target at U_0 (not U_0 - 1) would shift the density by one column
    shifted = rows * np.concatenate([[0.0], u[:-1]])
    z_bad = (counts[:K] - shifted[:K]) / np.sqrt(np.maximum(shifted[:K], 1.0))
    assert np.abs(z_bad).max() > 5.0


def test_uniform_weights():
    vals = np.concatenate([orc.jit_row(9, 19, r, 5000, orc.W_UNIFORM, 0.2, 0.7)[1] for r in range(40)])
    assert vals.min() >= 0.2 and vals.max() < 0.7
    assert abs(vals.mean() - 0.45) < 5 * 0.5 / math.sqrt(12 * len(vals))
    ks = stats.kstest((vals - 0.2) / 0.5, "uniform")
    assert ks.pvalue > 1e-4


def test_normal_weights():
    vals = np.concatenate([orc.jit_row(11, 19, r, 5000, orc.W_NORMAL, 0.5, 0.1)[1] for r in range(40)])
    n = len(vals)
    assert abs(vals.mean() - 0.5) < 5 * 0.1 / math.sqrt(n)
    assert abs(vals.std() - 0.1) < 5 * 0.1 / math.sqrt(2 * n)
    ks = stats.kstest((vals - 0.5) / 0.1, "norm")
    assert ks.pvalue > 1e-4


def test_rows_independent_of_other_events():
    K = orc.jit_K(0.05)
    n = 300
    e1 = wl.bernoulli_spikes(n, 0.1, 1)
    e2 = wl.bernoulli_spikes(n, 0.1, 2) & (1 - e1)
    y1 = orc.jitconn_event_mv(31, K, n, n, e1)
    y2 = orc.jitconn_event_mv(31, K, n, n, e2)
    y12 = orc.jitconn_event_mv(31, K, n, n, e1 | e2)
    assert np.array_equal(y1 + y2, y12)
    # and a row is regenerated identically on every call
    a = orc.jit_row(31, K, 17, n)[0]
    b = orc.jit_row(31, K, 17, n)[0]
    assert np.array_equal(a, b)


def test_listing_semantics_single_row_bruteforce():
    """A single spiking row adds the weight at q_0 = U_0 - 1, q_{k+1} = q_k + U_{k+1}."""
    K, n_post, seed, row = 7, 60, 99, 3
    draws = [orc.jit_draw(seed, row, 0, k) for k in range(n_post + 1)]
    gaps = [1 + (d * K >> 32) for d in draws]
    expect = np.zeros(n_post)
    q = gaps[0] - 1
    k = 0
    while q < n_post:
        expect[q] += 0.6
        k += 1
        q += gaps[k]
    ev = np.zeros(row + 1, np.uint8)
    ev[row] = 1
    got = orc.jitconn_event_mv(seed, K, row + 1, n_post, ev, orc.W_HOMO, 0.6)
    assert np.array_equal(got, expect)
