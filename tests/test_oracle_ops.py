"""Pins of the oracle's event-driven operators (Appendix B, Appendix C, Section 4.1).

What pins what:
* event CSR product         -> dense brute force W^T s (float), exact int counts,
                               invariant sum(c) = sum of spiking rows' lengths.
* gather (transpose) form   -> dense W x; adjoint identity <W^T s, x> = <s, W x>.
* weight gradient           -> dense outer product s delta^T masked by the pattern,
                               and central finite differences of <y, delta>.
* JIT products              -> the same products on the oracle's materialised CSR.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2311_05106_gb300 import workloads as wl


def _dense(indptr, indices, data, n_post):
    n_pre = len(indptr) - 1
    W = np.zeros((n_pre, n_post))
    for i in range(n_pre):
        for j in range(indptr[i], indptr[i + 1]):
            W[i, indices[j]] += data[j]
    return W


@pytest.mark.parametrize("n_pre,n_post,p,rho", [(37, 53, 0.2, 0.3), (200, 150, 0.05, 0.1), (1, 1, 1.0, 1.0),
                                                (64, 512, 0.01, 0.5)])
def test_event_csrmv_dense_bruteforce(n_pre, n_post, p, rho):
    ip, ix = wl.random_csr(n_pre, n_post, p, seed=n_pre + n_post)
    w = wl.normal_weights(len(ix), 0.5, 0.1, seed=3).astype(np.float64)
    s = wl.bernoulli_spikes(n_pre, rho, seed=4)
    W = _dense(ip, ix, w, n_post)
    y = orc.event_csrmv(ip, ix, w, s, n_post)
    np.testing.assert_allclose(y, W.T @ s, rtol=1e-12, atol=1e-12)
    # homogeneous weight
    yh = orc.event_csrmv(ip, ix, None, s, n_post, w_homo=0.6)
    np.testing.assert_allclose(yh, 0.6 * ((W != 0).astype(float).T @ s), rtol=1e-12, atol=1e-12)


def test_event_counts_exact_and_invariant():
    n_pre, n_post = 300, 257
    ip, ix = wl.random_csr(n_pre, n_post, 0.07, seed=8)
    s = wl.bernoulli_spikes(n_pre, 0.2, seed=9)
    c = orc.event_csr_count(ip, ix, s, n_post)
    A = _dense(ip, ix, np.ones(len(ix)), n_post).astype(np.int64)
    assert np.array_equal(c, A.T @ s.astype(np.int64))
    lens = np.diff(ip)
    assert c.sum() == int((lens * s).sum())


def test_event_csrmv_empty_cases():
    ip, ix = wl.random_csr(10, 20, 0.3, seed=1)
    assert np.all(orc.event_csrmv(ip, ix, None, np.zeros(10, np.uint8), 20) == 0)
    ip0 = np.zeros(11, np.int64)
    assert np.all(orc.event_csrmv(ip0, np.zeros(0, np.int32), None, np.ones(10, np.uint8), 20) == 0)


def test_csrmv_t_dense_and_adjoint():
    n_pre, n_post = 120, 90
    ip, ix = wl.random_csr(n_pre, n_post, 0.1, seed=21)
    w = wl.normal_weights(len(ix), 0.0, 1.0, seed=22).astype(np.float64)
    x = np.random.default_rng(5).normal(size=n_post)
    W = _dense(ip, ix, w, n_post)
    yp = orc.csrmv_t(ip, ix, w, x)
    np.testing.assert_allclose(yp, W @ x, rtol=1e-12, atol=1e-12)
    s = wl.bernoulli_spikes(n_pre, 0.3, seed=23)
    lhs = orc.event_csrmv(ip, ix, w, s, n_post) @ x
    rhs = s.astype(float) @ yp
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def test_event_csrmv_dw_dense_and_finite_difference():
    n_pre, n_post = 40, 30
    ip, ix = wl.random_csr(n_pre, n_post, 0.2, seed=31)
    w = wl.normal_weights(len(ix), 0.0, 1.0, seed=32).astype(np.float64)
    s = wl.bernoulli_spikes(n_pre, 0.4, seed=33)
    delta = np.random.default_rng(6).normal(size=n_post)
    dw = orc.event_csrmv_dw(ip, ix, s, delta)
    rows = np.repeat(np.arange(n_pre), np.diff(ip))
    np.testing.assert_allclose(dw, s[rows] * delta[ix], rtol=0, atol=0)
    # L(w) = <W^T s, delta> is linear in w: central differences are exact up to rounding
    h = 1e-3
    for j in [0, len(ix) // 2, len(ix) - 1]:
        wp, wm = w.copy(), w.copy()
        wp[j] += h
        wm[j] -= h
        fd = (orc.event_csrmv(ip, ix, wp, s, n_post) @ delta - orc.event_csrmv(ip, ix, wm, s, n_post) @ delta) / (2 * h)
        assert abs(fd - dw[j]) < 1e-9


@pytest.mark.parametrize("wkind,w0,w1", [(orc.W_HOMO, 0.6, 0.0), (orc.W_UNIFORM, -1.0, 1.0), (orc.W_NORMAL, 0.5, 0.1)])
def test_jit_products_equal_materialised_csr(wkind, w0, w1):
    n_pre, n_post = 500, 700
    K = orc.jit_K(0.03)
    ip, ix, d = orc.jit_materialize(41, K, n_pre, n_post, wkind, w0, w1)
    assert np.array_equal(np.diff(ip), orc.jit_row_lengths(41, K, n_pre, n_post))
    s = wl.bernoulli_spikes(n_pre, 0.2, seed=42)
    y_jit = orc.jitconn_event_mv(41, K, n_pre, n_post, s, wkind, w0, w1)
    y_csr = orc.event_csrmv(ip, ix, d, s, n_post)
    assert np.array_equal(y_jit, y_csr)
    x_pre = np.random.default_rng(7).normal(size=n_pre)
    W = _dense(ip, ix, d, n_post)
    np.testing.assert_allclose(orc.jitconn_mv(41, K, n_pre, n_post, x_pre, wkind, w0, w1), W.T @ x_pre,
                               rtol=1e-12, atol=1e-12)
    x_post = np.random.default_rng(8).normal(size=n_post)
    np.testing.assert_allclose(orc.jitconn_mv_t(41, K, n_pre, n_post, x_post, wkind, w0, w1), W @ x_post,
                               rtol=1e-12, atol=1e-12)


def test_spike_outer_brute_force_and_special_cases():
    """The spike-driven weight gradient out[m][n] = sum_k [x_km != 0] delta_kn
    (Section 3.1's reverse-mode rule of y = W^T x with binary x): brute force on
    a tiny case; all-ones x gives the column sums of delta in every row; a
    single spike at (k, m) copies delta's row k into row m (so a transposed
    operand or a swapped index fails); byte values other than 1 count as one
    spike."""
    rng = np.random.default_rng(3)
    K, M, N = 7, 5, 4
    x = (rng.random((K, M)) < 0.4).astype(np.uint8) * rng.integers(1, 255, size=(K, M)).astype(np.uint8)
    d = rng.standard_normal((K, N))
    want = np.zeros((M, N))
    for k in range(K):
        for m in range(M):
            if x[k, m]:
                for n in range(N):
                    want[m, n] += d[k, n]
    np.testing.assert_allclose(orc.spike_outer(x, d), want, rtol=0, atol=1e-12)
    ones = np.ones((K, M), np.uint8)
    np.testing.assert_allclose(orc.spike_outer(ones, d), np.tile(d.sum(axis=0), (M, 1)), rtol=1e-14)
    one = np.zeros((K, M), np.uint8)
    one[4, 2] = 1
    g = orc.spike_outer(one, d)
    np.testing.assert_array_equal(g[2], d[4])
    assert np.count_nonzero(np.delete(g, 2, axis=0)) == 0
    assert orc.spike_outer(np.zeros((0, M), np.uint8), np.zeros((0, N))).shape == (M, N)
