"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's.

This module holds no arithmetic of the method itself: it only draws inputs
(initial potentials, spike vectors, random sparse matrices, weights, network
sizes, Poisson input trains, labels) from numpy's seeded generators, with the
shapes and distributions of the paper's workloads:

* COBA E/I network (Appendix N, Listing S6): 80 % excitatory, V0 ~ N(-55, 5) mV.
* Operator sweep (Section 5.1 / Appendix B): Bernoulli spike vectors of density
  rho, connection probability p, weights N(0.5, 0.1) or homogeneous.
* Batched networks: sizes uniform in [1000, 50000].
* Differentiable network (Appendix I): Poisson input trains with rates uniform
  in [5, 50] Hz, Gaussian weights sqrt(s / n_in) N(0, 1), random labels.

Every generator takes an explicit integer seed; the same call returns the same
arrays on every machine.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "coba_v0", "bernoulli_spikes", "random_csr", "normal_weights", "lif_state",
    "batched_sizes", "poisson_inputs", "labels", "snn_weights",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.uint64(seed & (2**64 - 1)))


def coba_v0(n: int, seed: int = 7, mean: float = -55.0, std: float = 5.0) -> np.ndarray:
    """Initial membrane potentials, drawn in FP64 and rounded once to FP32."""
    return _rng(seed).normal(mean, std, size=n).astype(np.float32)


def bernoulli_spikes(n: int, rho: float, seed: int) -> np.ndarray:
    """Spike flags (uint8) with P(spike) = rho, independently per neuron."""
    return (_rng(seed).random(n) < rho).astype(np.uint8)


def random_csr(n_pre: int, n_post: int, p: float, seed: int, sort: bool = True):
    """Random pre-major CSR: each (pre, post) pair present with probability p.

    Row lengths are Binomial(n_post, p); columns are drawn without replacement.
    Returns (indptr int64 [n_pre+1], indices int32 [nnz]).  Sized for tests
    (a few million entries at most).
    """
    rng = _rng(seed)
    lens = rng.binomial(n_post, p, size=n_pre).astype(np.int64)
    indptr = np.zeros(n_pre + 1, np.int64)
    np.cumsum(lens, out=indptr[1:])
    indices = np.empty(int(indptr[-1]), np.int32)
    for i in range(n_pre):
        k = int(lens[i])
        if k == 0:
            continue
        cols = rng.choice(n_post, size=k, replace=False).astype(np.int32)
        if sort:
            cols.sort()
        indices[indptr[i]:indptr[i + 1]] = cols
    return indptr, indices


def normal_weights(nnz: int, mean: float, std: float, seed: int) -> np.ndarray:
    """Heterogeneous synaptic weights N(mean, std), FP32."""
    return _rng(seed).normal(mean, std, size=nnz).astype(np.float32)


def lif_state(n: int, seed: int, ref_steps: int = 50, p_ref: float = 0.2):
    """A mid-simulation-like COBA state for single-step tests.

    V uniform in [-62, -48] mV (straddling threshold and reset), conductances
    exponential with means 2 (E) and 10 (I), a fraction p_ref of neurons in
    their refractory period, and small event counts.
    """
    rng = _rng(seed)
    V = rng.uniform(-62.0, -48.0, n).astype(np.float32)
    ge = rng.exponential(2.0, n).astype(np.float32)
    gi = rng.exponential(10.0, n).astype(np.float32)
    ref = np.where(rng.random(n) < p_ref, rng.integers(1, ref_steps + 1, n), 0).astype(np.int32)
    ce = rng.poisson(1.5, n).astype(np.int32)
    ci = rng.poisson(0.5, n).astype(np.int32)
    return dict(V=V, ge=ge, gi=gi, ref=ref, ce=ce, ci=ci)


def batched_sizes(n_nets: int = 256, lo: int = 1000, hi: int = 50000, seed: int = 11) -> np.ndarray:
    """Network sizes uniform in [lo, hi] (rounded down to a multiple of 5 so the
    80/20 split is exact)."""
    n = _rng(seed).integers(lo, hi + 1, size=n_nets)
    return (n - n % 5).astype(np.int64)


def poisson_inputs(batch: int, T: int, n_in: int, seed: int, rate_lo: float = 5.0, rate_hi: float = 50.0,
                   dt_ms: float = 1.0) -> np.ndarray:
    """Input spike trains u[b, t, k] (uint8): channel k fires with probability
    rate_k * dt per step, rate_k uniform in [rate_lo, rate_hi] Hz."""
    rng = _rng(seed)
    rates = rng.uniform(rate_lo, rate_hi, size=n_in)
    prob = rates * dt_ms * 1e-3
    return (rng.random((batch, T, n_in)) < prob[None, None, :]).astype(np.uint8)


def labels(batch: int, n_classes: int, seed: int) -> np.ndarray:
    return _rng(seed).integers(0, n_classes, size=batch).astype(np.int64)


def snn_weights(n_in: int, n_rec: int, n_out: int, p_rec: float, seed: int, rec_std: float | None = None):
    """Weights of the differentiable recurrent network (Appendix I init).

    W_in [n_in, n_rec] ~ N(0, 1/sqrt(n_in)) dense; W_rec CSR [n_rec pre rows]
    with density p_rec and values N(0, rec_std) (default 1/sqrt(p_rec n_rec));
    W_out [n_rec, n_out] ~ N(0, 1/sqrt(n_rec)); b_out zeros.
    """
    rng = _rng(seed)
    W_in = rng.normal(0.0, 1.0 / np.sqrt(n_in), size=(n_in, n_rec)).astype(np.float32)
    indptr, indices = random_csr(n_rec, n_rec, p_rec, seed + 1)
    if rec_std is None:
        rec_std = 1.0 / np.sqrt(p_rec * n_rec)
    w_rec = rng.normal(0.0, rec_std, size=len(indices)).astype(np.float32)
    W_out = rng.normal(0.0, 1.0 / np.sqrt(n_rec), size=(n_rec, n_out)).astype(np.float32)
    b_out = np.zeros(n_out, np.float32)
    return dict(W_in=W_in, indptr=indptr, indices=indices, w_rec=w_rec, W_out=W_out, b_out=b_out)
