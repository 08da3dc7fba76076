"""FP64 oracle of the differentiable recurrent spiking network and its BPTT
adjoint (Appendix I: LIF recurrent layer with exponential synaptic current,
leaky readout, cross-entropy, surrogate-gradient back-propagation through
time).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy, FP64, one
time step after the other in the order the model is defined; the adjoint is
written out by hand, step by step in reverse.  Pinned in
tests/test_oracle_bptt.py against torch autograd of the same forward and
against finite differences of a smooth variant.

Model (readings of Appendix I fixed for this build):
  state at t = 0: I = V = y = 0, no spikes.
  for t = 1..T:
    I_t  = a_s I_{t-1} + W_rec^T z_{t-1} + W_in^T u_t      (synaptic current,
           Appendix I discrete form; W_rec presynaptic-row-major, delay 0)
    Vp_t = a_m V_{t-1} + (1 - a_m)(V_rest + R I_t)          (exponential Euler)
    z_t  = H(Vp_t - V_th)                                    (spike)
    V_t  = Vp_t + z_t (V_reset - Vp_t), with z_t treated as a constant in the
           gradient (reset path detached)
    y_t  = a_o y_{t-1} + dt (W_out^T z_t + b)                (leaky readout)
  m = mean_t y_t;  L = mean_b [logsumexp(m_b) - m_b[label_b]] + L_v
  surrogate: dH/dx ~ k s(k x)(1 - s(k x)), s the logistic, k = 4 (x = Vp - V_th),
    or the ReLU surrogate of Appendix I, dH/dx ~ max(0, alpha (width - |x|)),
    alpha = 0.3, width = 1 (surrogate="relu").
  voltage regulariser (Appendix I, training methods):
    L_v = (lambda_v / B) sum_b sum_t sum_i [ReLU(Vp - v_hi)^2 + ReLU(v_lo - Vp)^2],
    v_hi = 0.4, v_lo = -2; applied to the potential before reset (the one the
    surrogate sees), averaged over the batch like the cross-entropy;
    lambda_v = 0 (off) unless given.
"""
from __future__ import annotations

import math

import numpy as np

SNN_DEFAULTS = dict(dt=1.0, tau_m=20.0, tau_s=100.0, tau_o=20.0, V_rest=0.0, V_reset=0.0, V_th=1.0, R=1.0, slope=4.0,
                    surrogate="sigmoid", sg_alpha=0.3, sg_width=1.0, lambda_v=0.0, v_hi=0.4, v_lo=-2.0)


def _consts(p):
    return (math.exp(-p["dt"] / p["tau_s"]), math.exp(-p["dt"] / p["tau_m"]), math.exp(-p["dt"] / p["tau_o"]))


def _sig(x):
    return 1.0 / (1.0 + np.exp(-x))


def surrogate_grad(x, p):
    """Surrogate derivative of the Heaviside spike at x = Vp - V_th."""
    if p["surrogate"] == "relu":
        return np.maximum(0.0, p["sg_alpha"] * (p["sg_width"] - np.abs(x)))
    s = _sig(p["slope"] * x)
    return p["slope"] * s * (1.0 - s)


def voltage_penalty(Vp, p):
    """Per-element term of the voltage regulariser (before lambda_v / B)."""
    return np.maximum(Vp - p["v_hi"], 0.0) ** 2 + np.maximum(p["v_lo"] - Vp, 0.0) ** 2


def voltage_penalty_grad(Vp, p):
    return 2.0 * np.maximum(Vp - p["v_hi"], 0.0) - 2.0 * np.maximum(p["v_lo"] - Vp, 0.0)


def _dense(indptr, indices, w, n_rec):
    W = np.zeros((n_rec, n_rec))
    for i in range(n_rec):
        for j in range(indptr[i], indptr[i + 1]):
            W[i, indices[j]] += w[j]
    return W


def forward(u, W_in, indptr, indices, w_rec, W_out, b_out, params=None, smooth=False):
    """u [B, T, n_in] (0/1); returns dict with m [B, n_out] and the per-step
    tensors the adjoint needs (I, Vp, z for t = 1..T, stacked on axis 1).
    smooth=True: spike = logistic(k x) and a differentiable reset (for the
    finite-difference pin only)."""
    p = dict(SNN_DEFAULTS)
    if params:
        p.update(params)
    a_s, a_m, a_o = _consts(p)
    B, T, n_in = u.shape
    n_rec = W_in.shape[1]
    W = _dense(indptr, indices, w_rec, n_rec)
    I = np.zeros((B, n_rec))
    V = np.zeros((B, n_rec))
    z = np.zeros((B, n_rec))
    y = np.zeros((B, W_out.shape[1]))
    Is, Vps, zs, ys = [], [], [], []
    msum = np.zeros_like(y)
    vreg = np.zeros(B)
    for t in range(T):
        I = a_s * I + z @ W + u[:, t, :].astype(np.float64) @ W_in
        Vp = a_m * V + (1.0 - a_m) * (p["V_rest"] + p["R"] * I)
        x = Vp - p["V_th"]
        vreg += voltage_penalty(Vp, p).sum(axis=1)
        z = _sig(p["slope"] * x) if smooth else (x > 0).astype(np.float64)
        V = Vp + z * (p["V_reset"] - Vp)
        y = a_o * y + p["dt"] * (z @ W_out + b_out)
        Is.append(I)
        Vps.append(Vp)
        zs.append(z)
        ys.append(y)
        msum += y
    m = msum / T
    return dict(m=m, I=np.stack(Is, 1), Vp=np.stack(Vps, 1), z=np.stack(zs, 1), y=np.stack(ys, 1), W=W, params=p,
                vreg=vreg, L_v=p["lambda_v"] / B * float(vreg.sum()))


def loss_and_grad_m(m, labels):
    """Mean cross-entropy of softmax(m) and its gradient dL/dm."""
    B = m.shape[0]
    mx = m.max(axis=1, keepdims=True)
    e = np.exp(m - mx)
    sm = e / e.sum(axis=1, keepdims=True)
    lse = np.log(e.sum(axis=1)) + mx[:, 0]
    L = float(np.mean(lse - m[np.arange(B), labels]))
    g = sm.copy()
    g[np.arange(B), labels] -= 1.0
    return L, g / B


def lif_step_adjoint(Vp, z, Vbar, zbar, Ibar_next, params=None, smooth=False, vreg_scale=0.0):
    """Adjoint of one LIF step (reset detached unless smooth): from dL/dV_t,
    dL/dz_t and dL/dI_{t+1}, returns (dL/dI_t, dL/dV_{t-1}).  vreg_scale is
    the regulariser's weight on this step's potentials (lambda_v / B)."""
    p = dict(SNN_DEFAULTS)
    if params:
        p.update(params)
    a_s, a_m, _ = _consts(p)
    if smooth:  # the exact derivative of the logistic spike
        s = _sig(p["slope"] * (Vp - p["V_th"]))
        dz = p["slope"] * s * (1.0 - s)
        Vpbar = Vbar * (1.0 - z) + (zbar + Vbar * (p["V_reset"] - Vp)) * dz
    else:
        Vpbar = Vbar * (1.0 - z) + zbar * surrogate_grad(Vp - p["V_th"], p)
    Vpbar = Vpbar + vreg_scale * voltage_penalty_grad(Vp, p)
    Ibar = (1.0 - a_m) * p["R"] * Vpbar + a_s * Ibar_next
    return Ibar, a_m * Vpbar


def backward(fw, u, indptr, indices, W_out, g_m, smooth=False):
    """Hand-written adjoint, t = T..1.  Returns gradients of L with respect to
    W_in [n_in, n_rec], the stored recurrent weights w_rec [nnz], W_out and
    b_out."""
    p = fw["params"]
    a_s, a_m, a_o = _consts(p)
    I, Vp, z = fw["I"], fw["Vp"], fw["z"]
    W = fw["W"]
    B, T, n_rec = Vp.shape
    n_in = u.shape[2]
    dW_in = np.zeros((n_in, n_rec))
    dW = np.zeros((n_rec, n_rec))
    dW_out = np.zeros_like(W_out, dtype=np.float64)
    db = np.zeros(W_out.shape[1])
    ybar = np.zeros((B, W_out.shape[1]))
    Ibar_next = np.zeros((B, n_rec))
    Vbar = np.zeros((B, n_rec))
    for t in range(T - 1, -1, -1):
        ybar = a_o * ybar + g_m / T
        zbar = p["dt"] * ybar @ W_out.T + Ibar_next @ W.T
        # smooth: the reset path V = Vp (1 - z) + V_reset z is included
        Ibar, Vbar = lif_step_adjoint(Vp[:, t], z[:, t], Vbar, zbar, Ibar_next, p, smooth, p["lambda_v"] / B)
        dW_out += p["dt"] * z[:, t].T @ ybar
        db += p["dt"] * ybar.sum(axis=0)
        dW_in += u[:, t, :].astype(np.float64).T @ Ibar
        if t > 0:
            dW += z[:, t - 1].T @ Ibar
        Ibar_next = Ibar
    rows = np.repeat(np.arange(n_rec), np.diff(indptr))
    dw_rec = dW[rows, indices]
    return dict(W_in=dW_in, w_rec=dw_rec, W_out=dW_out, b_out=db)


def loss_and_grads(u, labels, W_in, indptr, indices, w_rec, W_out, b_out, params=None, smooth=False):
    fw = forward(u, W_in, indptr, indices, w_rec, W_out, b_out, params, smooth)
    L, g = loss_and_grad_m(fw["m"], labels)
    L += fw["L_v"]
    grads = backward(fw, u, indptr, indices, W_out, g, smooth)
    return L, fw["m"], grads, fw
