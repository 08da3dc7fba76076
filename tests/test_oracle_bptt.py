"""Pins of the BPTT oracle (oracle/bptt.py, Appendix I).

Forward:
* synaptic current of one input spike = W_in row x a_s^(t-1) (closed form);
* membrane update = scipy's ODE solver on tau dV/dt = -(V - V_rest) + R I with
  I held over the step (subthreshold);
* readout = closed-form leaky sum of a known spike train; loss = scipy logsumexp
  form of the cross-entropy.
Adjoint (hand-written):
* equals torch autograd (FP64 CPU) of the same model with a custom surrogate
  spike function and a detached reset;
* equals central finite differences of a fully smooth variant (logistic spikes,
  differentiable reset), where the surrogate is the exact derivative;
* with the ReLU surrogate and the voltage regulariser (Appendix I): equals
  torch autograd of the same model with that surrogate and the penalty written
  in torch; the regulariser's gradient equals finite differences of the smooth
  variant; the surrogate and the penalty match their closed forms.
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.special import logsumexp

from oracle import bptt
from paper_2311_05106_gb300 import workloads as wl


def small_problem(seed=0, B=2, T=30, n_in=12, n_rec=24, n_out=5, p_rec=0.2, rate_scale=8.0, rec_std=0.5):
    u = wl.poisson_inputs(B, T, n_in, seed, rate_lo=5.0 * rate_scale, rate_hi=50.0 * rate_scale)
    w = wl.snn_weights(n_in, n_rec, n_out, p_rec, seed + 1, rec_std=rec_std)
    w["W_in"] = w["W_in"] * 4.0
    labels = wl.labels(B, n_out, seed + 2)
    return u, labels, w


def test_synaptic_current_closed_form():
    n_in, n_rec, T = 3, 4, 9
    u = np.zeros((1, T, n_in), np.uint8)
    u[0, 0, 1] = 1
    W_in = np.arange(12, dtype=np.float64).reshape(3, 4) * 1e-3   # tiny: never reaches threshold
    ip = np.zeros(n_rec + 1, np.int64)
    fw = bptt.forward(u, W_in, ip, np.zeros(0, np.int32), np.zeros(0), np.zeros((n_rec, 2)), np.zeros(2))
    a_s = math.exp(-1.0 / 100.0)
    for t in range(T):
        np.testing.assert_allclose(fw["I"][0, t], W_in[1] * a_s ** t, rtol=1e-13)
    assert fw["z"].sum() == 0


def test_membrane_update_matches_ode_solver():
    rng = np.random.default_rng(1)
    n_in, n_rec, T = 4, 3, 6
    u = (rng.random((1, T, n_in)) < 0.5).astype(np.uint8)
    W_in = rng.uniform(0, 0.05, (n_in, n_rec))
    ip = np.zeros(n_rec + 1, np.int64)
    fw = bptt.forward(u, W_in, ip, np.zeros(0, np.int32), np.zeros(0), np.zeros((n_rec, 2)), np.zeros(2))
    V = np.zeros(n_rec)
    for t in range(T):
        I = fw["I"][0, t]
        sol = solve_ivp(lambda s, v: (-(v - 0.0) + 1.0 * I) / 20.0, (0, 1.0), V, rtol=1e-12, atol=1e-13)
        V = sol.y[:, -1]
        np.testing.assert_allclose(fw["Vp"][0, t], V, rtol=1e-9, atol=1e-12)
    assert fw["z"].sum() == 0


def test_spike_reset_and_readout_closed_form():
    # one strong input: the neuron crosses V_th = 1 at a known step, resets to 0
    n_in, n_rec, n_out, T = 1, 1, 2, 40
    u = np.zeros((1, T, n_in), np.uint8)
    u[0, :, 0] = 1
    W_in = np.array([[3.0]])
    ip = np.zeros(2, np.int64)
    W_out = np.array([[0.5, -1.0]])
    b = np.array([0.1, 0.2])
    fw = bptt.forward(u, W_in, ip, np.zeros(0, np.int32), np.zeros(0), W_out, b)
    z = fw["z"][0, :, 0]
    Vp = fw["Vp"][0, :, 0]
    assert np.all((Vp > 1.0) == (z == 1.0))
    assert z.sum() > 0
    # readout: y_t = a_o y_{t-1} + dt (W_out^T z_t + b)
    a_o = math.exp(-1.0 / 20.0)
    y = np.zeros(2)
    acc = np.zeros(2)
    for t in range(T):
        y = a_o * y + (W_out[0] * z[t] + b)
        acc += y
    np.testing.assert_allclose(fw["m"][0], acc / T, rtol=1e-13)
    # the potential after a spike starts again from the reset value 0
    t0 = int(np.nonzero(z)[0][0])
    I1 = fw["I"][0, t0 + 1, 0]
    a_m = math.exp(-1.0 / 20.0)
    assert abs(Vp[t0 + 1] - (1 - a_m) * I1) < 1e-13


def test_cross_entropy():
    m = np.random.default_rng(2).normal(size=(4, 7))
    labels = np.array([0, 3, 6, 2])
    L, g = bptt.loss_and_grad_m(m, labels)
    ref = np.mean(logsumexp(m, axis=1) - m[np.arange(4), labels])
    assert abs(L - ref) < 1e-13
    np.testing.assert_allclose(g.sum(axis=1), 0.0, atol=1e-15)


def test_relu_surrogate_closed_form():
    p = dict(bptt.SNN_DEFAULTS, surrogate="relu")
    x = np.array([0.0, 0.5, -0.5, 0.25, 1.0, -1.0, 1.5, -7.0])
    np.testing.assert_allclose(bptt.surrogate_grad(x, p), [0.3, 0.15, 0.15, 0.225, 0.0, 0.0, 0.0, 0.0], atol=1e-15)
    # a triangle of height alpha * width and half-width width: area alpha * width^2
    q = dict(p, sg_alpha=0.7, sg_width=2.0)
    xs = np.linspace(-3, 3, 600001)
    area = np.sum(bptt.surrogate_grad(xs, q)) * (xs[1] - xs[0])
    assert abs(area - 0.7 * 4.0) < 1e-6
    # the default remains the logistic surrogate: k/4 at x = 0
    assert abs(bptt.surrogate_grad(np.array([0.0]), bptt.SNN_DEFAULTS)[0] - 1.0) < 1e-15


def test_voltage_penalty_closed_form():
    p = bptt.SNN_DEFAULTS
    V = np.array([1.4, 0.4, 0.0, -2.0, -3.0, -1.0, 2.4])
    np.testing.assert_allclose(bptt.voltage_penalty(V, p), [1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 4.0], atol=1e-15)
    h = 1e-6
    Vs = np.array([1.3, -2.5, 0.1, 3.0])
    fd = (bptt.voltage_penalty(Vs + h, p) - bptt.voltage_penalty(Vs - h, p)) / (2 * h)
    np.testing.assert_allclose(bptt.voltage_penalty_grad(Vs, p), fd, rtol=1e-7, atol=1e-9)


def torch_model_loss(torch, u, labels, w, surrogate, lambda_v):
    """Loss and parameter leaves of the Appendix I model written in torch
    (FP64), with its own spike function and penalty."""
    p = bptt.SNN_DEFAULTS
    a_s, a_m, a_o = (math.exp(-1 / p["tau_s"]), math.exp(-1 / p["tau_m"]), math.exp(-1 / p["tau_o"]))
    k = p["slope"]

    class Spike(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x):
            ctx.save_for_backward(x)
            return (x > 0).to(x.dtype)

        @staticmethod
        def backward(ctx, go):
            (x,) = ctx.saved_tensors
            if surrogate == "relu":
                return go * torch.clamp(0.3 * (1.0 - x.abs()), min=0.0)
            s = torch.sigmoid(k * x)
            return go * k * s * (1 - s)

    d = torch.float64
    W_in = torch.tensor(w["W_in"], dtype=d, requires_grad=True)
    w_rec = torch.tensor(w["w_rec"], dtype=d, requires_grad=True)
    W_out = torch.tensor(w["W_out"], dtype=d, requires_grad=True)
    b_out = torch.tensor(w["b_out"], dtype=d, requires_grad=True)
    n_rec = W_in.shape[1]
    rows = torch.tensor(np.repeat(np.arange(n_rec), np.diff(w["indptr"])))
    cols = torch.tensor(w["indices"].astype(np.int64))
    W = torch.zeros((n_rec, n_rec), dtype=d).index_put((rows, cols), w_rec, accumulate=True)
    U = torch.tensor(u, dtype=d)
    B, T, _ = u.shape
    I = torch.zeros((B, n_rec), dtype=d)
    V = torch.zeros_like(I)
    z = torch.zeros_like(I)
    y = torch.zeros((B, W_out.shape[1]), dtype=d)
    msum = torch.zeros_like(y)
    pen = torch.zeros((), dtype=d)
    for t in range(T):
        I = a_s * I + z @ W + U[:, t] @ W_in
        Vp = a_m * V + (1 - a_m) * I
        pen = pen + (torch.relu(Vp - 0.4) ** 2 + torch.relu(-Vp - 2.0) ** 2).sum()
        z = Spike.apply(Vp - 1.0)
        V = Vp + z.detach() * (0.0 - Vp)
        y = a_o * y + (z @ W_out + b_out)
        msum = msum + y
    mt = msum / T
    loss = torch.nn.functional.cross_entropy(mt, torch.tensor(labels)) + lambda_v / B * pen
    return loss, (W_in, w_rec, W_out, b_out)


@pytest.mark.parametrize("surrogate,lambda_v", [("sigmoid", 0.0), ("relu", 0.0), ("relu", 0.05), ("sigmoid", 0.02)])
def test_adjoint_equals_torch_autograd(surrogate, lambda_v):
    torch = pytest.importorskip("torch")
    u, labels, w = small_problem()
    params = dict(surrogate=surrogate, lambda_v=lambda_v)
    L, m, g, fw = bptt.loss_and_grads(u, labels, w["W_in"].astype(np.float64), w["indptr"], w["indices"],
                                     w["w_rec"].astype(np.float64), w["W_out"].astype(np.float64),
                                     w["b_out"].astype(np.float64), params)
    assert fw["z"].mean() > 0.01        # the network spikes, so the surrogate paths are exercised
    if lambda_v:
        assert fw["L_v"] > 1e-3 * L     # and the penalty is active
    loss, leaves = torch_model_loss(torch, u, labels, w, surrogate, lambda_v)
    loss.backward()
    assert abs(loss.item() - L) < 1e-12
    for leaf, name in zip(leaves, ("W_in", "w_rec", "W_out", "b_out")):
        np.testing.assert_allclose(leaf.grad.numpy(), g[name], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("lambda_v", [0.0, 0.05])
def test_adjoint_finite_differences_smooth_variant(lambda_v):
    u, labels, w = small_problem(seed=4, T=20)
    args = [w["W_in"].astype(np.float64), w["indptr"], w["indices"], w["w_rec"].astype(np.float64),
            w["W_out"].astype(np.float64), w["b_out"].astype(np.float64), dict(lambda_v=lambda_v)]
    L, m, g, fw = bptt.loss_and_grads(u, labels, *args, smooth=True)
    if lambda_v:
        assert fw["L_v"] > 1e-3 * L
    rng = np.random.default_rng(5)
    h = 1e-6

    def loss_with(idx, pos, delta):
        a = [x.copy() if isinstance(x, np.ndarray) else x for x in args]
        a[idx].reshape(-1)[pos] += delta
        return bptt.loss_and_grads(u, labels, *a, smooth=True)[0]

    for idx, name in [(0, "W_in"), (3, "w_rec"), (4, "W_out"), (5, "b_out")]:
        flat = g[name].reshape(-1)
        for pos in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            fd = (loss_with(idx, pos, h) - loss_with(idx, pos, -h)) / (2 * h)
            assert abs(fd - flat[pos]) <= 1e-6 + 1e-4 * abs(flat[pos]), (name, pos, fd, flat[pos])
