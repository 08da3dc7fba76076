"""Pins of the oracle's COBA E/I network step (Appendices E, F, N).

What pins what:
* synaptic decay            -> closed form g_n = g_0 exp(-n dt / tau) (Appendix E).
* exponential Euler step    -> scipy's ODE solver on tau dV/dt = -(V - V_rest) + R I
                               with I held fixed over the step (Appendix F).
* COBA current              -> signs: an E event depolarises, an I event hyperpolarises.
* threshold/reset/refractory-> closed-form interspike interval of an isolated
                               neuron under constant input: first spike at step 139,
                               then every 189 steps; no spike within 51 steps.
* AlignPost merging         -> per-synapse conductances simulated one by one and
                               summed equal the merged per-neuron conductance
                               (Section 4.3: the merging is exact).
* event delivery            -> events per step = sum of out-degrees of spiking rows.
* synaptic delay            -> a single presynaptic spike at the closed-form step
                               t_s = 138 reaches the target's conductance exactly
                               at step t_s + 1 + d, with one weight, for each
                               projection and delay (Appendix D: spikes are
                               retrieved after the projection's delay).
* AlignPre                  -> equals AlignPost (Appendix D: the projections are
                               exact, not approximations; for exponential synapses
                               g = W^T s by linearity): identical rasters, equal
                               conductances and potentials up to FP64 rounding.
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle as orc
from paper_2311_05106_gb300 import workloads as wl


def _empty_csr(n):
    return ("csr", np.zeros(n + 1, np.int64), np.zeros(0, np.int32), None)


def test_synaptic_decay_closed_form():
    net = orc.CobaNet(4, 2, _empty_csr(4), np.full(4, -70.0))
    net.ge[:] = [1.0, 2.0, 0.0, 3.0]
    net.gi[:] = [5.0, 0.0, 1.0, 2.0]
    g0e, g0i = net.ge.copy(), net.gi.copy()
    for _ in range(137):
        net.step()
    np.testing.assert_allclose(net.ge, g0e * math.exp(-137 * 0.1 / 5.0), rtol=1e-12)
    np.testing.assert_allclose(net.gi, g0i * math.exp(-137 * 0.1 / 10.0), rtol=1e-12)


def test_exponential_euler_matches_ode_solver():
    rng = np.random.default_rng(0)
    for _ in range(5):
        V0 = rng.uniform(-65, -52)
        ge0, gi0 = rng.uniform(0, 3), rng.uniform(0, 5)
        net = orc.CobaNet(1, 1, _empty_csr(1), np.array([V0]))
        net.ge[:] = ge0
        net.gi[:] = gi0
        net.step()
        ge1, gi1 = ge0 * math.exp(-0.1 / 5.0), gi0 * math.exp(-0.1 / 10.0)
        I = ge1 * (0.0 - V0) + gi1 * (-80.0 - V0) + 20.0
        sol = solve_ivp(lambda t, v: (-(v - (-60.0)) + 1.0 * I) / 20.0, (0, 0.1), [V0], rtol=1e-12, atol=1e-12)
        expect = sol.y[0, -1]
        if expect > -50.0:
            assert net.V[0] == -60.0
        else:
            assert abs(net.V[0] - expect) < 1e-9


def test_coba_current_signs():
    def one_step(ce, ci):
        net = orc.CobaNet(1, 1, _empty_csr(1), np.array([-58.0]), I_ext=0.0)
        net.ye[:] = ce
        net.yi[:] = ci
        net.step()
        return net.V[0]
    base = one_step(0, 0)
    assert one_step(3, 0) > base
    assert one_step(0, 3) < base


def test_isolated_neuron_interspike_interval():
    n = 3
    net = orc.CobaNet(n, 2, _empty_csr(n), np.full(n, -60.0))
    out = net.run(2000, raster=True)
    for i in range(n):
        t = np.nonzero(out["raster"][:, i])[0] + 1            # 1-based step numbers
        # V_m = -40 - 20 a^m crosses -50 when a^m < 1/2: m* = ceil(200 ln 2) = 139
        assert t[0] == 139
        assert np.all(np.diff(t) == 139 + 50)                  # 50 clamped steps + 139 integrating
        assert len(t) == 1 + (2000 - 139) // 189


def test_refractory_clamp_holds_reset_value():
    net = orc.CobaNet(1, 1, _empty_csr(1), np.array([-60.0]))
    for _ in range(139):
        spk = net.step()
    assert spk[0] == 1 and net.V[0] == -60.0 and net.ref[0] == 50
    for k in range(50):
        net.ye[:] = 5.0                                         # strong input does not move V
        spk = net.step()
        assert spk[0] == 0 and net.V[0] == -60.0
    # the conductance built up during the clamp now drives the neuron over threshold at once
    assert net.step()[0] == 1


def test_alignpost_merging_exact():
    n, n_e = 60, 48
    ip, ix = wl.random_csr(n, n, 0.1, seed=3)
    V0 = wl.coba_v0(n, seed=4).astype(np.float64)
    net = orc.CobaNet(n, n_e, ("csr", ip, ix, None), V0)
    T = 300
    rows = np.repeat(np.arange(n), np.diff(ip))
    g_syn = np.zeros(len(ix))                 # one conductance per synapse (Appendix F)
    a_e, a_i = math.exp(-0.1 / 5.0), math.exp(-0.1 / 10.0)
    is_e = rows < n_e
    prev = np.zeros(n, np.uint8)
    total = 0
    for _ in range(T):
        g_syn = np.where(is_e, g_syn * a_e, g_syn * a_i)
        g_syn += np.where(prev[rows] == 1, np.where(is_e, 0.6, 6.7), 0.0)
        spk = net.step()
        ge_sum = np.bincount(ix[is_e], weights=g_syn[is_e], minlength=n)
        gi_sum = np.bincount(ix[~is_e], weights=g_syn[~is_e], minlength=n)
        np.testing.assert_allclose(net.ge, ge_sum, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(net.gi, gi_sum, rtol=1e-12, atol=1e-12)
        prev = spk
        total += spk.sum()
    assert total > 0


def test_event_totals_and_refractoriness_in_network():
    n, n_e = 4000, 3200
    K = orc.jit_K(0.02)
    se, si = orc.projection_seed(2024, 0), orc.projection_seed(2024, 1)
    net = orc.CobaNet(n, n_e, ("jit", se, si, K), wl.coba_v0(n, seed=7))
    out = net.run(600, raster=True, events=True)
    ras = out["raster"]
    lens_e = orc.jit_row_lengths(se, K, n_e, n)
    lens_i = orc.jit_row_lengths(si, K, n - n_e, n)
    lens = np.concatenate([lens_e, lens_i])
    assert np.array_equal(out["events"], ras.astype(np.int64) @ lens)
    assert np.array_equal(out["spikes_e"], ras[:, :n_e].sum(1))
    # no neuron fires twice within ref_steps + 1 = 51 steps
    for i in range(0, n, 97):
        t = np.nonzero(ras[:, i])[0]
        assert np.all(np.diff(t) >= 51)
    assert ras.sum() > 0


def test_stored_csr_equals_jit_network():
    """Materialising the JIT rows as a CSR gives the same trajectory bit for bit."""
    n, n_e = 1000, 800
    K = orc.jit_K(80.0 / n)
    se, si = orc.projection_seed(5, 0), orc.projection_seed(5, 1)
    ipe, ixe, _ = orc.jit_materialize(se, K, n_e, n)
    ipi, ixi, _ = orc.jit_materialize(si, K, n - n_e, n)
    ip = np.concatenate([ipe, ipi[1:] + ipe[-1]])
    ix = np.concatenate([ixe, ixi])
    V0 = wl.coba_v0(n, seed=7)
    a = orc.CobaNet(n, n_e, ("jit", se, si, K), V0).run(300, raster=True)
    b = orc.CobaNet(n, n_e, ("csr", ip, ix, None), V0).run(300, raster=True)
    assert np.array_equal(a["raster"], b["raster"])


@pytest.mark.parametrize("d_e,d_i", [(0, 0), (3, 0), (0, 5), (7, 2)])
def test_delay_shifts_arrival_closed_form(d_e, d_i):
    """Neuron 0 (E) and neuron 2 (I) start at V_reset and spike first at the
    closed-form step 138 (0-based: after 139 integrating steps); both project
    onto neuron 1, which sits far below threshold.  Its g_e must stay 0 until
    step 138 + 1 + d_e and then equal w_e = 0.6 (decaying afterwards); likewise
    g_i with w_i = 6.7 and d_i."""
    indptr = np.array([0, 1, 1, 2], np.int64)
    indices = np.array([1, 1], np.int32)
    V0 = np.array([-60.0, -1000.0, -60.0])
    net = orc.CobaNet(3, 2, ("csr", indptr, indices, None), V0, delay_e=d_e, delay_i=d_i)
    ge1, gi1 = [], []
    t_spike = None
    for t in range(138 + 12):
        spk = net.step()
        if spk[0]:
            assert spk[2] and t_spike is None
            t_spike = t
        ge1.append(net.ge[1])
        gi1.append(net.gi[1])
    assert t_spike == 138
    ge1, gi1 = np.array(ge1), np.array(gi1)
    te, ti = t_spike + 1 + d_e, t_spike + 1 + d_i
    assert np.all(ge1[:te] == 0.0) and ge1[te] == 0.6
    assert np.all(gi1[:ti] == 0.0) and gi1[ti] == 6.7
    # afterwards plain decay (no second spike within the window)
    assert abs(ge1[te + 1] - 0.6 * math.exp(-0.1 / 5.0)) < 1e-15


@pytest.mark.parametrize("form", ["csr_homo", "csr_weights", "jit"])
def test_align_pre_equals_align_post(form):
    n, n_e, seed, p = 2000, 1600, 77, 0.04
    K = orc.jit_K(p)
    se, si = orc.projection_seed(seed, 0), orc.projection_seed(seed, 1)
    if form == "jit":
        conn = ("jit", se, si, K)
    else:
        ipe, ixe, _ = orc.jit_materialize(se, K, n_e, n)
        ipi, ixi, _ = orc.jit_materialize(si, K, n - n_e, n)
        ip = np.concatenate([ipe, ipi[1:] + ipe[-1]])
        ix = np.concatenate([ixe, ixi])
        data = None
        if form == "csr_weights":
            data = np.where(np.arange(len(ix)) < len(ixe), 0.6, 6.7)
        conn = ("csr", ip, ix, data)
    V0 = wl.coba_v0(n, seed=9).astype(np.float64)
    post = orc.CobaNet(n, n_e, conn, V0, align="post")
    pre = orc.CobaNet(n, n_e, conn, V0, align="pre")
    total = 0
    for _ in range(300):
        a, b = post.step(), pre.step()
        assert np.array_equal(a, b)
        total += int(a.sum())
    assert total > 100
    np.testing.assert_allclose(pre.ge, post.ge, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(pre.gi, post.gi, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(pre.V, post.V, rtol=0, atol=1e-9)
