"""Teacher-forced per-step parity of the fused network step (a1-a7) against the
FP64 oracle (Appendix N Listing S6; Appendices E and F).

Before every compared step the oracle is loaded with the GPU's FP32 state
(V, g_e, g_i, the refractory counters and the pending event accumulators the
step consumes); both sides then take one step and are compared:

* V, g_e, g_i within 1e-5 relative (per array, max |a - b| / max |b|);
* spike flags equal except where the oracle's threshold decision was within
  1e-4 mV of V_th (an FP32-vs-FP64 flip; V and the counter are not compared
  for such a neuron);
* the events the step delivered into the accumulator half the next step
  reads: integer counts bit for bit, FP32 / BF16 weighted sums within 1e-5
  relative of the oracle's product over the same spiking rows (BF16: the
  oracle fed the same BF16-rounded weights; within 1e-2 of the unrounded
  weights);
* the synaptic-event total equal to the summed out-degrees of the spikes.

Cases: the 4 000-neuron network (p = 0.02) for 300 steps with JIT rows,
stored CSR with integer counts, stored FP32 weights equal per projection (the
headline form), heterogeneous FP32 and BF16 weights; and the scaled network at
N = 4e6 (p = 80/N) for six steps (the onset burst and steps 30-32) in the
stored FP32, stored BF16, integer-count and JIT forms, with the kernels and
launch shapes the bench times.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc
from paper_2311_05106_gb300 import binding as B
from paper_2311_05106_gb300 import workloads as wl
from paper_2311_05106_gb300.network import CobaNetwork, materialize_network_csr

pytestmark = pytest.mark.gpu

V_TH = -50.0
NEAR_MV = 1e-4
W_E, W_I = 0.6, 6.7


def rel_err(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(float(np.max(np.abs(b))), 1e-30))


class Case:
    """One network on both sides: the GPU network, the oracle network and the
    oracle's delivery of a given spike vector, (E accumulator, I accumulator)."""

    def __init__(self, gpu, ref, deliver, lens, counts, tol_sum=1e-5, deliver_unrounded=None, ref_scale=(1.0, 1.0)):
        self.gpu, self.ref, self.deliver, self.lens = gpu, ref, deliver, lens
        self.counts, self.tol_sum, self.deliver_unrounded = counts, tol_sum, deliver_unrounded
        # weight per event of the oracle's own pending accumulators (1 where
        # the oracle counts events that the GPU sums as stored weights)
        self.ref_scale = ref_scale


def teacher_forced_step(c, max_flips):
    g, r, n = c.gpu, c.ref, c.gpu.n
    t = B.bp_network_step_count(g.handle)
    h = t % 2
    torch.cuda.synchronize()
    r.V[:] = g.V.cpu().numpy()
    r.ge[:] = g.ge.cpu().numpy()
    r.gi[:] = g.gi.cpu().numpy()
    r.ref[:] = g.ref.cpu().numpy().astype(np.int32)
    r.ye[:] = g.ye[h * n:(h + 1) * n].cpu().numpy()
    r.yi[:] = g.yi[h * n:(h + 1) * n].cpu().numpy()
    ev_before = int(g.totals[2].item())
    spk_o, vdec = r.step(return_vdec=True)
    g.step()
    torch.cuda.synchronize()
    spk = g.spk.cpu().numpy()
    near = ~np.isnan(vdec) & (np.abs(np.nan_to_num(vdec, nan=1e9) - V_TH) < NEAR_MV)
    flips = spk != spk_o
    assert np.all(near[flips]), (t, np.nonzero(flips & ~near)[0][:10])
    assert flips.sum() <= max_flips, (t, int(flips.sum()))
    ok = ~flips
    V = g.V.cpu().numpy()
    assert rel_err(V[ok], r.V[ok]) <= 1e-5, t
    assert rel_err(g.ge.cpu().numpy(), r.ge) <= 1e-5, t
    assert rel_err(g.gi.cpu().numpy(), r.gi) <= 1e-5, t
    assert np.array_equal(g.ref.cpu().numpy()[ok].astype(np.int32), r.ref[ok]), t
    out_e = g.ye[(1 - h) * n:(2 - h) * n].cpu().numpy()
    out_i = g.yi[(1 - h) * n:(2 - h) * n].cpu().numpy()
    exp_e, exp_i = c.deliver(spk)
    if c.counts:
        assert np.array_equal(out_e.astype(np.int64), exp_e.astype(np.int64)), t
        assert np.array_equal(out_i.astype(np.int64), exp_i.astype(np.int64)), t
    else:
        if exp_e.any():
            assert rel_err(out_e, exp_e) <= c.tol_sum, t
        if exp_i.any():
            assert rel_err(out_i, exp_i) <= c.tol_sum, t
        if c.deliver_unrounded is not None:
            ue, ui = c.deliver_unrounded(spk)
            if ue.any():
                assert rel_err(out_e, ue) <= 1e-2, t
            if ui.any():
                assert rel_err(out_i, ui) <= 1e-2, t
    if not flips.any():
        # the oracle's own delivery from its own spikes is the same product
        se, si = c.ref_scale
        assert np.allclose(se * r.ye, exp_e, rtol=1e-12, atol=0) and np.allclose(si * r.yi, exp_i, rtol=1e-12, atol=0)
    ev = int(g.totals[2].item()) - ev_before
    assert ev == int(c.lens[spk.astype(bool)].sum()), t
    return int(spk.sum()), int(flips.sum())


def jit_rows(seed, p, n, n_e):
    K = orc.jit_K(p)
    return orc.projection_seed(seed, 0), orc.projection_seed(seed, 1), K


def jit_deliver(se, si, K, n, n_e, w_e=1.0, w_i=1.0):
    def f(spk):
        e = orc.jitconn_event_mv(se, K, n_e, n, spk[:n_e])
        i = orc.jitconn_event_mv(si, K, n - n_e, n, spk[n_e:])
        return w_e * e, w_i * i
    return f


def csr_deliver(ip, ix, data, n, n_e):
    def f(spk):
        e = spk.copy()
        e[n_e:] = 0
        i = spk.copy()
        i[:n_e] = 0
        if data is None:
            return (orc.event_csr_count(ip, ix, e, n).astype(np.float64),
                    orc.event_csr_count(ip, ix, i, n).astype(np.float64))
        return orc.event_csrmv(ip, ix, data, e, n), orc.event_csrmv(ip, ix, data, i, n)
    return f


def small_case(kind, n=4000, n_e=3200, seed=2024, p=0.02):
    V0 = wl.coba_v0(n, seed=7)
    se, si, K = jit_rows(seed, p, n, n_e)
    ipe, ixe, _ = orc.jit_materialize(se, K, n_e, n)
    ipi, ixi, _ = orc.jit_materialize(si, K, n - n_e, n)
    ip = np.concatenate([ipe, ipi[1:] + ipe[-1]])
    ix = np.concatenate([ixe, ixi])
    lens = np.diff(ip)
    nnz_e = len(ixe)
    if kind == "jit":
        gpu = CobaNetwork(n, n_e, conn="jit", seed=seed, p=p, V0=V0, keep_spk=True)
        ref = orc.CobaNet(n, n_e, ("jit", se, si, K), V0.astype(np.float64))
        return Case(gpu, ref, jit_deliver(se, si, K, n, n_e), lens, counts=True)
    if kind == "csr_counts":
        gpu = CobaNetwork(n, n_e, conn="csr", seed=seed, p=p, V0=V0, keep_spk=True)
        ref = orc.CobaNet(n, n_e, ("csr", ip, ix, None), V0.astype(np.float64))
        return Case(gpu, ref, csr_deliver(ip, ix, None, n, n_e), lens, counts=True)
    gip, gix, _ = materialize_network_csr(seed, p, n, n_e)
    if kind == "csr_f32_equal":
        w = np.empty(len(ix), np.float32)
        w[:nnz_e], w[nnz_e:] = W_E, W_I
    else:
        w = wl.normal_weights(len(ix), 1.0, 0.2, seed=31)
        w[:nnz_e] *= np.float32(W_E)
        w[nnz_e:] *= np.float32(W_I)
    unrounded = None
    if kind == "csr_bf16_hetero":
        wt = torch.from_numpy(w).to(torch.bfloat16)
        w64 = wt.to(torch.float64).numpy()
        unrounded = csr_deliver(ip, ix, w.astype(np.float64), n, n_e)
    else:
        wt = torch.from_numpy(w)
        w64 = w.astype(np.float64)
    gpu = CobaNetwork(n, n_e, conn="csr", csr=(gip, gix, wt.cuda()), seed=seed, p=p, V0=V0, keep_spk=True)
    ref = orc.CobaNet(n, n_e, ("csr", ip, ix, w64), V0.astype(np.float64))
    return Case(gpu, ref, csr_deliver(ip, ix, w64, n, n_e), lens, counts=False, deliver_unrounded=unrounded)


@pytest.mark.parametrize("kind", ["csr_f32_equal", "csr_f32_hetero", "csr_bf16_hetero", "csr_counts", "jit"])
def test_teacher_forced_4k_network_300_steps(kind):
    c = small_case(kind)
    spikes = flips = 0
    for _ in range(300):
        s, f = teacher_forced_step(c, max_flips=2)
        spikes += s
        flips += f
    # the network is active (the onset burst and ~20 Hz afterwards) and flips are rare
    assert spikes > 1000
    assert flips <= 5
    c.gpu.close()


@pytest.mark.parametrize("kind", ["csr_f32", "csr_bf16", "csr_counts", "jit"])
def test_teacher_forced_scaled_network_N4e6(kind):
    """N = 4e6 as the bench builds it: the stored matrix is the JIT matrix
    materialised with weights w_e / w_i stored per synapse (FP32 or BF16), or
    integer counts.  The oracle regenerates the same rows itself (Appendix C);
    for stored weights it is given weight 1 per event and fed the GPU's
    weighted sums, and the expected delivery is the stored weight times its
    exact event count (all weights of a projection are equal)."""
    n, n_e, seed = 4_000_000, 3_200_000, 2024
    p = 80.0 / n
    V0 = wl.coba_v0(n, seed=7)
    se, si, K = jit_rows(seed, p, n, n_e)
    lens = np.concatenate([orc.jit_row_lengths(se, K, n_e, n), orc.jit_row_lengths(si, K, n - n_e, n)])
    if kind == "jit":
        gpu = CobaNetwork(n, n_e, conn="jit", seed=seed, p=p, V0=V0, keep_spk=True)
        ref = orc.CobaNet(n, n_e, ("jit", se, si, K), V0.astype(np.float64))
        c = Case(gpu, ref, jit_deliver(se, si, K, n, n_e), lens, counts=True)
    elif kind == "csr_counts":
        gpu = CobaNetwork(n, n_e, conn="csr", seed=seed, p=p, V0=V0, keep_spk=True)
        ref = orc.CobaNet(n, n_e, ("jit", se, si, K), V0.astype(np.float64))
        c = Case(gpu, ref, jit_deliver(se, si, K, n, n_e), lens, counts=True)
    else:
        dt = torch.float32 if kind == "csr_f32" else torch.bfloat16
        csr = materialize_network_csr(seed, p, n, n_e, data_dtype=dt)
        we, wi = (float(torch.tensor(w, dtype=dt).to(torch.float64)) for w in (W_E, W_I))
        gpu = CobaNetwork(n, n_e, conn="csr", csr=csr, seed=seed, p=p, V0=V0, keep_spk=True)
        ref = orc.CobaNet(n, n_e, ("jit", se, si, K), V0.astype(np.float64), w_e=1.0, w_i=1.0)
        unrounded = jit_deliver(se, si, K, n, n_e, W_E, W_I) if kind == "csr_bf16" else None
        c = Case(gpu, ref, jit_deliver(se, si, K, n, n_e, we, wi), lens, counts=False,
                 deliver_unrounded=unrounded, ref_scale=(we, wi))
    spikes = 0
    for _ in range(3):
        spikes += teacher_forced_step(c, max_flips=8)[0]
    gpu.simulate(27)
    for _ in range(3):
        spikes += teacher_forced_step(c, max_flips=8)[0]
    assert spikes > 100_000
    gpu.close()
