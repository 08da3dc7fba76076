"""GPU parity of the batched networks (a9).

* Every network of a batch follows, bit for bit, the trajectory that the
  single-network path (itself pinned to the oracle) computes for it: same
  FP32 arithmetic, exact integer event counts.
* Sampled networks agree with the FP64 oracle until a near-threshold flip.
* Autotuning restores the state it probes from; totals are consistent.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc
from paper_2311_05106_gb300 import binding as B
from paper_2311_05106_gb300 import workloads as wl
from paper_2311_05106_gb300.network import BatchedNetworks, CobaNetwork

pytestmark = pytest.mark.gpu


def make_batch(n_nets, lo, hi, seed):
    sizes = wl.batched_sizes(n_nets, lo, hi, seed=seed)
    seeds = np.arange(n_nets, dtype=np.uint64) * 7919 + 17
    V0 = [wl.coba_v0(int(n), seed=100 + b) for b, n in enumerate(sizes)]
    return sizes, seeds, V0


def test_batch_equals_single_network_path():
    sizes, seeds, V0 = make_batch(12, 1000, 9000, seed=3)
    sizes[0] = 1003                     # a size that is not a multiple of 4
    V0[0] = wl.coba_v0(1003, seed=100)
    bat = BatchedNetworks(sizes, seeds, V0=V0)
    T = 230
    bat.simulate(T)
    torch.cuda.synchronize()
    for b in [0, 3, 7, 11]:
        single = CobaNetwork(int(sizes[b]), conn="jit", seed=int(seeds[b]), V0=V0[b])
        single.simulate(T)
        assert torch.equal(bat.view(bat.V, b), single.V), b
        assert torch.equal(bat.view(bat.ref, b), single.ref), b
        t = bat.totals[b].cpu().numpy()
        s = single.totals.cpu().numpy()
        assert t[0] == s[0] and t[1] == s[1] and t[2] == s[2] and t[3] == T
        single.close()
    bat.close()


def test_batch_sampled_networks_match_oracle():
    """Networks of a batch against the FP64 oracle over 60 free-running steps.
    Only networks whose oracle run never met a threshold decision within
    1e-3 mV of V_th are compared (elsewhere FP32 and FP64 may legitimately
    part); the seeds give several such networks, and for each the spike
    totals and event totals are exact and V, g_e, g_i agree within 1e-5
    relative."""
    sizes, seeds, V0 = make_batch(12, 1000, 4000, seed=5)
    bat = BatchedNetworks(sizes, seeds, V0=V0)
    T = 60
    bat.simulate(T)
    torch.cuda.synchronize()
    V, ge, gi = (t.cpu().numpy() for t in (bat.V, bat.ge, bat.gi))
    ref_c = bat.ref.cpu().numpy()
    tot = bat.totals.cpu().numpy()
    compared = 0
    for b in range(len(sizes)):
        n = int(sizes[b])
        n_e = (4 * n) // 5
        K = orc.jit_K(80.0 / n)
        se, si = orc.projection_seed(int(seeds[b]), 0), orc.projection_seed(int(seeds[b]), 1)
        ref = orc.CobaNet(n, n_e, ("jit", se, si, K), V0[b].astype(np.float64))
        lens = np.concatenate([orc.jit_row_lengths(se, K, n_e, n), orc.jit_row_lengths(si, K, n - n_e, n)])
        near = False
        spikes_e = spikes_i = events = 0
        for _ in range(T):
            spk, vdec = ref.step(return_vdec=True)
            if np.nanmin(np.abs(vdec + 50.0)) < 1e-3:
                near = True
                break
            spikes_e += int(spk[:n_e].sum())
            spikes_i += int(spk[n_e:].sum())
            events += int(lens[spk.astype(bool)].sum())
        if near:
            continue
        o = int(bat.off[b])
        sl = slice(o, o + n)
        for got, want in ((V[sl], ref.V), (ge[sl], ref.ge), (gi[sl], ref.gi)):
            scale = max(np.abs(want).max(), 1e-30)
            assert np.max(np.abs(got.astype(np.float64) - want)) / scale <= 1e-5, b
        assert np.array_equal(ref_c[sl].astype(np.int32), ref.ref), b
        assert tot[b, 0] == spikes_e and tot[b, 1] == spikes_i and tot[b, 2] == events and tot[b, 3] == T, b
        compared += 1
    assert compared >= 3
    bat.close()


def test_autotune_restores_state_and_continues():
    sizes, seeds, V0 = make_batch(40, 1000, 20000, seed=7)
    a = BatchedNetworks(sizes, seeds, V0=V0)
    b = BatchedNetworks(sizes, seeds, V0=V0)
    a.simulate(50)
    b.simulate(50)
    th = a.autotune(probe_steps=10)
    assert th in (256, 512, 1024)
    assert torch.equal(a.V, b.V) and torch.equal(a.totals, b.totals)
    a.simulate(120)
    b.simulate(120)
    assert torch.equal(a.V, b.V) and torch.equal(a.ref, b.ref) and torch.equal(a.totals, b.totals)
    bins, threads, total = a.info()
    assert threads == th and total == int(a.off[-1]) and 1 <= bins
    a.close()
    b.close()


def test_batch_rejects_oversized_network():
    with pytest.raises(B.BpError):
        BatchedNetworks(np.array([70000]), np.array([1], np.uint64))


def test_full_size_batch_networks_equal_single_path():
    """The batched configuration as the bench runs it: 256 networks,
    N ~ U[1000, 50000] (seed 11), autotuned, 200 steps; four networks
    (including the largest and the smallest) equal the single-network path
    bit for bit, and the totals are consistent."""
    sizes = wl.batched_sizes(256, 1000, 50000, seed=11)
    seeds = np.arange(256, dtype=np.uint64) * np.uint64(7919) + np.uint64(2024)
    V0 = [wl.coba_v0(int(n), seed=1000 + b) for b, n in enumerate(sizes)]
    bat = BatchedNetworks(sizes, seeds, V0=V0)
    bat.autotune(probe_steps=10)
    T = 200
    bat.simulate(T)
    torch.cuda.synchronize()
    picks = sorted({int(np.argmax(sizes)), int(np.argmin(sizes)), 17, 200})
    for b in picks:
        single = CobaNetwork(int(sizes[b]), conn="jit", seed=int(seeds[b]), V0=V0[b])
        single.simulate(T)
        assert torch.equal(bat.view(bat.V, b), single.V), b
        assert torch.equal(bat.view(bat.ref, b), single.ref), b
        t = bat.totals[b].cpu().numpy()
        s = single.totals.cpu().numpy()
        assert t[0] == s[0] and t[1] == s[1] and t[2] == s[2] and t[3] == T
        single.close()
    tot = bat.totals.cpu().numpy()
    assert np.all(tot[:, 3] == T) and tot[:, 0].sum() > 0
    bat.close()
