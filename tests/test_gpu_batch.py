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


@pytest.mark.parametrize("conn", ["jit", "csr"])
def test_batch_equals_single_network_path(conn):
    sizes, seeds, V0 = make_batch(12, 1000, 9000, seed=3)
    sizes[0] = 1003                     # a size that is not a multiple of 4
    V0[0] = wl.coba_v0(1003, seed=100)
    bat = BatchedNetworks(sizes, seeds, V0=V0, conn=conn)
    T = 230
    bat.simulate(T)
    torch.cuda.synchronize()
    for b in [0, 3, 7, 11]:
        single = CobaNetwork(int(sizes[b]), conn=conn, seed=int(seeds[b]), V0=V0[b])
        single.simulate(T)
        assert torch.equal(bat.view(bat.V, b), single.V), b
        assert torch.equal(bat.view(bat.ref, b), single.ref), b
        t = bat.totals[b].cpu().numpy()
        s = single.totals.cpu().numpy()
        assert t[0] == s[0] and t[1] == s[1] and t[2] == s[2] and t[3] == T
        single.close()
    bat.close()


@pytest.mark.parametrize("conn", ["jit", "csr"])
def test_batch_sampled_networks_match_oracle(conn):
    """Networks of a batch against the FP64 oracle over 60 free-running steps.
    Only networks whose oracle run never met a threshold decision within
    1e-3 mV of V_th are compared (elsewhere FP32 and FP64 may legitimately
    part); the seeds give several such networks, and for each the spike
    totals and event totals are exact and V, g_e, g_i agree within 1e-5
    relative."""
    sizes, seeds, V0 = make_batch(12, 1000, 4000, seed=5)
    bat = BatchedNetworks(sizes, seeds, V0=V0, conn=conn)
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


@pytest.mark.parametrize("conn", ["jit", "csr"])
def test_autotune_restores_state_and_continues(conn):
    sizes, seeds, V0 = make_batch(40, 1000, 20000, seed=7)
    a = BatchedNetworks(sizes, seeds, V0=V0, conn=conn)
    b = BatchedNetworks(sizes, seeds, V0=V0, conn=conn)
    a.simulate(50)
    b.simulate(50)
    th = a.autotune(probe_steps=10)
    assert th in (256, 512, 1024)
    t_th, t_g, t_ps, t_csr = a.tuning()
    assert t_th == th and t_csr == (conn == "csr") and t_ps in (1, 2)
    assert t_g in ((4, 8, 16, 32) if conn == "csr" else (16, 32))
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


@pytest.mark.parametrize("conn", ["jit", "csr"])
def test_every_tuning_computes_the_same_trajectories(conn):
    """CTA size, lanes per delivered row and bins per SM change only how the
    work is spread: with integer event counts every tuning gives the same
    potentials, counters and totals bit for bit (networks small enough for
    packings of 1, 2 and 4 CTAs per SM)."""
    sizes, seeds, V0 = make_batch(60, 1000, 12000, seed=21)
    groups = (4, 8, 16, 32) if conn == "csr" else (16, 32)
    tunings = [(1024, groups[0], 1), (256, groups[-1], 4), (512, groups[1], 2), (256, groups[0], 2),
               (1024, groups[-1], 1)]
    ref = None
    for th, g, ps in tunings:
        bat = BatchedNetworks(sizes, seeds, V0=V0, conn=conn)
        bat.set_tuning(th, g, ps)
        assert bat.tuning() == (th, g, ps, int(conn == "csr"))
        bat.simulate(120)
        torch.cuda.synchronize()
        got = (bat.V.clone(), bat.ref.clone(), bat.totals.clone())
        if ref is None:
            ref = got
            assert int(got[2][:, 2].sum().item()) > 0
        else:
            assert all(torch.equal(x, y) for x, y in zip(got, ref)), (th, g, ps)
        bat.close()


def test_batch_rejects_invalid_stored_rows():
    """bp_batch_create validates stored rows on the device: a repeated column,
    a target outside its network and an entry in a padding row are each
    rejected (the packed counts and the shared-memory targets rely on them)."""
    from paper_2311_05106_gb300.network import batch_csr
    sizes = np.array([1003, 2000, 1500], np.int64)
    seeds = np.array([1, 2, 3], np.uint64)
    off = B.bp_batch_layout(sizes)
    ip, ix = batch_csr(sizes, seeds, off)
    BatchedNetworks(sizes, seeds, conn="csr", csr=(ip, ix)).close()
    r = int(off[1]) + 5                         # a row of network 1 with >= 2 entries
    while int(ip[r + 1] - ip[r]) < 2:
        r += 1
    bad = ix.clone()
    bad[int(ip[r]) + 1] = bad[int(ip[r])]       # repeated column
    with pytest.raises(B.BpError):
        BatchedNetworks(sizes, seeds, conn="csr", csr=(ip, bad))
    bad = ix.clone()
    bad[int(ip[r + 1]) - 1] = 2000              # outside network 1 (n = 2000)
    with pytest.raises(B.BpError):
        BatchedNetworks(sizes, seeds, conn="csr", csr=(ip, bad))
    bip = ip.clone()
    bip[1003 + 1:] += 1                         # padding row 1003 of network 0 gets an entry
    bix = torch.cat([ix[:int(ip[1003])], torch.zeros(1, dtype=torch.int32, device="cuda"), ix[int(ip[1003]):]])
    with pytest.raises(B.BpError):
        BatchedNetworks(sizes, seeds, conn="csr", csr=(bip, bix))
