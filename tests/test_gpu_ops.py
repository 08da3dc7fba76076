"""GPU parity of the operators (a1-a6) against the FP64 oracle, through the C ABI.

Tolerances: integer event counts and index work are bit-exact; FP32 results
must be within 1e-5 of the oracle in the relative-to-max norm
max|gpu - ref| / max|ref| (per array); BF16-stored weights are compared with
the oracle fed the same BF16-rounded weights (1e-5) and with the unrounded
FP32 weights (1e-2).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc
from paper_2311_05106_gb300 import binding as B
from paper_2311_05106_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

RTOL_F32 = 1e-5
RTOL_BF16 = 1e-2


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-30))


def cuda(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def spike_list_of(events):
    ids = np.nonzero(events)[0].astype(np.int32)
    sl = torch.zeros(max(len(events), 1), dtype=torch.int32, device="cuda")
    if len(ids):
        sl[: len(ids)] = cuda(ids)
    ns = torch.tensor([len(ids)], dtype=torch.int32, device="cuda")
    return sl, ns


# ---------------------------------------------------------------------- a1-a4
@pytest.mark.parametrize("n,counts,tau_ref", [(1, True, 5.0), (255, True, 5.0), (70001, True, 5.0),
                                               (70001, False, 5.0), (300000, True, 5.0), (70001, True, 25.5)])
def test_lif_step_matches_oracle(n, counts, tau_ref):
    """One step from a random state against the oracle; tau_ref = 25.5 ms is
    the longest refractory period the one-byte counters hold (255 steps)."""
    ref_steps = int(round(tau_ref / 0.1))
    st = wl.lif_state(n, seed=n, ref_steps=ref_steps)
    n_e = (4 * n) // 5
    empty = ("csr", np.zeros(n + 1, np.int64), np.zeros(1, np.int32), None if counts else np.zeros(1))
    net = orc.CobaNet(n, n_e, empty, st["V"].astype(np.float64), tau_ref=tau_ref)
    net.ge[:] = st["ge"]
    net.gi[:] = st["gi"]
    net.ref[:] = st["ref"]
    ye_in = st["ce"] if counts else (st["ce"] * 0.37).astype(np.float32)
    yi_in = st["ci"] if counts else (st["ci"] * 1.9).astype(np.float32)
    net.ye[:] = ye_in
    net.yi[:] = yi_in
    spk_ref, vdec = net.step(return_vdec=True)

    p = B.bp_coba_params_default(tau_ref=tau_ref)
    V, ge, gi, ref = cuda(st["V"]), cuda(st["ge"]), cuda(st["gi"]), cuda(st["ref"].astype(np.uint8))
    ye, yi = cuda(ye_in), cuda(yi_in)
    spk = torch.zeros(n, dtype=torch.uint8, device="cuda")
    sl = torch.zeros(n, dtype=torch.int32, device="cuda")
    ns = torch.zeros(1, dtype=torch.int32, device="cuda")
    tot = torch.zeros(2, dtype=torch.int64, device="cuda")
    B.bp_lif_step(p, n_e, V, ge, gi, ref, ye, yi, sl, ns, spk=spk, spike_totals=tot)
    torch.cuda.synchronize()

    assert rel_err(ge.cpu().numpy(), net.ge) < RTOL_F32
    assert rel_err(gi.cpu().numpy(), net.gi) < RTOL_F32
    near = np.abs(np.nan_to_num(vdec, nan=1e9) - (-50.0)) < 1e-4
    s_gpu = spk.cpu().numpy()
    assert np.array_equal(s_gpu[~near], spk_ref[~near])
    ok = ~near
    assert rel_err(V.cpu().numpy()[ok], net.V[ok]) < RTOL_F32
    assert np.array_equal(ref.cpu().numpy()[ok], net.ref[ok])
    if n >= 70001:  # counters set by this step's spikes and counters counting down from the top
        assert (net.ref[ok] == ref_steps).any() and (net.ref[ok] == ref_steps - 1).any()
    assert not ye.any().item() and not yi.any().item()
    k = int(ns.item())
    ids = np.sort(sl[:k].cpu().numpy())
    assert np.array_equal(ids, np.nonzero(s_gpu)[0])
    t = tot.cpu().numpy()
    assert t[0] == s_gpu[:n_e].sum() and t[1] == s_gpu[n_e:].sum()


def test_spike_compact():
    for n, rho in [(1, 1.0), (1000, 0.0), (123457, 0.01), (500000, 0.5)]:
        ev = wl.bernoulli_spikes(n, rho, seed=n)
        sl = torch.zeros(n, dtype=torch.int32, device="cuda")
        ns = torch.zeros(1, dtype=torch.int32, device="cuda")
        B.bp_spike_compact(cuda(ev), sl, ns)
        k = int(ns.item())
        assert k == ev.sum()
        assert np.array_equal(np.sort(sl[:k].cpu().numpy()), np.nonzero(ev)[0])


# ---------------------------------------------------------------------- a5
CSR_CASES = [
    # n_pre, n_post, p, rho
    (1, 1, 1.0, 1.0),
    (300, 257, 0.1, 0.3),
    (5000, 4001, 0.02, 0.05),
    (2000, 150001, 0.004, 0.2),     # several post tiles and a ragged tail
    (20000, 30000, 0.001, 0.0),     # no spikes
]


def _csr(n_pre, n_post, p, seed):
    ip, ix = wl.random_csr(n_pre, n_post, p, seed)
    return ip, ix


@pytest.mark.parametrize("case", CSR_CASES)
@pytest.mark.parametrize("flags", [0, B.BP_ACC_GLOBAL, B.BP_ACC_SHARED])
def test_event_csrmv_counts_bit_exact(case, flags):
    n_pre, n_post, p, rho = case
    ip, ix = _csr(n_pre, n_post, p, seed=n_pre)
    ev = wl.bernoulli_spikes(n_pre, rho, seed=n_pre + 1)
    expect = orc.event_csr_count(ip, ix, ev, n_post)
    dip, dix = cuda(ip), cuda(ix)
    tcols = B.bp_tile_cols() if n_post > B.bp_tile_cols() else 0
    tp = None
    if tcols:
        tp = torch.empty(B.bp_csr_tile_index_size(n_pre, n_post, tcols), dtype=torch.int32, device="cuda")
        B.bp_csr_tile_index(dip, dix, n_post, tcols, tp)
    sl, ns = spike_list_of(ev)
    y = torch.zeros(n_post, dtype=torch.int32, device="cuda")
    B.bp_event_csrmv(dip, dix, None, 1.0, sl, ns, y, tile_ptr=tp, tile_cols=tcols, flags=flags)
    assert np.array_equal(y.cpu().numpy(), expect)
    # accumulate semantics: a second call doubles; BP_OVERWRITE resets
    B.bp_event_csrmv(dip, dix, None, 1.0, sl, ns, y, tile_ptr=tp, tile_cols=tcols, flags=flags)
    assert np.array_equal(y.cpu().numpy(), 2 * expect)
    B.bp_event_csrmv(dip, dix, None, 1.0, sl, ns, y, tile_ptr=tp, tile_cols=tcols, flags=flags | B.BP_OVERWRITE)
    assert np.array_equal(y.cpu().numpy(), expect)


@pytest.mark.parametrize("case", CSR_CASES[1:4])
@pytest.mark.parametrize("flags", [0, B.BP_ACC_GLOBAL, B.BP_ACC_SHARED])
def test_event_csrmv_float_weights(case, flags):
    n_pre, n_post, p, rho = case
    ip, ix = _csr(n_pre, n_post, p, seed=n_pre + 7)
    w = wl.normal_weights(len(ix), 0.5, 0.1, seed=3)
    ev = wl.bernoulli_spikes(n_pre, rho, seed=11)
    dip, dix = cuda(ip), cuda(ix)
    tcols = B.bp_tile_cols() if n_post > B.bp_tile_cols() else 0
    tp = None
    if tcols:
        tp = torch.empty(B.bp_csr_tile_index_size(n_pre, n_post, tcols), dtype=torch.int32, device="cuda")
        B.bp_csr_tile_index(dip, dix, n_post, tcols, tp)
    sl, ns = spike_list_of(ev)
    # FP32 weights
    y = torch.zeros(n_post, dtype=torch.float32, device="cuda")
    B.bp_event_csrmv(dip, dix, cuda(w), 0.0, sl, ns, y, tile_ptr=tp, tile_cols=tcols, flags=flags)
    ref = orc.event_csrmv(ip, ix, w.astype(np.float64), ev, n_post)
    assert rel_err(y.cpu().numpy(), ref) < RTOL_F32
    # BF16 weights
    wb = cuda(w).to(torch.bfloat16)
    yb = torch.zeros(n_post, dtype=torch.float32, device="cuda")
    B.bp_event_csrmv(dip, dix, wb, 0.0, sl, ns, yb, tile_ptr=tp, tile_cols=tcols, flags=flags)
    ref_b = orc.event_csrmv(ip, ix, wb.float().cpu().numpy().astype(np.float64), ev, n_post)
    assert rel_err(yb.cpu().numpy(), ref_b) < RTOL_F32
    assert rel_err(yb.cpu().numpy(), ref) < RTOL_BF16
    # homogeneous float weight
    yh = torch.zeros(n_post, dtype=torch.float32, device="cuda")
    B.bp_event_csrmv(dip, dix, None, 0.6, sl, ns, yh, tile_ptr=tp, tile_cols=tcols, flags=flags)
    assert rel_err(yh.cpu().numpy(), orc.event_csrmv(ip, ix, None, ev, n_post, w_homo=0.6)) < RTOL_F32


def test_event_csrmv_float_weights_many_rows_per_cta():
    """FP32 and BF16 weights with enough spiking rows per post tile that each
    CTA fetches the segment bounds of its rows in batches of one per thread
    (two batches, the second partial): the sums match the oracle's."""
    n_pre, n_post, p = 120_000, 150_001, 0.002
    ip, ix = _csr(n_pre, n_post, p, seed=5)
    w = wl.normal_weights(len(ix), 0.5, 0.1, seed=6)
    ev = wl.bernoulli_spikes(n_pre, 0.5, seed=7)
    dip, dix = cuda(ip), cuda(ix)
    tcols = B.bp_tile_cols()
    tp = torch.empty(B.bp_csr_tile_index_size(n_pre, n_post, tcols), dtype=torch.int32, device="cuda")
    B.bp_csr_tile_index(dip, dix, n_post, tcols, tp)
    sl, ns = spike_list_of(ev)
    ref = orc.event_csrmv(ip, ix, w.astype(np.float64), ev, n_post)
    y = torch.zeros(n_post, dtype=torch.float32, device="cuda")
    B.bp_event_csrmv(dip, dix, cuda(w), 0.0, sl, ns, y, tile_ptr=tp, tile_cols=tcols, flags=B.BP_ACC_SHARED)
    assert rel_err(y.cpu().numpy(), ref) < RTOL_F32
    wb = cuda(w).to(torch.bfloat16)
    yb = torch.zeros(n_post, dtype=torch.float32, device="cuda")
    B.bp_event_csrmv(dip, dix, wb, 0.0, sl, ns, yb, tile_ptr=tp, tile_cols=tcols, flags=B.BP_ACC_SHARED)
    ref_b = orc.event_csrmv(ip, ix, wb.float().cpu().numpy().astype(np.float64), ev, n_post)
    assert rel_err(yb.cpu().numpy(), ref_b) < RTOL_F32


def test_event_csrmv_dense_events():
    n_pre, n_post = 7000, 9000
    ip, ix = _csr(n_pre, n_post, 0.01, seed=5)
    ev = wl.bernoulli_spikes(n_pre, 0.1, seed=6)
    ws = torch.zeros(B.bp_event_csrmv_dense_workspace_bytes(n_pre), dtype=torch.uint8, device="cuda")
    y = torch.zeros(n_post, dtype=torch.int32, device="cuda")
    B.bp_event_csrmv_dense(cuda(ip), cuda(ix), None, 1.0, cuda(ev), ws, y)
    assert np.array_equal(y.cpu().numpy(), orc.event_csr_count(ip, ix, ev, n_post))


def test_tile_index_matches_searchsorted():
    n_pre, n_post, tc = 3000, 200000, B.bp_tile_cols()
    ip, ix = _csr(n_pre, n_post, 0.002, seed=9)
    tp = torch.empty(B.bp_csr_tile_index_size(n_pre, n_post, tc), dtype=torch.int32, device="cuda")
    B.bp_csr_tile_index(cuda(ip), cuda(ix), n_post, tc, tp)
    S = -(-n_post // tc)
    flat = tp.cpu().numpy()
    assert flat.size == n_pre * (S + 1) + 2 and flat[-1] == 0 and flat[-2] == 0  # the bound slots start empty
    got = flat[:-2].reshape(n_pre, S + 1)
    for i in range(0, n_pre, 37):
        row = ix[ip[i]:ip[i + 1]]
        bounds = np.searchsorted(row, np.arange(S) * tc, side="left")
        assert np.array_equal(got[i, :S], bounds)
        assert got[i, S] == len(row)


@pytest.mark.parametrize("wdt", [None, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("form", ["l2", "one_tile", "one_tile_overwrite"])
def test_csrmv_t_gather(wdt, form):
    """Gather through L2, and with a one-tile index (x wholly in shared
    memory, each row written by one owner)."""
    n_pre, n_post = 6000, 5000
    ip, ix = _csr(n_pre, n_post, 0.01, seed=13)
    w = wl.normal_weights(len(ix), 0.0, 1.0, seed=14)
    x = np.random.default_rng(1).normal(size=n_post).astype(np.float32)
    dw = None if wdt is None else cuda(w).to(wdt)
    wref = None if wdt is None else dw.float().cpu().numpy().astype(np.float64)
    y = torch.full((n_pre,), 0.25, dtype=torch.float32, device="cuda")
    tp, tc = None, 0
    if form != "l2":
        tc = (n_post + 31) // 32 * 32
        tp = torch.empty(B.bp_csr_tile_index_size(n_pre, n_post, tc), dtype=torch.int32, device="cuda")
        B.bp_csr_tile_index(cuda(ip), cuda(ix), n_post, tc, tp)
    flags = B.BP_OVERWRITE if form == "one_tile_overwrite" else 0
    B.bp_event_csrmv_t(cuda(ip), cuda(ix), dw, 0.6, cuda(x), y, flags=flags, tile_ptr=tp, tile_cols=tc)
    base = 0.0 if flags else 0.25
    ref = base + orc.csrmv_t(ip, ix, wref, x.astype(np.float64), w_homo=0.6)
    assert rel_err(y.cpu().numpy(), ref) < RTOL_F32


@pytest.mark.parametrize("wdt", [None, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("mode", ["tiles", "l2", "tiles_overwrite"])
def test_csrmv_t_gather_tiles(wdt, mode):
    """n_post = 130 000 spans three shared-memory tiles of x (57 344 columns,
    ragged last tile): the tiled gather, the L2 gather and the overwrite form
    against the oracle's sequential product."""
    n_pre, n_post = 7001, 130000
    ip, ix = _csr(n_pre, n_post, 0.002, seed=23)
    w = wl.normal_weights(len(ix), 0.0, 1.0, seed=24)
    x = np.random.default_rng(2).normal(size=n_post).astype(np.float32)
    dw = None if wdt is None else cuda(w).to(wdt)
    wref = None if wdt is None else dw.float().cpu().numpy().astype(np.float64)
    tc = B.bp_tile_cols()
    tp = torch.empty(B.bp_csr_tile_index_size(n_pre, n_post, tc), dtype=torch.int32, device="cuda")
    B.bp_csr_tile_index(cuda(ip), cuda(ix), n_post, tc, tp)
    y = torch.full((n_pre,), 0.25, dtype=torch.float32, device="cuda")
    flags = {"tiles": 0, "l2": B.BP_ACC_GLOBAL, "tiles_overwrite": B.BP_OVERWRITE}[mode]
    B.bp_event_csrmv_t(cuda(ip), cuda(ix), dw, 0.6, cuda(x), y, flags=flags, tile_ptr=tp, tile_cols=tc)
    base = 0.0 if mode == "tiles_overwrite" else 0.25
    ref = base + orc.csrmv_t(ip, ix, wref, x.astype(np.float64), w_homo=0.6)
    assert rel_err(y.cpu().numpy(), ref) < RTOL_F32


def test_csrmv_bwd():
    n_pre, n_post = 3000, 4000
    ip, ix = _csr(n_pre, n_post, 0.02, seed=15)
    w = wl.normal_weights(len(ix), 0.0, 1.0, seed=16)
    ev = wl.bernoulli_spikes(n_pre, 0.2, seed=17)
    dy = np.random.default_rng(2).normal(size=n_post).astype(np.float32)
    sl, ns = spike_list_of(ev)
    dwt = torch.zeros(len(ix), dtype=torch.float32, device="cuda")
    dx = torch.zeros(n_pre, dtype=torch.float32, device="cuda")
    B.bp_event_csrmv_bwd(cuda(ip), cuda(ix), cuda(w), 0.0, sl, ns, cuda(dy), dw=dwt, dx_pre=dx)
    # each entry receives exactly one addition onto zero: bit-exact
    assert np.array_equal(dwt.cpu().numpy(), orc.event_csrmv_dw(ip, ix, ev, dy.astype(np.float64)).astype(np.float32))
    assert rel_err(dx.cpu().numpy(), orc.csrmv_t(ip, ix, w.astype(np.float64), dy.astype(np.float64))) < RTOL_F32


# ---------------------------------------------------------------------- a6
@pytest.mark.parametrize("n_pre,n_post,p", [(1, 1, 1.0), (3000, 2500, 0.05), (4000, 4000, 0.02), (500, 100000, 0.01)])
def test_jit_materialize_bit_exact(n_pre, n_post, p):
    seed = 1234 + n_pre
    d = B.bp_jit_desc_init(seed, p)
    K = orc.jit_K(p)
    assert d.K == K
    ip, ix, _ = B.jit_materialize(d, n_pre, n_post)
    eip, eix, _ = orc.jit_materialize(seed, K, n_pre, n_post)
    assert np.array_equal(ip.cpu().numpy(), eip)
    assert np.array_equal(ix.cpu().numpy(), eix)


@pytest.mark.parametrize("wkind,w0,w1", [(B.BP_JIT_UNIFORM, -0.5, 1.5), (B.BP_JIT_NORMAL, 0.5, 0.1)])
def test_jit_materialized_weights(wkind, w0, w1):
    n_pre, n_post, p, seed = 800, 3000, 0.05, 77
    d = B.bp_jit_desc_init(seed, p, wkind, w0, w1)
    ip, ix, data = B.jit_materialize(d, n_pre, n_post, data_dtype=torch.float32)
    eip, eix, edata = orc.jit_materialize(seed, orc.jit_K(p), n_pre, n_post, wkind, w0, w1)
    assert np.array_equal(ix.cpu().numpy(), eix)
    assert rel_err(data.cpu().numpy(), edata) < RTOL_F32


# (2000, 100000, 0.01, 0.05) and (500, 50000, 0.05, 0.1): few long rows, walked
# by whole CTAs (L2 and shared-memory accumulation)
@pytest.mark.parametrize("n_pre,n_post,p,rho", [(3000, 3000, 0.05, 0.1), (2000, 100000, 0.01, 0.05),
                                                (50000, 60000, 0.001, 0.01), (500, 50000, 0.05, 0.1)])
@pytest.mark.parametrize("flags", [0, B.BP_ACC_GLOBAL])
def test_jitconn_event_mv_counts_bit_exact(n_pre, n_post, p, rho, flags):
    seed = 99 + n_pre
    d = B.bp_jit_desc_init(seed, p)
    ev = wl.bernoulli_spikes(n_pre, rho, seed=3)
    sl, ns = spike_list_of(ev)
    y = torch.zeros(n_post, dtype=torch.int32, device="cuda")
    B.bp_jitconn_event_mv(d, n_pre, sl, ns, y, flags=flags)
    expect = orc.jitconn_event_mv(seed, orc.jit_K(p), n_pre, n_post, ev)
    assert np.array_equal(y.cpu().numpy(), expect.astype(np.int64))


@pytest.mark.parametrize("wkind,w0,w1", [(B.BP_JIT_HOMO, 0.6, 0.0), (B.BP_JIT_UNIFORM, 0.0, 1.0),
                                         (B.BP_JIT_NORMAL, 0.5, 0.1)])
def test_jitconn_float_products(wkind, w0, w1):
    n_pre, n_post, p, seed = 4000, 5000, 0.02, 5
    K = orc.jit_K(p)
    d = B.bp_jit_desc_init(seed, p, wkind, w0, w1)
    ev = wl.bernoulli_spikes(n_pre, 0.1, seed=8)
    sl, ns = spike_list_of(ev)
    y = torch.zeros(n_post, dtype=torch.float32, device="cuda")
    B.bp_jitconn_event_mv(d, n_pre, sl, ns, y)
    assert rel_err(y.cpu().numpy(), orc.jitconn_event_mv(seed, K, n_pre, n_post, ev, wkind, w0, w1)) < RTOL_F32
    x = np.random.default_rng(3).normal(size=n_pre).astype(np.float32)
    yy = torch.zeros(n_post, dtype=torch.float32, device="cuda")
    B.bp_jitconn_mv(d, cuda(x), yy)
    assert rel_err(yy.cpu().numpy(), orc.jitconn_mv(seed, K, n_pre, n_post, x.astype(np.float64), wkind, w0,
                                                    w1)) < RTOL_F32
    dy = np.random.default_rng(4).normal(size=n_post).astype(np.float32)
    dx = torch.zeros(n_pre, dtype=torch.float32, device="cuda")
    B.bp_jitconn_event_mv_bwd(d, cuda(dy), dx)
    assert rel_err(dx.cpu().numpy(), orc.jitconn_mv_t(seed, K, n_pre, n_post, dy.astype(np.float64), wkind, w0,
                                                      w1)) < RTOL_F32


@pytest.mark.parametrize("wkind,w0,w1", [(B.BP_JIT_UNIFORM, 0.0, 1.0), (B.BP_JIT_NORMAL, 0.5, 0.1)])
def test_jitconn_float_few_long_rows(wkind, w0, w1):
    """About 30 spiking rows of ~1 600 targets: the whole-CTA row walk with
    drawn weights against the oracle."""
    n_pre, n_post, p, seed = 300, 80000, 0.02, 41
    K = orc.jit_K(p)
    d = B.bp_jit_desc_init(seed, p, wkind, w0, w1)
    ev = wl.bernoulli_spikes(n_pre, 0.1, seed=42)
    sl, ns = spike_list_of(ev)
    y = torch.zeros(n_post, dtype=torch.float32, device="cuda")
    B.bp_jitconn_event_mv(d, n_pre, sl, ns, y)
    assert rel_err(y.cpu().numpy(), orc.jitconn_event_mv(seed, K, n_pre, n_post, ev, wkind, w0, w1)) < RTOL_F32


def test_jit_and_stored_csr_agree_on_gpu():
    n_pre, n_post, p, seed = 20000, 20000, 0.004, 31
    d = B.bp_jit_desc_init(seed, p)
    ip, ix, _ = B.jit_materialize(d, n_pre, n_post)
    ev = wl.bernoulli_spikes(n_pre, 0.05, seed=32)
    sl, ns = spike_list_of(ev)
    a = torch.zeros(n_post, dtype=torch.int32, device="cuda")
    b = torch.zeros(n_post, dtype=torch.int32, device="cuda")
    B.bp_jitconn_event_mv(d, n_pre, sl, ns, a)
    B.bp_event_csrmv(ip, ix, None, 1.0, sl, ns, b)
    assert torch.equal(a, b)


def test_invalid_arguments_rejected_on_host():
    d = B.bp_jit_desc_init(1, 0.1)
    y = torch.zeros(10, dtype=torch.float32, device="cuda")
    sl = torch.zeros(10, dtype=torch.int32, device="cuda")
    ns = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(B.BpError):
        B.bp_jit_desc_init(1, 0.0)
    with pytest.raises(B.BpError):
        B.bp_jit_desc_init(1, 1.5)
    with pytest.raises(B.BpError):   # counts with non-homogeneous weights
        B.bp_event_csrmv(cuda(np.zeros(11, np.int64)), cuda(np.zeros(1, np.int32)), cuda(np.zeros(1, np.float32)),
                         0.0, sl, ns, torch.zeros(10, dtype=torch.int32, device="cuda"))
    with pytest.raises(B.BpError):   # max_spikes beyond n_pre
        B.bp_jitconn_event_mv(d, 10, sl, ns, y, max_spikes=11)
    assert B.bp_sync_status() == 0


# ---------------------------------------------------------------------- degenerate cases
@pytest.mark.parametrize("n_post", [1000, 70000])
def test_jit_p_one_hits_every_column(n_post):
    """p = 1 gives K = 1: every gap is 1, so every spiking row targets every
    column once; counts equal the number of spikes everywhere (and the
    oracle's), in shared-memory (n_post <= 57 344) and L2 accumulation."""
    n_pre = 300
    d = B.bp_jit_desc_init(5, 1.0)
    assert d.K == 1
    ev = wl.bernoulli_spikes(n_pre, 0.3, seed=6)
    sl, ns = spike_list_of(ev)
    y = torch.zeros(n_post, dtype=torch.int32, device="cuda")
    B.bp_jitconn_event_mv(d, n_pre, sl, ns, y)
    got = y.cpu().numpy()
    assert np.all(got == int(ev.sum()))
    assert np.array_equal(got, orc.jitconn_event_mv(5, 1, n_pre, n_post, ev).astype(np.int64))


@pytest.mark.parametrize("flags", [0, B.BP_ACC_GLOBAL, B.BP_ACC_SHARED])
def test_scatter_into_one_column(flags):
    """Every row holds the single column 0: all events collide on one
    accumulator (integer counts: exactly the number of spikes)."""
    n_pre = 50000
    ip = np.arange(n_pre + 1, dtype=np.int64)
    ix = np.zeros(n_pre, np.int32)
    ev = wl.bernoulli_spikes(n_pre, 0.5, seed=9)
    sl, ns = spike_list_of(ev)
    y = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.bp_event_csrmv(cuda(ip), cuda(ix), None, 1.0, sl, ns, y, flags=flags)
    assert int(y.item()) == int(ev.sum())


def test_matrix_without_entries():
    """No stored entries at all: the scatter and both gather forms leave their
    outputs as they were."""
    n_pre, n_post = 5000, 100000
    ip = cuda(np.zeros(n_pre + 1, np.int64))
    ix = cuda(np.zeros(1, np.int32))
    ev = wl.bernoulli_spikes(n_pre, 0.2, seed=10)
    sl, ns = spike_list_of(ev)
    y = torch.full((n_post,), 3, dtype=torch.int32, device="cuda")
    B.bp_event_csrmv(ip, ix, None, 1.0, sl, ns, y)
    assert torch.all(y == 3)
    x = torch.ones(n_post, dtype=torch.float32, device="cuda")
    tc = B.bp_tile_cols()
    tp = torch.empty(B.bp_csr_tile_index_size(n_pre, n_post, tc), dtype=torch.int32, device="cuda")
    B.bp_csr_tile_index(ip, ix, n_post, tc, tp)
    for kw in ({}, {"tile_ptr": tp, "tile_cols": tc}):
        yp = torch.full((n_pre,), 0.5, dtype=torch.float32, device="cuda")
        B.bp_event_csrmv_t(ip, ix, None, 1.0, x, yp, **kw)
        assert torch.all(yp == 0.5)


def test_lif_step_with_no_neurons():
    p = B.bp_coba_params_default()
    z = lambda dt: torch.zeros(0, dtype=dt, device="cuda")
    sl = torch.zeros(1, dtype=torch.int32, device="cuda")
    ns = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.bp_lif_step(p, 0, z(torch.float32), z(torch.float32), z(torch.float32), z(torch.uint8), z(torch.int32),
                  z(torch.int32), sl, ns)
    torch.cuda.synchronize()
    assert int(ns.item()) == 0


def test_full_size_operator_cell():
    """A graded operator cell at full size: n = 1e6, p = 0.001 (1e9 stored
    entries), rho = 0.1 (about 1e8 events), matrix = the JIT rows
    materialised.  The scatter's integer counts equal the oracle's over the
    whole output vector bit for bit (tiled shared-memory path, as timed: the
    equal tiles of bp_tile_cols_for, and full-width tiles with a short last
    one); FP32 and BF16 weights N(0.5, 0.1) with fixed-point tiles (as timed)
    stay within the fixed-point bound of the oracle's FP64 product; the tiled
    gather of a random x matches the oracle's sequential sum."""
    n, p, seed = 1_000_000, 0.001, 1000 + 1_000_000 % 997 + 10
    d = B.bp_jit_desc_init(seed, p)
    ip, ix, _ = B.jit_materialize(d, n, n)
    ev = wl.bernoulli_spikes(n, 0.1, seed=seed + 1000)
    sl, ns = spike_list_of(ev)
    h_ip, h_ix = ip.cpu().numpy(), ix.cpu().numpy()
    expect = orc.event_csr_count(h_ip, h_ix, ev, n)
    tiles = {}
    for tc in (B.bp_tile_cols_for(n), B.bp_tile_cols()):
        tp = torch.empty(B.bp_csr_tile_index_size(n, n, tc), dtype=torch.int32, device="cuda")
        B.bp_csr_tile_index(ip, ix, n, tc, tp)
        tiles[tc] = tp
        y = torch.zeros(n, dtype=torch.int32, device="cuda")
        B.bp_event_csrmv(ip, ix, None, 1.0, sl, ns, y, tile_ptr=tp, tile_cols=tc)
        assert np.array_equal(y.cpu().numpy(), expect.astype(np.int64)), tc
    tc = B.bp_tile_cols_for(n)
    rng = np.random.default_rng(12)
    w = (0.5 + 0.1 * rng.standard_normal(len(h_ix))).astype(np.float32)
    cnt = expect.astype(np.float64)
    for dw in (cuda(w), cuda(w).to(torch.bfloat16)):
        wref = dw.float().cpu().numpy().astype(np.float64)
        tp = tiles[tc].clone()
        B.bp_csr_tile_weight_bound(ip, ix, dw, 0.0, n, tc, tp)
        b = float(tp[-2:-1].cpu().numpy().view(np.float32)[0])
        y = torch.zeros(n, dtype=torch.float32, device="cuda")
        B.bp_event_csrmv(ip, ix, dw, 0.0, sl, ns, y, tile_ptr=tp, tile_cols=tc, flags=B.BP_ACC_FIXED)
        assert B.bp_sync_status() == 0
        ref = orc.event_csrmv(h_ip, h_ix, wref, ev, n)
        absc = orc.event_csrmv(h_ip, h_ix, np.abs(wref), ev, n)
        err = np.abs(y.cpu().numpy().astype(np.float64) - ref)
        assert np.all(err <= _fixed_bound(cnt, absc, int(ev.sum()), b)), str(dw.dtype)
        assert rel_err(y.cpu().numpy(), ref) < RTOL_F32
    x = np.random.default_rng(11).normal(size=n).astype(np.float32)
    yp = torch.zeros(n, dtype=torch.float32, device="cuda")
    B.bp_event_csrmv_t(ip, ix, None, 1.0, cuda(x), yp, tile_ptr=tiles[tc], tile_cols=tc)
    ref = orc.csrmv_t(h_ip, h_ix, None, x.astype(np.float64))
    assert rel_err(yp.cpu().numpy(), ref) < RTOL_F32


def test_csr_check_counts_defects():
    """bp_csr_check on a valid matrix reports nothing; planted defects (an
    index past n_post, a negative index, a descending row, a repeated column,
    an extent that runs past the buffer) are each counted, and rows with a bad
    extent are not read."""
    n_pre, n_post = 3000, 2000
    ip, ix = _csr(n_pre, n_post, 0.01, seed=51)
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    B.bp_csr_check(cuda(ip), cuda(ix), n_post, out)
    assert out.cpu().tolist() == [0, 0, 0, 0]
    lens = np.diff(ip)
    rows = [int(r) for r in np.nonzero(lens >= 3)[0][:4]]
    bad = ix.copy()
    bad[ip[rows[0] + 1] - 1] = n_post                                # out of range (last entry: still ascending)
    bad[ip[rows[1]] + 1] = -1                                        # negative (and descending)
    bad[ip[rows[2]]], bad[ip[rows[2]] + 1] = bad[ip[rows[2]] + 1], bad[ip[rows[2]]]   # descending
    bad[ip[rows[3]] + 1] = bad[ip[rows[3]]]                          # repeated column
    B.bp_csr_check(cuda(ip), cuda(bad), n_post, out)
    assert out.cpu().tolist() == [0, 2, 2, 1]
    bip = ip.copy()
    bip[n_pre] = len(ix) + 100                                       # last row runs past the buffer
    B.bp_csr_check(cuda(bip), cuda(ix), n_post, out)
    assert out.cpu().tolist()[0] == 2                                # its extent, and indptr[n_pre] != nnz


@pytest.mark.parametrize("case", [
    # n_pre, n_post, p, rho: very short rows (most (row, tile) segments empty),
    # dense rows (segments of a whole tile), and a single tile
    (20000, 200000, 0.00005, 0.5),
    (64, 120000, 1.0, 0.5),
    (3000, 40000, 0.05, 0.9),
])
def test_tiled_scatter_segment_shapes(case):
    """The tiled scatter lays each batch's (row, tile) segments end to end and
    streams them: counts equal the oracle's bit for bit whatever the segment
    lengths (empty, a whole tile, whole rows), and FP32 weights within 1e-5."""
    n_pre, n_post, p, rho = case
    ip, ix = _csr(n_pre, n_post, p, seed=n_pre + 3)
    ev = wl.bernoulli_spikes(n_pre, rho, seed=n_pre + 4)
    dip, dix = cuda(ip), cuda(ix)
    tc = B.bp_tile_cols() if n_post > B.bp_tile_cols() else 0
    tp = None
    if tc:
        tp = torch.empty(B.bp_csr_tile_index_size(n_pre, n_post, tc), dtype=torch.int32, device="cuda")
        B.bp_csr_tile_index(dip, dix, n_post, tc, tp)
    sl, ns = spike_list_of(ev)
    y = torch.zeros(n_post, dtype=torch.int32, device="cuda")
    B.bp_event_csrmv(dip, dix, None, 1.0, sl, ns, y, tile_ptr=tp, tile_cols=tc, flags=B.BP_ACC_SHARED)
    assert np.array_equal(y.cpu().numpy(), orc.event_csr_count(ip, ix, ev, n_post))
    w = wl.normal_weights(len(ix), 0.5, 0.1, seed=8)
    yf = torch.zeros(n_post, dtype=torch.float32, device="cuda")
    B.bp_event_csrmv(dip, dix, cuda(w), 0.0, sl, ns, yf, tile_ptr=tp, tile_cols=tc, flags=B.BP_ACC_SHARED)
    assert rel_err(yf.cpu().numpy(), orc.event_csrmv(ip, ix, w.astype(np.float64), ev, n_post)) < RTOL_F32


def test_tiled_scatter_repeated_columns():
    """Sorted rows with repeated columns (a column may be hit several times by
    one row): every repetition is an event, counted exactly."""
    n_pre, n_post = 4000, 130000
    rng = np.random.default_rng(12)
    lens = rng.integers(0, 300, n_pre)
    ip = np.zeros(n_pre + 1, np.int64)
    np.cumsum(lens, out=ip[1:])
    ix = np.concatenate([np.sort(rng.integers(0, n_post, int(k))) for k in lens]).astype(np.int32)
    ix = np.repeat(ix, 2)                     # every entry twice, rows still sorted
    ip = ip * 2
    ev = wl.bernoulli_spikes(n_pre, 0.4, seed=13)
    dip, dix = cuda(ip), cuda(ix)
    tc = B.bp_tile_cols()
    tp = torch.empty(B.bp_csr_tile_index_size(n_pre, n_post, tc), dtype=torch.int32, device="cuda")
    B.bp_csr_tile_index(dip, dix, n_post, tc, tp)
    sl, ns = spike_list_of(ev)
    y = torch.zeros(n_post, dtype=torch.int32, device="cuda")
    B.bp_event_csrmv(dip, dix, None, 1.0, sl, ns, y, tile_ptr=tp, tile_cols=tc, flags=B.BP_ACC_SHARED)
    assert np.array_equal(y.cpu().numpy(), orc.event_csr_count(ip, ix, ev, n_post))


def test_tiled_scatter_segments_beyond_the_flat_list():
    """Rows whose tile segments are far longer than a tile without repeated
    columns allows (1030 rows of 2.205e6 entries, every column of [0, 52 500)
    repeated 42 times, n_post = 9e6 so that each tile has a single CTA, 1009
    rows spiking): each warp's 32 segments exceed the flat list's limit, so
    they are walked segment by segment, and every column receives exactly 42
    events per spiking row, the other columns none (2.2e9 events in all)."""
    n_pre, n_post, per_row, rep = 1030, 9_000_000, 2_205_000, 42
    row = (torch.arange(per_row, dtype=torch.int64, device="cuda") // rep).to(torch.int32)
    ix = row.repeat(n_pre)
    ip = torch.arange(n_pre + 1, dtype=torch.int64, device="cuda") * per_row
    del row
    tc = B.bp_tile_cols()
    tp = torch.empty(B.bp_csr_tile_index_size(n_pre, n_post, tc), dtype=torch.int32, device="cuda")
    B.bp_csr_tile_index(ip, ix, n_post, tc, tp)
    ev = np.ones(n_pre, np.uint8)
    ev[::50] = 0
    sl, ns = spike_list_of(ev)
    y = torch.zeros(n_post, dtype=torch.int32, device="cuda")
    B.bp_event_csrmv(ip, ix, None, 1.0, sl, ns, y, tile_ptr=tp, tile_cols=tc, flags=B.BP_ACC_SHARED)
    torch.cuda.synchronize()
    k = int(ev.sum())
    assert k <= 1024 and k * per_row > 2**31
    cols = per_row // rep
    assert torch.all(y[:cols] == k * rep).item()
    assert int(y[cols:].abs().sum().item()) == 0
    del ix, tp
    torch.cuda.empty_cache()


def test_tiled_counts_accumulate_into_negative_outputs():
    """Integer counts added to an output that holds negative values (the
    tile flush adds column pairs as one 64-bit number only when the pair's
    first word is not negative): y0 + counts bit for bit, with odd n_post."""
    n_pre, n_post = 6000, 150001
    ip, ix = _csr(n_pre, n_post, 0.003, seed=71)
    ev = wl.bernoulli_spikes(n_pre, 0.3, seed=72)
    dip, dix = cuda(ip), cuda(ix)
    tc = B.bp_tile_cols()
    tp = torch.empty(B.bp_csr_tile_index_size(n_pre, n_post, tc), dtype=torch.int32, device="cuda")
    B.bp_csr_tile_index(dip, dix, n_post, tc, tp)
    sl, ns = spike_list_of(ev)
    y0 = np.random.default_rng(73).integers(-5, 6, n_post).astype(np.int32)
    y = torch.from_numpy(y0).cuda()
    B.bp_event_csrmv(dip, dix, None, 1.0, sl, ns, y, tile_ptr=tp, tile_cols=tc, flags=B.BP_ACC_SHARED)
    expect = y0.astype(np.int64) + orc.event_csr_count(ip, ix, ev, n_post)
    assert np.array_equal(y.cpu().numpy().astype(np.int64), expect)
    assert (y0 < 0).sum() > 10000


# ---------------------------------------------------------------------- fixed-point tile sums
def _tile_index(dip, dix, n_pre, n_post, tcols):
    tp = torch.empty(B.bp_csr_tile_index_size(n_pre, n_post, tcols), dtype=torch.int32, device="cuda")
    B.bp_csr_tile_index(dip, dix, n_post, tcols, tp)
    return tp


def _fixed_bound(counts_col, abs_col, n_spk, b):
    """Bound on |fixed-point result - exact| per column (bp_event_csrmv,
    BP_ACC_FIXED): each event off by at most 2^-(s+1) <= max(2 m b 2^-29,
    2^-127) with m at most the number of spiking rows, plus the FP32
    conversion of each CTA's tile and the FP32 adds into y (at most 152 of
    them per column), each rounding by 2^-24 of a partial sum no larger than
    the column's sum of absolute values."""
    per_event = max(2.0 * n_spk * b * 2.0 ** -29, 2.0 ** -127)
    return counts_col * per_event + abs_col * 2.0 ** -24 * 2 * 153 + 1e-300


@pytest.mark.parametrize("n_pre,n_post,p,rho,tcols", [(300, 257, 0.1, 0.3, 64), (5000, 40001, 0.02, 0.05, 4096),
                                                      (2000, 150001, 0.004, 0.2, 54944), (1, 1, 1.0, 1.0, 32)])
@pytest.mark.parametrize("wdt", ["f32", "bf16"])
def test_fixed_point_tiles_within_their_bound(n_pre, n_post, p, rho, tcols, wdt):
    """BP_ACC_FIXED against the oracle's FP64 product, with weights of both
    signs over four decades, within the bound the fixed-point arithmetic
    gives (bp.h); the recorded weight bound is the largest |w| (rows have no
    repeated column here), rounded up."""
    ip, ix = _csr(n_pre, n_post, p, seed=n_pre + 31)
    rng = np.random.default_rng(n_pre)
    w = (rng.choice([-1.0, 1.0], size=len(ix)) * 10.0 ** rng.uniform(-3, 1, size=len(ix))).astype(np.float32)
    ev = wl.bernoulli_spikes(n_pre, rho, seed=n_pre + 5)
    dip, dix = cuda(ip), cuda(ix)
    tp = _tile_index(dip, dix, n_pre, n_post, tcols)
    dw = cuda(w) if wdt == "f32" else cuda(w).to(torch.bfloat16)
    wref = dw.float().cpu().numpy().astype(np.float64)
    B.bp_csr_tile_weight_bound(dip, dix, dw, 0.0, n_post, tcols, tp)
    b = float(tp[-2:-1].cpu().numpy().view(np.float32)[0])
    amax = float(np.abs(wref).max()) if len(wref) else 0.0
    assert amax <= b <= amax * (1 + 2.0 ** -15) or (amax == 0.0 and b > 0.0)
    sl, ns = spike_list_of(ev)
    y = torch.zeros(n_post, dtype=torch.float32, device="cuda")
    B.bp_event_csrmv(dip, dix, dw, 0.0, sl, ns, y, tile_ptr=tp, tile_cols=tcols,
                     flags=B.BP_ACC_SHARED | B.BP_ACC_FIXED)
    assert B.bp_sync_status() == 0
    ref = orc.event_csrmv(ip, ix, wref, ev, n_post)
    cnt = orc.event_csr_count(ip, ix, ev, n_post).astype(np.float64)
    absc = orc.event_csrmv(ip, ix, np.abs(wref), ev, n_post)
    err = np.abs(y.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= _fixed_bound(cnt, absc, int(ev.sum()), b))
    # and typically as close as an FP32 sum
    if ref.size and np.abs(ref).max() > 0:
        assert rel_err(y.cpu().numpy(), ref) < RTOL_F32


def test_fixed_point_tiles_do_not_depend_on_event_order():
    """With one CTA per tile (as many tiles as SMs, n_post above the one-tile
    size) every column's sum is one CTA's integer tile sum: any order of the
    spike list gives the same result bit for bit."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cap = B.bp_tile_cols()  # at or below this n_post one tile covers y and the index is not used
    tcols = 32 * (-(-(cap + 1) // (32 * sms)))
    n_post = sms * tcols
    assert n_post > cap
    n_pre = 3000
    ip, ix = _csr(n_pre, n_post, 0.02, seed=77)
    w = wl.normal_weights(len(ix), 0.5, 0.3, seed=78)
    ev = wl.bernoulli_spikes(n_pre, 0.3, seed=79)
    dip, dix, dw = cuda(ip), cuda(ix), cuda(w)
    tp = _tile_index(dip, dix, n_pre, n_post, tcols)
    B.bp_csr_tile_weight_bound(dip, dix, dw, 0.0, n_post, tcols, tp)
    ids = np.nonzero(ev)[0].astype(np.int32)
    outs = []
    for perm in (ids, ids[::-1], np.random.default_rng(1).permutation(ids)):
        sl = torch.zeros(n_pre, dtype=torch.int32, device="cuda")
        sl[: len(perm)] = cuda(perm.astype(np.int32))
        ns = torch.tensor([len(perm)], dtype=torch.int32, device="cuda")
        y = torch.zeros(n_post, dtype=torch.float32, device="cuda")
        B.bp_event_csrmv(dip, dix, dw, 0.0, sl, ns, y, tile_ptr=tp, tile_cols=tcols,
                         flags=B.BP_ACC_SHARED | B.BP_ACC_FIXED)
        outs.append(y.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    assert rel_err(outs[0], orc.event_csrmv(ip, ix, w.astype(np.float64), ev, n_post)) < RTOL_F32


def test_weight_bound_sums_repeated_columns():
    """A row that repeats a column contributes the sum of those entries: the
    bound is the largest such per-row, per-column absolute sum."""
    ip = np.array([0, 3, 5], np.int64)
    ix = np.array([2, 2, 7, 1, 1], np.int32)
    w = np.array([0.5, -0.75, 0.25, 1.0, 0.125], np.float32)
    tcols = 32
    dip, dix, dw = cuda(ip), cuda(ix), cuda(w)
    tp = _tile_index(dip, dix, 2, 40, tcols)
    assert int(tp[-1].item()) == 0 and int(tp[-2].item()) == 0  # no bound yet
    B.bp_csr_tile_weight_bound(dip, dix, dw, 0.0, 40, tcols, tp)
    b = float(tp[-2:-1].cpu().numpy().view(np.float32)[0])
    assert 1.25 <= b <= 1.25 * (1 + 2.0 ** -15)
    assert int(tp[-1].item()) == 1  # no column holds entries of both rows
    B.bp_csr_tile_weight_bound(dip, dix, None, -3.0, 40, tcols, tp)  # homogeneous: |w| times the longest run
    b = float(tp[-2:-1].cpu().numpy().view(np.float32)[0])
    assert 6.0 <= b <= 6.0 * (1 + 2.0 ** -15)


@pytest.mark.parametrize("n_pre,n_post,p", [(3000, 700, 0.05), (50, 100000, 0.2), (1, 5, 1.0)])
def test_column_bound_counts_rows_per_column(n_pre, n_post, p):
    """The second bound slot holds the largest number of rows with an entry
    in one column (a row that repeats a column counts once; indices outside
    [0, n_post) are not counted), against a brute-force count."""
    ip, ix = _csr(n_pre, n_post, p, seed=n_pre + 77)
    ix = ix.copy()
    lens = np.diff(ip)
    rows = np.nonzero(lens >= 2)[0]
    if len(rows):
        r = int(rows[0])
        ix[ip[r] + 1] = ix[ip[r]]  # a repeated column (rows stay sorted)
    dip, dix = cuda(ip), cuda(ix)
    tcols = 32 * max(1, min(B.bp_tile_cols() // 32, (n_post + 31) // 32))
    tp = _tile_index(dip, dix, n_pre, n_post, tcols)
    B.bp_csr_tile_weight_bound(dip, dix, None, 1.0, n_post, tcols, tp)
    per_col = np.zeros(n_post, np.int64)
    for i in range(n_pre):
        per_col[np.unique(ix[ip[i]:ip[i + 1]])] += 1
    assert int(tp[-1].item()) == int(per_col.max())


def test_fixed_point_without_a_bound_is_reported():
    """BP_ACC_FIXED on a tile index whose bound was never recorded: the kernel
    adds nothing and records BP_ERR_DEVICE; without any tile index the call
    is rejected on the host."""
    n_pre, n_post, tcols = 500, 4000, 1024
    ip, ix = _csr(n_pre, n_post, 0.05, seed=3)
    dip, dix = cuda(ip), cuda(ix)
    dw = cuda(wl.normal_weights(len(ix), 0.5, 0.1, seed=4))
    tp = _tile_index(dip, dix, n_pre, n_post, tcols)
    sl, ns = spike_list_of(wl.bernoulli_spikes(n_pre, 0.5, seed=5))
    y = torch.zeros(n_post, dtype=torch.float32, device="cuda")
    B.bp_event_csrmv(dip, dix, dw, 0.0, sl, ns, y, tile_ptr=tp, tile_cols=tcols,
                     flags=B.BP_ACC_SHARED | B.BP_ACC_FIXED)
    assert B.bp_sync_status() == B.BP_ERR_DEVICE
    assert B.bp_sync_status() == 0  # the status word was cleared
    assert torch.count_nonzero(y).item() == 0
    with pytest.raises(B.BpError):
        B.bp_event_csrmv(dip, dix, dw, 0.0, sl, ns, y, flags=B.BP_ACC_SHARED | B.BP_ACC_FIXED)


@pytest.mark.parametrize("off", [0, 1, 2, 4, 8])
@pytest.mark.parametrize("wdt", [None, torch.float32, torch.bfloat16])
def test_tiled_scatter_operand_alignments(off, wdt):
    """The tiled walk picks its unit by the operands' alignment (8 entries for
    32-byte aligned BF16 weights, 4 for 16-byte aligned operands, single
    entries otherwise): index and weight buffers offset by `off` elements
    reach every unit size, each against the oracle (counts exactly), with FP32
    atomics and with fixed-point tile sums."""
    n_pre, n_post, tc = 3000, 150001, B.bp_tile_cols()
    ip, ix = _csr(n_pre, n_post, 0.004, seed=41)
    ev = wl.bernoulli_spikes(n_pre, 0.2, seed=42)
    nnz = len(ix)
    ixb = torch.zeros(nnz + 16, dtype=torch.int32, device="cuda")
    ixb[off:off + nnz] = cuda(ix)
    dix = ixb[off:off + nnz]
    dip = cuda(ip)
    tp = torch.empty(B.bp_csr_tile_index_size(n_pre, n_post, tc), dtype=torch.int32, device="cuda")
    B.bp_csr_tile_index(dip, dix, n_post, tc, tp)
    sl, ns = spike_list_of(ev)
    if wdt is None:
        y = torch.zeros(n_post, dtype=torch.int32, device="cuda")
        B.bp_event_csrmv(dip, dix, None, 1.0, sl, ns, y, tile_ptr=tp, tile_cols=tc, flags=B.BP_ACC_SHARED)
        assert np.array_equal(y.cpu().numpy(), orc.event_csr_count(ip, ix, ev, n_post))
        return
    w = wl.normal_weights(nnz, 0.5, 0.1, seed=43)
    wb = torch.zeros(nnz + 16, dtype=wdt, device="cuda")
    wb[off:off + nnz] = cuda(w).to(wdt)
    dw = wb[off:off + nnz]
    ref = orc.event_csrmv(ip, ix, dw.float().cpu().numpy().astype(np.float64), ev, n_post)
    B.bp_csr_tile_weight_bound(dip, dix, dw, 0.0, n_post, tc, tp)
    for fl in (B.BP_ACC_SHARED, B.BP_ACC_SHARED | B.BP_ACC_FIXED):
        y = torch.zeros(n_post, dtype=torch.float32, device="cuda")
        B.bp_event_csrmv(dip, dix, dw, 0.0, sl, ns, y, tile_ptr=tp, tile_cols=tc, flags=fl)
        assert B.bp_sync_status() == 0
        assert rel_err(y.cpu().numpy(), ref) < RTOL_F32


@pytest.mark.parametrize("scale", [1e-30, 1e30])
def test_fixed_point_tiles_extreme_weight_magnitudes(scale):
    """Weight bounds near the ends of the FP32 range: the fixed-point scale is
    taken from the exponents of m and b separately (m b may overflow FP32)
    and stays a normal float, and the result keeps the bound of the
    arithmetic against the oracle."""
    n_pre, n_post, tc = 2000, 60001, 4096
    ip, ix = _csr(n_pre, n_post, 0.01, seed=51)
    rng = np.random.default_rng(52)
    w = (rng.choice([-1.0, 1.0], size=len(ix)) * rng.uniform(0.1, 1.0, size=len(ix)) * scale).astype(np.float32)
    ev = wl.bernoulli_spikes(n_pre, 0.3, seed=53)
    dip, dix, dw = cuda(ip), cuda(ix), cuda(w)
    tp = _tile_index(dip, dix, n_pre, n_post, tc)
    B.bp_csr_tile_weight_bound(dip, dix, dw, 0.0, n_post, tc, tp)
    b = float(tp[-2:-1].cpu().numpy().view(np.float32)[0])
    sl, ns = spike_list_of(ev)
    y = torch.zeros(n_post, dtype=torch.float32, device="cuda")
    B.bp_event_csrmv(dip, dix, dw, 0.0, sl, ns, y, tile_ptr=tp, tile_cols=tc, flags=B.BP_ACC_SHARED | B.BP_ACC_FIXED)
    assert B.bp_sync_status() == 0
    wref = w.astype(np.float64)
    ref = orc.event_csrmv(ip, ix, wref, ev, n_post)
    cnt = orc.event_csr_count(ip, ix, ev, n_post).astype(np.float64)
    absc = orc.event_csrmv(ip, ix, np.abs(wref), ev, n_post)
    got = y.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= _fixed_bound(cnt, absc, int(ev.sum()), b))
    assert rel_err(got, ref) < RTOL_F32



def test_binding_launches_on_the_current_stream():
    """The binding's default stream is torch's current stream (raw handle),
    on the device's default stream and inside a side-stream context; a
    kernel enqueued there is ordered after earlier work on that stream."""
    assert (B._stream(None).value or 0) == torch.cuda.current_stream().cuda_stream
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert B._stream(None).value == s.cuda_stream
        n = 1000
        events = torch.zeros(n, dtype=torch.uint8, device="cuda")
        events[::3] = 1
        sl = torch.zeros(n, dtype=torch.int32, device="cuda")
        ns = torch.zeros(1, dtype=torch.int32, device="cuda")
        B.bp_spike_compact(events, sl, ns)
    s.synchronize()
    assert int(ns.item()) == (n + 2) // 3
