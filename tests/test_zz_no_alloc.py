"""bp_event_csrmv_dense_noalloc: the dense-event CSR product for callers that
cannot allocate device memory (a framework owning the device memory pool, a
real-time loop that must not risk an allocation's device synchronisation).

On two consecutive calls that reuse its fixed scratch it must return what
bp_event_csrmv_dense (caller-owned workspace) returns under the same flags,
and what the FP64 oracle's event product (Appendix B) gives: integer counts
bit for bit, FP32 / BF16 weights within 1e-5 relative (BF16: the oracle is fed
the same BF16-rounded weights).  It must reject inputs larger than its
scratch.  This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc
from paper_2311_05106_gb300 import binding as B
from paper_2311_05106_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FLAGS = {"accumulate": 0, "overwrite": B.BP_OVERWRITE, "acc_global": B.BP_ACC_GLOBAL,
         "acc_shared": B.BP_ACC_SHARED}


def _inputs(n_pre, n_post, p, rho, seed, kind):
    ip, ix = wl.random_csr(n_pre, n_post, p, seed)
    w = wl.normal_weights(len(ix), 0.5, 0.1, seed + 1)
    ev = wl.bernoulli_spikes(n_pre, rho, seed + 2)
    wt = None
    w64 = None
    if kind == "f32":
        wt = torch.from_numpy(w).cuda()
        w64 = w.astype(np.float64)
    elif kind == "bf16":
        wb = torch.from_numpy(w).to(torch.bfloat16)
        wt = wb.cuda()
        w64 = wb.to(torch.float64).numpy()
    return (torch.from_numpy(ip).cuda(), torch.from_numpy(ix).cuda(), wt, torch.from_numpy(ev).cuda()), \
        (ip, ix, w64, ev)


def _y0(n_post, counts, seed):
    """A non-zero starting output, so that accumulation and overwriting differ."""
    rng = np.random.default_rng(seed)
    if counts:
        return rng.integers(0, 5, n_post).astype(np.int32)
    return rng.normal(0.0, 1.0, n_post).astype(np.float32)


@pytest.mark.parametrize("flag", list(FLAGS))
@pytest.mark.parametrize("kind", ["counts", "f32", "bf16"])
def test_noalloc_matches_oracle_and_workspace_version(kind, flag):
    counts = kind == "counts"
    fl = FLAGS[flag]
    cases = [(6000, 5000, 0.01, 0.2, 11), (9000, 7000, 0.005, 0.05, 12)]
    for n_pre, n_post, p, rho, seed in cases:   # two calls in a row share the scratch
        (ip, ix, w, ev), (hip, hix, hw, hev) = _inputs(n_pre, n_post, p, rho, seed, kind)
        y0 = _y0(n_post, counts, seed + 3)
        if counts:
            prod = orc.event_csr_count(hip, hix, hev, n_post)
        else:
            prod = orc.event_csrmv(hip, hix, hw, hev, n_post)
        expect = prod if fl & B.BP_OVERWRITE else y0.astype(prod.dtype) + prod
        ws = torch.zeros(B.bp_event_csrmv_dense_workspace_bytes(n_pre), dtype=torch.uint8, device="cuda")
        ref = torch.from_numpy(y0).cuda()
        B.bp_event_csrmv_dense(ip, ix, w, 1.0, ev, ws, ref, flags=fl)
        y = torch.from_numpy(y0).cuda()
        B.bp_event_csrmv_dense_noalloc(ip, ix, w, 1.0, ev, y, flags=fl)
        torch.cuda.synchronize()
        got, got_ref = y.cpu().numpy(), ref.cpu().numpy()
        if counts:
            assert np.array_equal(got, expect.astype(np.int64))
            assert np.array_equal(got, got_ref)
        else:
            scale = max(np.abs(expect).max(), 1e-30)
            assert np.max(np.abs(got - expect)) / scale < 1e-5
            assert np.max(np.abs(got - got_ref)) / scale < 1e-5
        assert int(prod.sum()) != 0
    assert B.bp_sync_status() == 0


def test_noalloc_rejects_inputs_beyond_its_scratch():
    m = B.bp_event_csrmv_dense_noalloc_max_pre()
    assert m == 1 << 20
    ip = torch.zeros(m + 2, dtype=torch.int64, device="cuda")
    ix = torch.zeros(1, dtype=torch.int32, device="cuda")
    ev = torch.zeros(m + 1, dtype=torch.uint8, device="cuda")
    y = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(B.BpError) as e:
        B.bp_event_csrmv_dense_noalloc(ip, ix, None, 1.0, ev, y)
    assert "exceeds the fixed scratch" in str(e.value)
    assert B.bp_sync_status() == 0
