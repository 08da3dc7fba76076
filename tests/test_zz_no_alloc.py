"""bp_event_csrmv_dense_noalloc: the dense-event CSR product for callers that
cannot allocate device memory (a framework owning the device memory pool, a
real-time loop that must not risk an allocation's device synchronisation).

It must return what bp_event_csrmv_dense (caller-owned workspace) returns, on
consecutive calls that reuse its fixed scratch, and reject inputs larger than
that scratch.  This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2311_05106_gb300 import binding as B
from paper_2311_05106_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _inputs(n_pre, n_post, p, rho, seed):
    ip, ix = wl.random_csr(n_pre, n_post, p, seed)
    w = wl.normal_weights(len(ix), 0.5, 0.1, seed + 1)
    ev = wl.bernoulli_spikes(n_pre, rho, seed + 2)
    return (torch.from_numpy(ip).cuda(), torch.from_numpy(ix).cuda(), torch.from_numpy(w).cuda(),
            torch.from_numpy(ev).cuda())


def _reference(ip, ix, w, ev, n_post, counts):
    ws = torch.zeros(B.bp_event_csrmv_dense_workspace_bytes(ip.numel() - 1), dtype=torch.uint8, device="cuda")
    y = torch.zeros(n_post, dtype=torch.int32 if counts else torch.float32, device="cuda")
    B.bp_event_csrmv_dense(ip, ix, None if counts else w, 1.0, ev, ws, y)
    return y


def test_noalloc_matches_workspace_version_on_consecutive_calls():
    cases = [(6000, 5000, 0.01, 0.2, 11), (9000, 7000, 0.005, 0.05, 12)]
    for counts in (True, False):
        for n_pre, n_post, p, rho, seed in cases:   # two calls in a row share the scratch
            ip, ix, w, ev = _inputs(n_pre, n_post, p, rho, seed)
            ref = _reference(ip, ix, w, ev, n_post, counts)
            y = torch.zeros(n_post, dtype=torch.int32 if counts else torch.float32, device="cuda")
            B.bp_event_csrmv_dense_noalloc(ip, ix, None if counts else w, 1.0, ev, y)
            torch.cuda.synchronize()
            if counts:
                assert torch.equal(y, ref)
            else:
                err = (y - ref).abs().max().item() / max(ref.abs().max().item(), 1e-30)
                assert err < 1e-5


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
