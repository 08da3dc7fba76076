"""Parity of the tensor-core spike-driven weight gradient (bp_spike_outer:
out[m][n] += sum_k [x_km != 0] delta_kn, Section 3.1's reverse-mode rule of an
event-driven dense product) against the oracle's FP64 definition.

* Values on a 2^-8 grid below 17 in magnitude need both BF16 terms
  (hi = bf16(delta), lo = bf16(delta - hi)) and give sums that FP32 holds
  exactly, so the result must equal the oracle BIT FOR BIT: any error in the
  operand layout, the swizzle, the tiling or the split reduction fails here.
* Normal deltas: within the bound of the arithmetic,
  |err| <= S (2^-16 + (K / 16 + 16 + splits) 2^-23),  S = sum_k |x_km delta_kn|
  (2^-17 for the dropped third BF16 term of each product, rounded up; one FP32
  rounding, taken as truncation (2^-23), per accumulation into the tensor
  memory accumulator: K / 16 MMAs, up to 16 products inside one, and the sum
  over at most 16 K splits).
* Shapes span several tiles with ragged edges in K (64 per block), M (256 per
  tile) and N (128 per tile).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc
from paper_2311_05106_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _spikes(rng, K, M, rate):
    x = (rng.random((K, M)) < rate).astype(np.uint8)
    x *= rng.integers(1, 256, size=(K, M)).astype(np.uint8)  # any non-zero byte is a spike
    return x


def _grid_values(rng, K, N):
    return rng.integers(-16, 17, size=(K, N)) + rng.integers(0, 256, size=(K, N)) / 256.0


def _run(x, d, out=None, overwrite=True):
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    dt = torch.from_numpy(np.ascontiguousarray(d, np.float32)).cuda()
    if out is None:
        out = torch.zeros(x.shape[1], d.shape[1], dtype=torch.float32, device="cuda")
    B.bp_spike_outer(xt, dt, out, overwrite=overwrite)
    assert B.bp_sync_status() == 0
    return out


@pytest.mark.parametrize("K,M,N", [(1000, 300, 200), (64, 256, 128), (1, 1, 1), (130, 513, 129),
                                   (2999, 40, 1030)])
def test_grid_values_bit_exact(K, M, N):
    rng = np.random.default_rng(K * 7 + M)
    x = _spikes(rng, K, M, 0.3)
    d = _grid_values(rng, K, N)
    got = _run(x, d).cpu().numpy().astype(np.float64)
    want = orc.spike_outer(x, d.astype(np.float32))
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("K,M,N,rate", [(5000, 700, 1024, 0.05), (777, 300, 260, 0.5)])
def test_normal_deltas_within_the_arithmetic_bound(K, M, N, rate):
    rng = np.random.default_rng(K + N)
    x = _spikes(rng, K, M, rate)
    d = rng.standard_normal((K, N)).astype(np.float32) * np.exp(rng.uniform(-8, 2, size=(K, 1))).astype(np.float32)
    got = _run(x, d).cpu().numpy().astype(np.float64)
    want = orc.spike_outer(x, d)
    S = orc.spike_outer(x, np.abs(d.astype(np.float64)))
    bound = S * (2.0 ** -16 + (K / 16 + 16 + 16) * 2.0 ** -23) + 1e-30
    err = np.abs(got - want)
    assert np.all(err <= bound), float((err / np.maximum(S, 1e-30)).max())
    # and typically far inside it
    assert float(np.median(err / np.maximum(S, 1e-30))) < 1e-5


def test_accumulates_unless_overwrite_and_is_reproducible():
    rng = np.random.default_rng(5)
    K, M, N = 700, 300, 200
    x = _spikes(rng, K, M, 0.2)
    d = rng.standard_normal((K, N)).astype(np.float32)
    base = torch.full((M, N), 1.5, dtype=torch.float32, device="cuda")
    g = _run(x, d)
    acc = _run(x, d, out=base.clone(), overwrite=False)
    torch.testing.assert_close(acc, g + 1.5, rtol=0, atol=1e-5)
    again = _run(x, d)
    assert torch.equal(g, again)


def test_empty_sizes():
    out = torch.full((3, 4), 2.0, dtype=torch.float32, device="cuda")
    x = torch.zeros((0, 3), dtype=torch.uint8, device="cuda")
    d = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
    B.bp_spike_outer(x, d, out, overwrite=False, work=torch.zeros(0, dtype=torch.uint8, device="cuda"))
    assert torch.all(out == 2.0)
    B.bp_spike_outer(x, d, out, overwrite=True, work=torch.zeros(0, dtype=torch.uint8, device="cuda"))
    assert torch.all(out == 0.0)


def test_bptt_sized_contraction_sampled_rows():
    """K = B T = 128 x 100, M = 700 inputs + 1024 recurrent spike rows,
    N = 1024 (the differentiable network's weight gradients); 48 sampled rows
    m compared with the oracle."""
    rng = np.random.default_rng(11)
    K, M, N = 12800, 1724, 1024
    x = _spikes(rng, K, M, 0.04)
    d = (rng.standard_normal((K, N)) * 1e-3).astype(np.float32)
    got = _run(x, d).cpu().numpy().astype(np.float64)
    rows = np.sort(rng.choice(M, size=48, replace=False))
    want = orc.spike_outer(x[:, rows], d)
    S = orc.spike_outer(x[:, rows], np.abs(d.astype(np.float64)))
    bound = S * (2.0 ** -16 + (K / 16 + 32) * 2.0 ** -23) + 1e-30
    assert np.all(np.abs(got[rows] - want) <= bound)


def test_workspace_too_small_is_rejected():
    x = torch.zeros((100, 10), dtype=torch.uint8, device="cuda")
    d = torch.zeros((100, 20), dtype=torch.float32, device="cuda")
    out = torch.zeros((10, 20), dtype=torch.float32, device="cuda")
    small = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.BpError):
        B.bp_spike_outer(x, d, out, work=small)
