"""The measurement kernels that give the roofline denominators do the work
they claim: the Philox-only kernel draws the blocks the oracle's Philox4x32-10
gives (so its rate counts real draws), the scattered-reduction kernel lands
exactly threads x per_thread additions inside y, and the copy kernel copies."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc
from paper_2311_05106_gb300 import binding as B

pytestmark = pytest.mark.gpu


def test_philox_roof_draws_the_oracle_blocks():
    threads = B.bp_roof_philox_threads()
    sink = torch.zeros(threads, dtype=torch.int32, device="cuda")
    seed = 0x1234_5678_9ABC_DEF0
    blocks = 3
    B.bp_roof_philox(blocks, sink, seed=seed)
    got = sink.cpu().numpy().view(np.uint32)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    for tid in (0, 1, 255, 256, threads - 1):
        acc = np.uint32(0)
        for b in range(blocks):
            x = orc.philox4x32_10(np.array([b, tid, 0, 0], np.uint32), key)
            acc ^= x[0] ^ x[1] ^ x[2] ^ x[3]
        assert got[tid] == acc, tid


def test_l2_red_roof_adds_exactly_its_count():
    y = torch.zeros(1_000_000, dtype=torch.int32, device="cuda")
    per = 7
    B.bp_roof_l2_red(y, per)
    t = y.to(torch.int64)
    assert int(t.sum().item()) == B.bp_roof_l2_red_threads() * per
    assert int((t > 0).sum().item()) > 500_000      # spread over the array


def test_copy_roof_copies():
    src = torch.arange(1 << 20, dtype=torch.float32, device="cuda")
    dst = torch.zeros_like(src)
    B.bp_roof_copy(src, dst, 3)
    assert torch.equal(src, dst)
