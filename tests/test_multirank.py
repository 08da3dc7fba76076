"""The multi-rank path of the benchmark on CPU (gloo, world size 2): every rank
runs its own replica (no data-path collective); the job's time is the slowest
rank's and its events are the sum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank          # rank 1 is the slower replica
    events = 1000 * (rank + 1)
    dist.barrier()
    got = bench.aggregate_ranks(torch, dist, ms, events, "cpu")
    out[rank] = got
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()   # no fork of this (threaded) process
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (15.0, 3000)


def test_failed_variant_child_is_reported():
    """A network variant whose child process fails (here: an unknown variant,
    rejected by the child's own argument handling) raises in the parent with
    the child's error text, which the bench records in that variant's entry
    instead of ending the run."""
    import argparse
    import importlib
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    bench = importlib.import_module("bench")
    args = argparse.Namespace(steps=1, warmup=0, settle=0)
    with pytest.raises(RuntimeError, match="variant no_such_variant failed"):
        bench.network_variant("no_such_variant", args, 0)
