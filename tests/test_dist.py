"""The multi-rank path of the bench on CPU: two gloo ranks launched like
torchrun's workers (RANK / WORLD_SIZE / MASTER_* in the environment, rendezvous
on 127.0.0.1).  Replicas carry no data-path collective: the only exchanges
are the barrier and the max of the per-rank step time, and the job's
throughput is the sum of every rank's pixels over that slowest time.  Only
rank 0 runs the reference arm."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import argparse

    import torch.distributed as dist

    import bench
    args = argparse.Namespace(impl="reference")  # gloo process group (the reference arm's backend)
    w, r, _ = bench.dist_setup(args)
    assert (w, r) == (world, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    ms_max, value = bench.aggregate(1_000_000, ms, w)
    # only rank 0 runs the reference arm; the others return at once
    rc = bench.run_reference(argparse.Namespace(), w, r) if r != 0 else 0
    bench.barrier(w)
    dist.destroy_process_group()
    out[rank] = (ms_max, value, rc)


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_aggregate_and_barrier(world):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    for p in procs:
        if p.is_alive():
            p.kill()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    for r in range(world):
        ms_max, value, rc = out[r]
        assert ms_max == 15.0
        assert abs(value - world * 1_000_000 / 0.015 / 1e6) < 1e-9
        assert rc == 0
