"""Multi-GPU runs are independent replicas (one process per GPU, own
operators, own ruptures, no collective on the data path); the host logic of
bench.py that joins them (distinct ruptures per rank, max-over-ranks time,
whole-job rate) runs here as world_size-2 gloo ranks on the CPU."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    pool = np.arange(8 * 3, dtype=np.float32).reshape(8, 3)
    mine = bench.replica_ruptures(pool, rank)
    firsts = [torch.zeros(1) for _ in range(world)]
    dist.all_gather(firsts, torch.tensor([float(mine[0, 0])]))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, [float(f.item()) for f in firsts], mine.tolist()))


def test_two_replicas_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, f0, m0), (r1, t1, f1, m1) = res
    assert t0 == t1 == 15.0                      # the slowest rank's time, on every rank
    assert f0 == f1 and f0[0] != f0[1]           # each replica starts on its own rupture
    assert sorted(map(tuple, m0)) == sorted(map(tuple, m1))  # same pool, rotated


def test_single_rank_and_job_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    pool = np.arange(6).reshape(6, 1)
    assert np.array_equal(bench.replica_ruptures(pool, 0), pool)
    # two replicas of 256 ruptures per step over 10 steps in 2 s (slowest rank)
    assert bench.job_rate(2, 256 * 10, 2.0) == 2560.0


def test_tensor_dtype_names_the_mma_type():
    """The bench line's dtype is the stage-1 MMA arithmetic: FP8 operators run
    two e4m3 x e4m3 MMAs per product (hi + lo activations, the default), one
    (e4m3 activations), or FP16 MMAs (operator widened)."""
    import argparse
    sys.path.insert(0, ROOT)
    import bench
    ns = argparse.Namespace
    assert bench.tensor_dtype(ns(prec_g="bf16", fp8_act="hilo")) == "bf16"
    assert bench.tensor_dtype(ns(prec_g="bf16_hilo", fp8_act="hilo")) == "bf16x3"
    assert bench.tensor_dtype(ns(prec_g="fp8", fp8_act="hilo")) == "e4m3x2"
    assert bench.tensor_dtype(ns(prec_g="fp8", fp8_act="e4m3")) == "e4m3"
    assert bench.tensor_dtype(ns(prec_g="fp8", fp8_act="f16")) == "f16"
