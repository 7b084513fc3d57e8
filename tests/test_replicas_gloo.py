"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank
evaluates its own walkers against the same environment (no collective on the
data path); the step time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pos = bench.replica_positions(rank, 64) if rank > 0 else np.zeros((64, 3))
        ms = bench.max_over_ranks(10.0 + rank, world, "cpu")
        np.save(os.path.join(out_dir, "r%d.npy" % rank), np.concatenate([pos.ravel(), [ms]]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_gloo(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    # the slowest rank's time on every rank
    assert r0[-1] == 11.0 and r1[-1] == 11.0
    # rank 1's walkers: the workload's law (inside the QM sphere), its own seed
    p1 = r1[:-1].reshape(64, 3)
    assert np.all(np.linalg.norm(p1, axis=1) < 6.0)
    assert not np.array_equal(p1, bench.replica_positions(2, 64))
    assert np.array_equal(p1, bench.replica_positions(1, 64))
