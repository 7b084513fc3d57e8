"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank
evaluates its own walkers against the same environment (no collective on the
data path); the step time is the maximum over ranks.  Each rank builds the
environment with the library's host-only builder and evaluates its walkers
with the kernels' own per-tile code run on the host (esp_debug_host_eval),
and the per-rank results equal a single-process evaluation of the same
walkers."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402

N_POS = 64


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _environment():
    from workloads import realistic_environment
    return realistic_environment(seed=5151, n_atoms=30, n_walkers=2, n_elec=32)


def _host_eval(wl, pos, precision):
    from paper_1011_4687_gb300 import build_lib, esp
    build_lib.build()
    with esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision=precision,
                         flags=esp.FLAG_HOST_ONLY) as env:
        return env.debug_host_eval(pos)


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = _environment()
        pos = bench.replica_positions(rank, N_POS, "realistic") if rank > 0 else wl.positions[:N_POS]
        V = _host_eval(wl, pos, "fp32c")
        ms = bench.max_over_ranks(10.0 + rank, world, "cpu")
        np.save(os.path.join(out_dir, "r%d.npy" % rank), np.concatenate([pos.ravel(), V, [ms]]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_gloo(tmp_path):
    world = 2
    from paper_1011_4687_gb300 import build_lib
    build_lib.build()  # once, before the ranks start
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / ("r%d.npy" % k)) for k in range(world)]
    # the slowest rank's time on every rank
    assert r[0][-1] == 11.0 and r[1][-1] == 11.0
    # rank 1's walkers: the workload's law (inside the QM sphere), its own seed
    p1 = r[1][:3 * N_POS].reshape(N_POS, 3)
    assert np.all(np.linalg.norm(p1, axis=1) < 6.0)
    assert not np.array_equal(p1, bench.replica_positions(2, N_POS, "realistic"))
    assert np.array_equal(p1, bench.replica_positions(1, N_POS, "realistic"))
    # each rank's potentials equal a single-process evaluation of its walkers
    wl = _environment()
    for k in range(world):
        pos = r[k][:3 * N_POS].reshape(N_POS, 3)
        V = r[k][3 * N_POS:3 * N_POS + N_POS]
        assert np.array_equal(V, _host_eval(wl, pos, "fp32c"))
