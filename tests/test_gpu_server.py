"""Several host threads sharing one context through the server (the paper's
proposal of several processes / OpenMP threads sharing one GPU): every
client's potentials equal a single-client evaluation of its positions, and
agree with the FP64 oracle; a client overlaps host work with its request."""
import threading

import numpy as np
import pytest

import oracle
from paper_1011_4687_gb300 import build_lib, esp
from workloads import qm_positions, realistic_environment

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env_wl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build_lib.build()
    wl = realistic_environment(seed=7722, n_atoms=150, n_walkers=4, n_elec=32)
    env = esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision="fp32c")
    yield env, wl
    env.close()


def test_clients_get_their_own_results(env_wl):
    env, wl = env_wl
    n_clients, reqs = 4, 3
    rng = np.random.default_rng(5)
    pos = [[qm_positions(rng, int(rng.integers(1, 700))) for _ in range(reqs)] for _ in range(n_clients)]
    single = [[env.eval(p) for p in row] for row in pos]  # before the server takes the context
    outs = [[np.full(p.shape[0], np.nan) for p in row] for row in pos]
    with esp.Server(env, 1 << 14) as srv:
        def client(c):
            for k in range(reqs):
                t = srv.submit(pos[c][k], outs[c][k])
                srv.wait(t)
        th = [threading.Thread(target=client, args=(c,)) for c in range(n_clients)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        st = srv.stats()
    assert st["positions"] == sum(p.shape[0] for row in pos for p in row)
    for c in range(n_clients):
        for k in range(reqs):
            assert np.abs(outs[c][k] - single[c][k]).max() <= 2e-6
    sample = np.concatenate([pos[c][0][:8] for c in range(n_clients)])
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, sample)
    got = np.concatenate([outs[c][0][:8] for c in range(n_clients)])
    assert np.abs(got - ref).max() <= 2e-6


def test_submit_overlaps_host_work(env_wl):
    env, wl = env_wl
    p = qm_positions(np.random.default_rng(6), 2048)
    out = np.zeros(p.shape[0])
    with esp.Server(env, 4096) as srv:
        t = srv.submit(p, out)
        busy = np.linalg.norm(np.random.default_rng(7).normal(size=(200, 200)) @ np.ones(200))  # host work meanwhile
        srv.wait(t)
        assert np.isfinite(busy)
    assert np.abs(out - env.eval(p)).max() <= 2e-6


def test_server_rejects_bad_requests(env_wl):
    env, wl = env_wl
    with esp.Server(env, 16) as srv:
        with pytest.raises(esp.EspError):
            srv.submit(np.zeros((17, 3)), np.zeros(17))
        with pytest.raises(esp.EspError):
            srv.wait(12345)
