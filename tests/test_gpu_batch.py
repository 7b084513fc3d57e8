"""Batched evaluation (persistent kernel + CUDA graph + autotuner) on the GPU.

Each system of a batch must give what esp_eval gives for that system alone
(within the FP32C / FP64 tolerances of the parity tests), and the small
systems are also checked against the FP64 oracle directly."""
import numpy as np
import pytest

import oracle
from paper_1011_4687_gb300 import build_lib, esp
from workloads import realistic_environment, small_environment, tiny_pd_environment, qm_positions

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build_lib.build()
    esp.load()
    return t


def systems(seed):
    wls = [realistic_environment(seed=seed + k, n_atoms=na, n_walkers=nw, n_elec=32)
           for k, (na, nw) in enumerate([(150, 20), (40, 3), (90, 1), (20, 40)])]
    wls.append(small_environment(seed=seed + 9, n_nuclei=50, n_charges=300, n_walkers=7, n_elec=11))
    wls.append(tiny_pd_environment(seed + 10, n_pairs=50, n_nuclei=5, n_pos=0))
    return wls


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_batch_matches_single_evaluations(torch, prec):
    wls = systems(300)
    stream = torch.cuda.current_stream()
    envs = [esp.Environment(w.nuclei_xyz, w.nuclei_Z, w.pairs, precision=prec, stream=stream.cuda_stream)
            for w in wls]
    pos = [torch.from_numpy(w.positions.reshape(-1, 3)).cuda() for w in wls]
    with esp.Batch(envs, stream=stream.cuda_stream) as b:
        outs = b.eval(pos)
        stream.synchronize()
        for k, (w, e) in enumerate(zip(wls, envs)):
            if w.positions.shape[0] == 0:
                assert outs[k].numel() == 0
                continue
            single = e.eval(w.positions)
            got = outs[k].cpu().numpy()
            if prec == "fp64":
                assert np.all(np.abs(got - single) <= 1e-10 * np.maximum(np.abs(single), 1.0)), k
            else:
                assert np.abs(got - single).max() <= 2e-6, k
        # graph replay with new positions for every system
        rng = np.random.default_rng(1)
        new = [qm_positions(rng, int(p.shape[0])) for p in pos]
        pos2 = [torch.from_numpy(x).cuda() for x in new]
        outs2 = b.eval(pos2)
        stream.synchronize()
        for k in (1, 2, 4):
            ref = oracle.potential(wls[k].nuclei_xyz, wls[k].nuclei_Z, wls[k].pairs, new[k])
            got = outs2[k].cpu().numpy()
            if prec == "fp64":
                assert np.all(np.abs(got - ref) <= 1e-10 * np.maximum(np.abs(ref), 1.0)), k
            else:
                assert np.abs(got - ref).max() <= 2e-6, k
    for e in envs:
        e.close()


def test_batch_spatial_order(torch):
    """Systems of >= 4,096 positions are staged in spatial order inside the
    batch's graph: results return in input order and match the oracle, across
    replays with new positions."""
    wls = [realistic_environment(seed=510, n_atoms=60, n_walkers=130, n_elec=32),   # 4,160 positions: ordered
           realistic_environment(seed=511, n_atoms=30, n_walkers=5, n_elec=32)]     # 160 positions: not ordered
    stream = torch.cuda.current_stream()
    envs = [esp.Environment(w.nuclei_xyz, w.nuclei_Z, w.pairs, stream=stream.cuda_stream) for w in wls]
    rng = np.random.default_rng(7)
    with esp.Batch(envs, stream=stream.cuda_stream) as b:
        for rep in range(2):
            host = [w.positions if rep == 0 else qm_positions(rng, w.positions.shape[0]) for w in wls]
            outs = b.eval([torch.from_numpy(x).cuda() for x in host])
            stream.synchronize()
            for k, w in enumerate(wls):
                pick = np.arange(0, host[k].shape[0], 37)
                ref = oracle.potential(w.nuclei_xyz, w.nuclei_Z, w.pairs, host[k][pick])
                assert np.abs(outs[k].cpu().numpy()[pick] - ref).max() <= 2e-6, (rep, k)
                single = envs[k].eval(host[k])
                assert np.abs(outs[k].cpu().numpy() - single).max() <= 2e-6, (rep, k)
    for e in envs:
        e.close()


def test_batch_autotune_and_cache(torch, tmp_path):
    wls = systems(400)[:4]
    stream = torch.cuda.current_stream()
    envs = [esp.Environment(w.nuclei_xyz, w.nuclei_Z, w.pairs, stream=stream.cuda_stream) for w in wls]
    pos = [torch.from_numpy(w.positions).cuda() for w in wls]
    cache = str(tmp_path / "tune.json")
    with esp.Batch(envs, stream=stream.cuda_stream) as b:
        rep = b.autotune(pos, cache_path=cache)
        assert not rep["cached"] and len(rep["tried"]) == 12 and rep["best_ms"] > 0
        again = b.autotune(pos, cache_path=cache)
        assert again["cached"] and again["threads_per_block"] == rep["threads_per_block"]
        outs = b.eval(pos)
        stream.synchronize()
        for k in (1, 2):
            ref = oracle.potential(wls[k].nuclei_xyz, wls[k].nuclei_Z, wls[k].pairs, wls[k].positions)
            assert np.abs(outs[k].cpu().numpy() - ref).max() <= 2e-6
        assert b.last_ms() > 0
    for e in envs:
        e.close()


def test_batch_rejects_mixed_precision_and_host_memory(torch):
    w = tiny_pd_environment(5, n_pairs=10, n_nuclei=2, n_pos=4)
    e1 = esp.Environment(w.nuclei_xyz, w.nuclei_Z, w.pairs, precision="fp32c")
    e2 = esp.Environment(w.nuclei_xyz, w.nuclei_Z, w.pairs, precision="fp64")
    with pytest.raises(esp.EspError) as ei:
        esp.Batch([e1, e2])
    assert ei.value.status == esp.ESP_ERR_INVALID
    with esp.Batch([e1]) as b:
        import ctypes
        hp = np.zeros((4, 3))
        hv = np.zeros(4)
        P = (ctypes.c_void_p * 1)(hp.ctypes.data)
        V = (ctypes.c_void_p * 1)(hv.ctypes.data)
        N = (ctypes.c_int64 * 1)(4)
        assert esp.load().esp_batch_eval(b._b, P, N, V) == esp.ESP_ERR_INVALID
    e1.close()
    e2.close()
