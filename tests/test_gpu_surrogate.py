"""The learned surrogate on the GPU: gradients of the library's BF16 tensor-core
kernels against the CPU reference network, and the surrogate + exact-fallback
contract against the FP64 oracle."""
import functools
import os

import numpy as np
import pytest

import oracle
from oracle import mlp_reference as ref
from paper_1011_4687_gb300 import build_lib, esp
from workloads import qm_positions, small_environment

pytestmark = pytest.mark.gpu

TOL = 2e-6


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build_lib.build()
    esp.load()
    return t


@functools.lru_cache(maxsize=None)
def env_small():
    return small_environment(seed=8801, n_nuclei=60, n_charges=600, n_walkers=4, n_elec=64)


def test_gradients_match_cpu_reference(torch):
    wl = env_small()
    env = esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs)
    with esp.Surrogate(env, n_train=2048, n_valid=512, epochs=0, degree=4) as sur:
        rng = np.random.default_rng(5)
        pos = qm_positions(rng, 512)
        t = rng.normal(size=512).astype(np.float32)
        params, grad, y = sur.debug_step(pos, t)
        freq, c, inv_r = sur.features()
        yr, _ = ref.forward(params.astype(np.float64), freq, c, inv_r, pos, use_bf16=True)
        assert np.abs(y - yr).max() <= 2e-2 * max(1.0, np.abs(yr).max())
        _, gr = ref.loss_and_grad(params.astype(np.float64), freq, c, inv_r, pos, t.astype(np.float64),
                                  use_bf16=True)
        spec, _ = ref.layout()
        for name, off, shape in spec:
            n = int(np.prod(shape)) if shape else 1
            a, b = grad[off:off + n].astype(np.float64), gr[off:off + n]
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
            assert rel <= 5e-2, (name, rel)
    env.close()


@functools.lru_cache(maxsize=None)
def trained(torch_mod):
    wl = env_small()
    env = esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs)
    sur = esp.Surrogate(env, n_train=1 << 17, n_valid=1 << 15, epochs=6, batch=4096)
    return wl, env, sur


def _check_fused_network(sur, pos):
    """The fused tcgen05 inference kernel against the CPU reference network
    (FP64 with the kernels' BF16 rounding points) and against the unfused
    mma.sync forward pass of the training path."""
    y_tc = sur.debug_net(pos).astype(np.float64)
    params, _, y_mma = sur.debug_step(pos, np.zeros(pos.shape[0], np.float32))
    freq, c, inv_r = sur.features()
    yr, _ = ref.forward(params.astype(np.float64), freq, c, inv_r, pos, use_bf16=True)
    scale = max(1e-3, np.abs(yr).max())
    assert np.all(np.isfinite(y_tc))
    assert np.abs(y_tc - yr).max() <= 2e-2 * scale
    assert np.abs(y_tc - y_mma).max() <= 5e-3 * scale
    # outputs spread across the rows: a transposed or misplaced operand tile
    # would not keep the per-position values in step with the reference
    if pos.shape[0] > 2:
        assert np.corrcoef(y_tc, yr)[0, 1] > 0.999


def test_fused_network_matches_reference_untrained(torch):
    wl = env_small()
    env = esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs)
    with esp.Surrogate(env, n_train=2048, n_valid=512, epochs=0, degree=4) as sur:
        # 1,000 positions: 7 full CTAs of 128 rows and a ragged last one
        _check_fused_network(sur, qm_positions(np.random.default_rng(11), 1000))
        _check_fused_network(sur, qm_positions(np.random.default_rng(12), 1))
    env.close()


def test_fused_network_matches_reference_trained(torch):
    wl, env, sur = trained(torch)
    _check_fused_network(sur, qm_positions(np.random.default_rng(13), 4099))


def test_surrogate_with_fallback_meets_tolerance(torch):
    wl, env, sur = trained(torch)
    info = sur.info()
    # the network improves on the baseline alone
    assert info["valid_rms_err"] < info["baseline_rms_err"]
    rng = np.random.default_rng(77)
    pos = qm_positions(rng, 4096)
    V, st = sur.eval(torch.from_numpy(pos).cuda())
    torch.cuda.synchronize()
    ref_v = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, pos)
    assert np.abs(V.cpu().numpy() - ref_v).max() <= TOL
    assert 0 < st["n_fallback"] <= pos.shape[0]
    # a second call: the probe moves, results stay within tolerance
    V2, st2 = sur.eval(torch.from_numpy(pos).cuda())
    torch.cuda.synchronize()
    assert np.abs(V2.cpu().numpy() - ref_v).max() <= TOL


def test_save_load_round_trip(torch, tmp_path):
    wl, env, sur = trained(torch)
    path = str(tmp_path / "sur.bin")
    sur.save(path)
    other = esp.Surrogate.load(env, path)
    pos = torch.from_numpy(qm_positions(np.random.default_rng(3), 1000)).cuda()
    a = sur.predict(pos)
    b = other.predict(pos)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    with open(path, "r+b") as f:
        f.seek(200)
        byte = f.read(1)
        f.seek(200)
        f.write(bytes([byte[0] ^ 0xFF]))
    with pytest.raises(esp.EspError):
        esp.Surrogate.load(env, path)
    other.close()
