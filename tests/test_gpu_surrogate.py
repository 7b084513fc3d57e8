"""The learned surrogate on the GPU: gradients of the library's BF16 tensor-core
kernels against the CPU reference network, the fused inference kernel against
that reference, and the surrogate's contract against the FP64 oracle: values
served by expansion + network (not by the fallback) are checked element by
element at 2e-6 Ha, walker energies at 1e-5 Ha, and a probe that fails makes
its voxel's positions exact within the same call."""
import functools

import numpy as np
import pytest

import oracle
from oracle import mlp_reference as ref
from paper_1011_4687_gb300 import build_lib, esp
from workloads import qm_positions, realistic_environment, small_environment

pytestmark = pytest.mark.gpu

TOL = 2e-6
WALKER_TOL = 1e-5


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


@pytest.mark.parametrize("n", [512, 40960])
def test_gradients_match_cpu_reference(torch, n):
    """Every parameter's gradient against the FP64 reference network with the
    kernels' BF16 rounding points, element by element: |g - g_ref| <= 2e-2 |g_ref|
    + 2^-8 max|g_ref| of its block (BF16 keeps 8 significant bits).  512
    positions run the tcgen05 GEMMs on 64-column tiles; 40,960 positions (320
    row tiles) on 256-column tiles for the forward and input-gradient GEMMs."""
    wl = env_small()
    env = esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs)
    with esp.Surrogate(env, n_train=2048, n_valid=512, epochs=0, degree=4) as sur:
        rng = np.random.default_rng(5)
        pos = qm_positions(rng, n)
        t = rng.normal(size=n).astype(np.float32)
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
            lim = 2e-2 * np.abs(b) + 2.0 ** -8 * np.abs(b).max()
            bad = np.abs(a - b) > lim
            assert not bad.any(), (name, int(bad.sum()), float((np.abs(a - b) / np.maximum(lim, 1e-300)).max()))
    env.close()


def _check_fused_network(sur, pos):
    """The fused tcgen05 inference kernel against the CPU reference network
    (FP64 with the kernels' BF16 rounding points) and against the unfused
    forward pass of the training path (its own tcgen05 GEMMs)."""
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


# ---------------------------------------------------------------------------
# the realistic environment (2,000 atoms): near tiles exact, far tiles by
# expansion + network
# ---------------------------------------------------------------------------
@functools.lru_cache(maxsize=None)
def realistic():
    return realistic_environment(seed=6602, n_atoms=2000, n_walkers=16, n_elec=32)


@pytest.fixture(scope="module")
def trained_sur(torch):
    """One surrogate of the realistic environment for the tests below; closed
    (surrogate first, then its environment) when the module's tests end."""
    wl = realistic()
    env = esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs)
    sur = esp.Surrogate(env, n_train=1 << 18, n_valid=1 << 16, epochs=8)
    yield wl, env, sur
    sur.close()
    env.close()


@functools.lru_cache(maxsize=None)
def oracle_at(n):
    wl = realistic()
    pos = np.concatenate([wl.positions, qm_positions(np.random.default_rng(90), n - wl.positions.shape[0])])
    return pos, oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, pos)


def test_fused_network_matches_reference_trained(trained_sur):
    wl, env, sur = trained_sur
    _check_fused_network(sur, qm_positions(np.random.default_rng(13), 4099))


def test_served_positions_match_oracle(torch, trained_sur):
    """Positions the surrogate serves (expansion + network, no fallback) agree
    with the FP64 oracle element by element at 2e-6 Ha; at least a third of the
    positions are served; the 16 whole walkers meet 1e-5 Ha."""
    wl, env, sur = trained_sur
    info = sur.info()
    assert info["n_far_entries"] > 0 and info["n_near_entries"] > 0
    assert info["trusted_fraction"] > 0.3, info
    pos, ref_v = oracle_at(1024)
    V, st = sur.eval(torch.from_numpy(pos).cuda())
    torch.cuda.synchronize()
    V = V.cpu().numpy()
    # which positions were served: the trust map decides, plus every 64th probe
    Vp = sur.predict(torch.from_numpy(pos).cuda())
    torch.cuda.synchronize()
    served = V == Vp.cpu().numpy()
    assert served.mean() >= 1.0 / 3.0, (served.mean(), st)
    assert np.abs(V[served] - ref_v[served]).max() <= TOL
    assert np.abs(V - ref_v).max() <= TOL
    n = wl.n_walkers * wl.n_elec
    E = -V[:n].reshape(wl.n_walkers, wl.n_elec).sum(1)
    Eref = oracle.walker_energies(ref_v[:n], wl.n_walkers, wl.n_elec)
    assert np.abs(E - Eref).max() <= WALKER_TOL


def test_network_gains_over_expansion_alone(trained_sur):
    """The method without the network (the far field's expansion alone) against
    the same with the network, on the validation set of the far field: at the
    default degree the network lowers the error and serves at least as many
    voxels."""
    wl, env, sur = trained_sur
    info = sur.info()
    assert info["valid_rms_err"] < info["baseline_rms_err"], info
    assert info["valid_max_err"] < info["baseline_max_err"], info
    assert info["trusted_fraction"] >= info["baseline_trusted_fraction"], info


def test_network_gain_at_low_expansion_degree(torch):
    """With a degree-8 expansion the far field's truncation error is well above
    the tolerance; the trained network removes most of it (rms at least 4x
    lower) and earns many more trusted voxels than the expansion alone."""
    wl = realistic()
    with esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs) as env:
        with esp.Surrogate(env, n_train=1 << 18, n_valid=1 << 16, epochs=8, degree=8) as sur:
            info = sur.info()
    assert info["baseline_max_err"] > TOL, info
    assert info["valid_rms_err"] * 4 <= info["baseline_rms_err"], info
    assert info["trusted_fraction"] >= info["baseline_trusted_fraction"] + 0.2, info


def test_failed_probe_makes_its_voxel_exact_in_the_same_call(torch, trained_sur, tmp_path):
    """A planted error (1e-3 Ha added to the expansion) fails every probe; the
    positions are laid out 64 to a voxel, so every voxel holds one probe of the
    call, and every returned value must still meet 2e-6 against the oracle."""
    wl, env, sur = trained_sur
    path = str(tmp_path / "sur.bin")
    sur.save(path)
    other = esp.Surrogate.load(env, path)
    try:
        vox = 0.25
        rng = np.random.default_rng(91)
        centres = qm_positions(rng, 12, sd=1.5)
        centres = (np.floor(centres / vox) + 0.5) * vox
        pos = np.concatenate([c + rng.uniform(-0.45 * vox, 0.45 * vox, size=(64, 3)) for c in centres])
        ref_v = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, pos)
        other.debug_expansion(1e-3)
        V, st = other.eval(torch.from_numpy(pos).cuda())
        torch.cuda.synchronize()
        assert st["n_probe_fail"] > 0
        assert np.abs(V.cpu().numpy() - ref_v).max() <= TOL
    finally:
        other.close()


def test_save_load_round_trip(torch, trained_sur, tmp_path):
    wl, env, sur = trained_sur
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
