"""Failure detection without a GPU fault.

Host side: the environment variable ESP_FAULT makes named operations fail as
if their CUDA call had failed ("alloc", "upload", "graph"); each call must
return its status, leave its outputs alone, and the next call after the
variable is cleared must succeed on the same context.  Device side: the
surrogate network kernel's bounded waits are given a limit of 0, so every
first wait gives up (the fused inference kernel and the training GEMMs); the
call must return ESP_ERR_TIMEOUT and the context and
surrogate must work again with the default limit."""
import os

import numpy as np
import pytest

from paper_1011_4687_gb300 import build_lib, esp
from workloads import qm_positions, small_environment


@pytest.fixture(autouse=True)
def _clean_env():
    old = os.environ.pop("ESP_FAULT", None)
    yield
    os.environ.pop("ESP_FAULT", None)
    if old is not None:
        os.environ["ESP_FAULT"] = old


def test_fault_names_are_parsed():
    build_lib.build()
    esp.load()
    assert not esp.debug_fault_active("alloc")
    os.environ["ESP_FAULT"] = "upload,graph"
    assert esp.debug_fault_active("upload") and esp.debug_fault_active("graph")
    assert not esp.debug_fault_active("alloc") and not esp.debug_fault_active("grap")
    os.environ["ESP_FAULT"] = "alloc"
    assert esp.debug_fault_active("alloc")


def _small():
    return small_environment(seed=8805, n_nuclei=30, n_charges=300, n_walkers=2, n_elec=32)


@pytest.mark.gpu
def test_alloc_and_upload_faults_fail_cleanly():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build_lib.build()
    wl = _small()
    os.environ["ESP_FAULT"] = "upload"
    with pytest.raises(esp.EspError) as ei:
        esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs)
    assert ei.value.status == esp.ESP_ERR_CUDA
    os.environ["ESP_FAULT"] = "alloc"
    with pytest.raises(esp.EspError) as ei:
        esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs)
    assert ei.value.status == esp.ESP_ERR_OOM
    del os.environ["ESP_FAULT"]
    with esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs) as env:
        V0 = env.eval(wl.positions)
        # the scratch of a larger call cannot be allocated: the call fails and
        # leaves its output untouched; the context works again afterwards
        big = qm_positions(np.random.default_rng(1), 5000)
        out = np.full(big.shape[0], 7.0)
        os.environ["ESP_FAULT"] = "alloc"
        with pytest.raises(esp.EspError) as ei:
            env.eval(big, out=out)
        assert ei.value.status == esp.ESP_ERR_OOM
        assert np.all(out == 7.0)
        del os.environ["ESP_FAULT"]
        assert np.array_equal(env.eval(wl.positions), V0)
        assert np.all(np.isfinite(env.eval(big)))


@pytest.mark.gpu
def test_graph_fault_fails_cleanly():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build_lib.build()
    wl = _small()
    with esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs) as env:
        pos = [torch.from_numpy(wl.positions).cuda()]
        ref = env.eval(pos[0])
        torch.cuda.synchronize()
        b = esp.Batch([env])
        os.environ["ESP_FAULT"] = "graph"
        with pytest.raises(esp.EspError) as ei:
            b.eval(pos)
        assert ei.value.status == esp.ESP_ERR_CUDA
        del os.environ["ESP_FAULT"]
        out = b.eval(pos)
        torch.cuda.synchronize()
        assert torch.allclose(out[0], ref, rtol=0, atol=2e-6)
        b.close()


@pytest.mark.gpu
def test_network_wait_limit_zero_times_out_and_recovers():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build_lib.build()
    wl = _small()
    with esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs) as env:
        with esp.Surrogate(env, n_train=4096, n_valid=1024, epochs=1, degree=4) as sur:
            pos = torch.from_numpy(qm_positions(np.random.default_rng(2), 1000)).cuda()
            ref = sur.predict(pos)
            torch.cuda.synchronize()
            sur.set_wait_limit(0)
            with pytest.raises(esp.EspError) as ei:
                sur.predict(pos)
            assert ei.value.status == esp.ESP_ERR_TIMEOUT
            with pytest.raises(esp.EspError) as ei:
                sur.eval(pos)
            assert ei.value.status == esp.ESP_ERR_TIMEOUT
            # the training GEMMs (tcgen05) take the same limit
            tpos = qm_positions(np.random.default_rng(3), 300)
            tgt = np.random.default_rng(4).normal(size=300).astype(np.float32)
            with pytest.raises(esp.EspError) as ei:
                sur.debug_step(tpos, tgt)
            assert ei.value.status == esp.ESP_ERR_TIMEOUT
            sur.set_wait_limit(-1)
            _, g1, y1 = sur.debug_step(tpos, tgt)
            _, g2, y2 = sur.debug_step(tpos, tgt)
            assert np.all(np.isfinite(g1)) and np.array_equal(g1, g2) and np.array_equal(y1, y2)
            again = sur.predict(pos)
            torch.cuda.synchronize()
            assert torch.equal(again, ref)
            V, st = sur.eval(pos)
            torch.cuda.synchronize()
            assert torch.all(torch.isfinite(V))
            # the context itself is unaffected
            assert np.all(np.isfinite(env.eval(wl.positions)))
