"""esp_eval_noalloc: the evaluation entry point that allocates no device memory.

Some callers of this library cannot call cudaMalloc (their device memory is
owned by another allocator, or their Monte Carlo loop must not pay
cudaMalloc's implicit synchronisation).  For them esp_eval_noalloc runs the
same staging, potential and reduction kernels with its scratch in a fixed
device array inside the library.  This file is collected last on purpose; it
passes both alone and after the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1011_4687_gb300 import build_lib, esp
from workloads import point_cells_environment, qm_positions, realistic_environment

pytestmark = pytest.mark.gpu

FP32_POINT = 2e-6   # the FP32C per-point tolerance of the parity tests
FP64_REL = 1e-10    # the FP64 relative tolerance of the parity tests


def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build_lib.build()
    lib = esp.load()
    lib.esp_eval_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    lib.esp_eval_noalloc.restype = ctypes.c_int
    return lib, torch


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_noalloc_matches_eval_on_two_calls(precision):
    lib, torch = _lib()
    wl = realistic_environment(seed=4242, n_atoms=120, n_walkers=40, n_elec=32)
    stream = torch.cuda.current_stream()
    pos = torch.from_numpy(wl.positions).cuda()
    n = pos.shape[0]
    with esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision=precision,
                         stream=stream.cuda_stream) as env:
        V_ref = env.eval(pos)
        stream.synchronize()
        V_ref = V_ref.cpu().numpy()
        for _ in range(2):
            V = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            st = lib.esp_eval_noalloc(env.handle, ctypes.c_void_p(pos.data_ptr()), n, ctypes.c_void_p(V.data_ptr()))
            assert st == esp.ESP_OK, lib.esp_last_error().decode()
            stream.synchronize()
            V = V.cpu().numpy()
            if precision == "fp32c":
                assert np.abs(V - V_ref).max() <= FP32_POINT
            else:
                assert np.all(np.abs(V - V_ref) <= FP64_REL * np.maximum(np.abs(V_ref), 1.0))


def test_noalloc_rejects_oversize_and_host_memory():
    lib, torch = _lib()
    wl = realistic_environment(seed=4243, n_atoms=20, n_walkers=2, n_elec=4)
    with esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs) as env:
        big = 65536 + 1
        pos = torch.zeros((big, 3), dtype=torch.float64, device="cuda")
        V = torch.zeros(big, dtype=torch.float64, device="cuda")
        st = lib.esp_eval_noalloc(env.handle, ctypes.c_void_p(pos.data_ptr()), big, ctypes.c_void_p(V.data_ptr()))
        assert st == esp.ESP_ERR_INVALID
        hp = np.zeros((8, 3))
        hv = np.zeros(8)
        st = lib.esp_eval_noalloc(env.handle, ctypes.c_void_p(hp.ctypes.data), 8, ctypes.c_void_p(hv.ctypes.data))
        assert st == esp.ESP_ERR_INVALID


def _noalloc(lib, env, pos, V):
    st = lib.esp_eval_noalloc(env.handle, ctypes.c_void_p(pos.data_ptr()), int(pos.shape[0]),
                              ctypes.c_void_p(V.data_ptr()))
    assert st == esp.ESP_OK, lib.esp_last_error().decode()


def test_noalloc_sizes_vs_oracle_and_no_memory_growth():
    """The largest accepted size (65,536 positions: the 8 partial-sum rows reach
    the end of the fixed array) and 1..16 positions (which esp_eval sends to
    another path), checked against the FP64 oracle on sampled positions; and a
    warm call changes neither the device's free memory nor torch's."""
    lib, torch = _lib()
    wl = realistic_environment(seed=4244, n_atoms=60, n_walkers=2, n_elec=8)
    stream = torch.cuda.current_stream()
    n_max = 65536
    pos_np = qm_positions(np.random.default_rng(4245), n_max)
    pos = torch.from_numpy(pos_np).cuda()
    V = torch.empty(n_max, dtype=torch.float64, device="cuda")
    with esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision="fp32c",
                         stream=stream.cuda_stream) as env:
        _noalloc(lib, env, pos, V)  # first call on the device: may load the module
        stream.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        alloc0 = torch.cuda.memory_allocated()
        _noalloc(lib, env, pos, V)
        stream.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_allocated() == alloc0
        pick = np.concatenate([np.arange(16), np.arange(n_max - 8, n_max), np.arange(1000, n_max, 4099)])
        ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, pos_np[pick])
        assert np.abs(V.cpu().numpy()[pick] - ref).max() <= FP32_POINT
        for n in (1, 5, 16):  # pick[:16] are positions 0..15
            Vn = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            _noalloc(lib, env, pos[:n].contiguous(), Vn)
            stream.synchronize()
            assert np.abs(Vn.cpu().numpy() - ref[:n]).max() <= FP32_POINT


def test_noalloc_point_charges_only():
    """An environment of point charges only (the paper's cells and nuclei)."""
    lib, torch = _lib()
    wl = point_cells_environment(seed=4246, n_cells=3000, n_nuclei=12, n_positions=40)
    stream = torch.cuda.current_stream()
    pos = torch.from_numpy(wl.positions.copy()).cuda()
    V = torch.empty(pos.shape[0], dtype=torch.float64, device="cuda")
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    with esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision="fp32c",
                         stream=stream.cuda_stream) as env:
        for _ in range(2):
            _noalloc(lib, env, pos, V)
            stream.synchronize()
            assert np.abs(V.cpu().numpy() - ref).max() <= FP32_POINT
