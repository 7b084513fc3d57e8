"""CPU tests of the library's host side (no GPU needed).

* the C-ABI library builds, loads and exports every function include/esp.h declares;
* the device Boys algorithm (tables + Taylor + recursions + asymptotic form), run
  on the host through a test hook, matches the oracle's independent Boys function;
* the pair builder (canonical orientation, folding into Hermite distributions,
  McMurchie-Davidson coefficients, screening, tiling), checked through the host
  test hook of a host-only context against the Obara-Saika oracle;
* input validation returns ESP_ERR_INVALID without touching a GPU.
"""
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_1011_4687_gb300 import build_lib, esp
from workloads import PairList, small_environment, tiny_pd_environment
from workloads.generate import CART

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return esp.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "esp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(esp_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_header_function(lib):
    names = header_functions()
    assert "esp_create" in names and "esp_eval" in names and "esp_destroy" in names
    for name in names:
        assert hasattr(lib, name), name
    assert lib.esp_abi_version() == 1


def test_status_strings(lib):
    for s in range(7):
        assert lib.esp_status_string(s).decode()


@pytest.mark.parametrize("prec,rtol", [("fp64", 5e-15), ("fp32c", 1e-6)])
def test_device_boys_algorithm_matches_oracle(lib, prec, rtol):
    Ts = np.concatenate([[0.0, 1e-9, 1e-5, 0.0624, 0.0626], np.geomspace(1e-3, 2e3, 200),
                         [29.99, 30.0, 30.01, 44.99, 45.0, 45.01]])
    for T in Ts:
        if prec == "fp32c":
            T = float(np.float32(T))
        ref = oracle.boys(4, float(T))
        for nmax in range(5):
            F = esp.debug_boys(prec, nmax, float(T))
            assert np.allclose(F, ref[:nmax + 1], rtol=rtol, atol=0), (prec, T, nmax, F, ref)


def _host_env(wl, screen_tol=0.0, tile_size=0, precision="fp64", near_radius=-1.0):
    lib = esp.load()
    import ctypes
    opt = esp.default_options()
    opt.flags = 1  # ESP_FLAG_HOST_ONLY
    opt.precision = esp.PRECISIONS[precision]
    opt.near_radius = near_radius
    opt.screen_tol = screen_tol
    opt.tile_size = tile_size
    opt.qm_center[:] = list(map(float, wl.qm_center))
    ch = esp.pack_charges(wl.nuclei_xyz, wl.nuclei_Z)
    pr = esp.pack_pairs(wl.pairs)
    w = np.ascontiguousarray(wl.pairs.w)
    ctx = ctypes.c_void_p()
    esp._check(lib.esp_create(ch.ctypes.data if ch.size else None, ch.size, pr.ctypes.data if pr.size else None,
                              w.ctypes.data if w.size else None, pr.size, ctypes.byref(opt), ctypes.byref(ctx)))
    env = esp.Environment.__new__(esp.Environment)
    env._ctx = ctx
    env.stream = None
    return env


def test_builder_pd_pairs_vs_oracle(lib):
    for seed in range(6):
        wl = tiny_pd_environment(100 + seed, n_pairs=40, n_nuclei=5, n_pos=12, exp_range=(0.1, 60.0))
        env = _host_env(wl, tile_size=64)
        V = env.debug_host_eval(wl.positions)
        ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
        assert np.allclose(V, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max()), (seed, V - ref)
        env.close()


def test_builder_folds_shared_shell_pairs(lib):
    """Component pairs of one shell pair (same A, alpha, B, beta) fold into one
    distribution; a reversed orientation of the same pair folds into it too."""
    rng = np.random.default_rng(5)
    A, B = rng.normal(size=3), rng.normal(size=3)
    rows = []
    for la in CART[1]:
        for lb in CART[2]:
            rows.append((A, 0.7, la, B, 1.9, lb, rng.normal()))
    # the same functions with A and B swapped
    for la in CART[1]:
        rows.append((B, 1.9, (0, 0, 0), A, 0.7, la, rng.normal()))
    pl = PairList(np.array([r[0] for r in rows]), np.array([r[1] for r in rows]),
                  np.array([r[2] for r in rows], np.int32), np.array([r[3] for r in rows]),
                  np.array([r[4] for r in rows]), np.array([r[5] for r in rows], np.int32),
                  np.array([r[6] for r in rows]))
    from workloads import Workload
    pos = rng.normal(size=(7, 3)) * 2
    wl = Workload("fold", np.zeros((0, 3)), np.zeros(0), pl, pos, 1, 7, np.zeros(3), {})
    env = _host_env(wl)
    info = env.info()
    assert info["n_distributions"] == 1 and info["n_by_L"][3] == 1
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, pl, pos)
    assert np.allclose(env.debug_host_eval(pos), ref, rtol=1e-12, atol=1e-13)


def test_builder_small_environment_vs_oracle(lib):
    wl = small_environment(n_walkers=2, n_elec=10)
    env = _host_env(wl, screen_tol=1e-12)
    info = env.info()
    assert info["n_point_charges"] == 200 and info["n_distributions"] == 2000
    V = env.debug_host_eval(wl.positions)
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    assert np.max(np.abs(V - ref)) <= 1e-10 * max(1.0, np.abs(ref).max())


def test_recentering_is_exact_translation(lib):
    wl = tiny_pd_environment(77, n_pairs=20, n_nuclei=4, n_pos=6)
    wl.qm_center = np.array([12.5, -3.25, 7.0])
    env = _host_env(wl)
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    assert np.allclose(env.debug_host_eval(wl.positions), ref, rtol=1e-12, atol=1e-12)


def test_screening_drops_only_negligible_charge(lib):
    wl = tiny_pd_environment(31, n_pairs=30, n_nuclei=0, n_pos=5)
    wl.pairs.w[:10] *= 1e-15
    env = _host_env(wl, screen_tol=1e-12)
    info = env.info()
    assert info["n_screened"] >= 1
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    assert np.allclose(env.debug_host_eval(wl.positions), ref, rtol=1e-10, atol=1e-12)


def _bad_create(pairs=None, charges=None, **optkw):
    import ctypes
    lib = esp.load()
    opt = esp.default_options()
    opt.flags = 1
    for k, v in optkw.items():
        setattr(opt, k, v)
    if pairs is None:
        pairs = PairList.empty()
    ch = charges if charges is not None else esp.pack_charges(np.zeros((0, 3)), np.zeros(0))
    pr = esp.pack_pairs(pairs)
    w = np.ascontiguousarray(pairs.w)
    ctx = ctypes.c_void_p()
    return lib.esp_create(ch.ctypes.data if ch.size else None, ch.size, pr.ctypes.data if pr.size else None,
                          w.ctypes.data if w.size else None, pr.size, ctypes.byref(opt), ctypes.byref(ctx)), ctx


@pytest.mark.parametrize("field,value", [("alpha", -1.0), ("alpha", 0.0), ("alpha", float("nan")),
                                         ("A", float("inf")), ("w", float("nan")), ("la", 3)])
def test_invalid_pairs_rejected(lib, field, value):
    wl = tiny_pd_environment(3, n_pairs=4, n_nuclei=0, lmax=1)
    pl = wl.pairs.copy()
    arr = getattr(pl, field)
    if field == "la":
        arr[1] = [value, 0, 0]
        pl.lb[1] = [2, 0, 0]
    elif arr.ndim == 2:
        arr[1, 0] = value
    else:
        arr[1] = value
    st, ctx = _bad_create(pl)
    assert st == esp.ESP_ERR_INVALID and not ctx.value
    assert esp.load().esp_last_error().decode()


def test_invalid_options_rejected(lib):
    assert _bad_create(tile_size=100)[0] == esp.ESP_ERR_INVALID
    assert _bad_create(precision=7)[0] == esp.ESP_ERR_INVALID
    assert _bad_create(screen_tol=-1.0)[0] == esp.ESP_ERR_INVALID
    ch = esp.pack_charges(np.array([[0.0, float("nan"), 0.0]]), np.array([1.0]))
    assert _bad_create(charges=ch)[0] == esp.ESP_ERR_INVALID


def test_host_only_context_refuses_evaluation(lib):
    wl = tiny_pd_environment(4, n_pairs=3, n_nuclei=1)
    env = _host_env(wl)
    with pytest.raises(esp.EspError) as ei:
        env.eval(np.zeros((2, 3)))
    assert ei.value.status == esp.ESP_ERR_STATE
    env.close()
    esp.load().esp_destroy(None)  # NULL-safe


# ---------------------------------------------------------------------------
# error budget of the FP32-compensated arithmetic (host emulation of the kernel)
# ---------------------------------------------------------------------------
def test_fp32c_budget_small_environment(lib):
    wl = small_environment(n_walkers=10, n_elec=100)
    env = _host_env(wl, screen_tol=1e-12, precision="fp32c")
    V = env.debug_host_eval(wl.positions)
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    assert np.abs(V - ref).max() <= 2e-6
    E = -V.reshape(10, 100).sum(1)
    Eref = oracle.walker_energies(ref, 10, 100)
    assert np.abs(E - Eref).max() <= 1e-5
    # no bias: the mean error is far below the per-point scatter
    assert abs(np.mean(V - ref)) <= 3e-8


def test_fp32c_budget_realistic_environment(lib):
    from workloads import realistic_environment
    wl = realistic_environment(seed=7711, n_atoms=200, n_walkers=4, n_elec=32)
    env = _host_env(wl, screen_tol=1e-12, precision="fp32c")
    V = env.debug_host_eval(wl.positions)
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    assert np.abs(V - ref).max() <= 2e-6
    E = -V.reshape(4, 32).sum(1)
    assert np.abs(E - oracle.walker_energies(ref, 4, 32)).max() <= 1e-5


def test_onsite_monopoles_move_to_point_charges(lib):
    """On-site distributions centred on a nucleus give their monopole to it; the
    evaluated sum is unchanged (FP64) and the point count does not grow."""
    from workloads import realistic_environment
    wl = realistic_environment(seed=99, n_atoms=30, n_walkers=2, n_elec=8)
    env = _host_env(wl, screen_tol=0.0, precision="fp64")
    info = env.info()
    assert info["n_point_charges"] == 30
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    assert np.allclose(env.debug_host_eval(wl.positions), ref, rtol=1e-12, atol=1e-12)
    env32 = _host_env(wl, screen_tol=0.0, precision="fp32c")
    assert np.abs(env32.debug_host_eval(wl.positions) - ref).max() <= 2e-6
    # a position 1e-3 bohr from a nucleus (|V| ~ 7e3): FP64 to 1e-12, FP32C to a
    # few FP32 ulps relative (the short-range remainder is large there)
    C = wl.nuclei_xyz[3] + np.array([1e-3, 0.0, 0.0])
    r1 = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, C[None])
    assert np.allclose(env.debug_host_eval(C[None]), r1, rtol=1e-12)
    assert np.allclose(env32.debug_host_eval(C[None]), r1, rtol=2e-7)


def test_batch_refuses_host_only_contexts(lib):
    import ctypes
    wl = tiny_pd_environment(6, n_pairs=4, n_nuclei=1)
    env = _host_env(wl)
    arr = (ctypes.c_void_p * 1)(env.handle.value)
    b = ctypes.c_void_p()
    assert lib.esp_batch_create(arr, 1, None, ctypes.byref(b)) == esp.ESP_ERR_STATE
    assert lib.esp_batch_create(arr, 0, None, ctypes.byref(b)) == esp.ESP_ERR_INVALID
    lib.esp_batch_destroy(None)


def test_small_point_charges_fp32_class_on_host():
    """Small point charges (the paper's cells) go to the FP32 point class; the
    kernels' own per-tile code run on the host meets the FP32C bound against
    the oracle, and with the threshold at 0 every charge stays FP64."""
    from workloads import point_cells_environment
    wl = point_cells_environment(77, n_cells=3000, n_nuclei=12, n_positions=20)
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    with esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision="fp32c",
                         flags=esp.FLAG_HOST_ONLY) as env:
        assert env.info()["n_point_charges"] == 3012
        V = env.debug_host_eval(wl.positions)
    assert np.abs(V - ref).max() <= 2e-6
    with esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision="fp64",
                         flags=esp.FLAG_HOST_ONLY, point32_max_charge=0.0) as env:
        V = env.debug_host_eval(wl.positions)
    assert np.allclose(V, ref, rtol=1e-12, atol=1e-12)
