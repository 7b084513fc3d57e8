"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (written here; the FP32C bounds are the paper's accuracy target
restated per point and per walker):
  FP64 path : |V - V_oracle| <= 1e-10 * max(|V_oracle|, 1 Ha/e) per point;
  FP32C path: |V - V_oracle| <= 2e-6 Ha/e per point and
              |E_w - E_w,oracle| <= 1e-5 Ha per walker (E_w = -sum_e V);
              in the synthetic p/d environments, where positions sit inside
              large charges, the per-point bound is max(2e-6, 1.2e-7 * kappa)
              with kappa = sum of |terms| (two FP32 ulps of the sum's condition).
Sizes span several tiles and a ragged tail; the full-size realistic case runs
in the benchmark's launch configuration and is checked on sampled positions.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_1011_4687_gb300 import build_lib, esp
from workloads import (PairList, point_cells_environment, realistic_environment, small_environment,
                       tiny_pd_environment)

pytestmark = pytest.mark.gpu

FP64_REL = 1e-10
FP32_POINT = 2e-6
FP32_WALKER = 1e-5
FP32_KAPPA = 1.2e-7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build_lib.build()
    esp.load()


def check_fp64(V, ref, what=""):
    err = np.abs(V - ref)
    lim = FP64_REL * np.maximum(np.abs(ref), 1.0)
    assert np.all(err <= lim), "%s: worst %.3e (limit %.1e) at %d" % (what, err.max(), FP64_REL, int(np.argmax(err / lim)))


# points of the kappa-bounded cases beyond the flat 2e-6 bound, reported in
# the terminal summary (tests/conftest.py): [cases, points, beyond, worst err]
KAPPA_STATS = [0, 0, 0, 0.0]


def check_fp32(V, ref, what="", kappa=None):
    err = np.abs(V - ref)
    lim = FP32_POINT if kappa is None else np.maximum(FP32_POINT, FP32_KAPPA * kappa)
    if kappa is not None:
        KAPPA_STATS[0] += 1
        KAPPA_STATS[1] += int(err.size)
        KAPPA_STATS[2] += int(np.count_nonzero(err > FP32_POINT))
        KAPPA_STATS[3] = max(KAPPA_STATS[3], float(err.max()) if err.size else 0.0)
    assert np.all(err <= lim), "%s: worst per-point error %.3e Ha" % (what, err.max())


def env_of(wl, precision, **kw):
    return esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision=precision,
                           qm_center=wl.qm_center, **kw)


@functools.lru_cache(maxsize=None)
def small():
    return small_environment()


@functools.lru_cache(maxsize=None)
def small_ref():
    wl = small()
    return oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)


# ---------------------------------------------------------------------------
# small environment (point nuclei + s-Gaussian charges), every position
# ---------------------------------------------------------------------------
def test_small_environment_fp64_all_points():
    wl = small()
    with env_of(wl, "fp64") as env:
        V, E = env.eval_walkers(wl.positions, wl.n_walkers, wl.n_elec)
    check_fp64(V, small_ref(), "small fp64")
    Eref = oracle.walker_energies(small_ref(), wl.n_walkers, wl.n_elec)
    assert np.allclose(E, Eref, rtol=1e-10, atol=1e-9)


def test_small_environment_fp32c_all_points():
    wl = small()
    with env_of(wl, "fp32c") as env:
        V, E = env.eval_walkers(wl.positions, wl.n_walkers, wl.n_elec)
    check_fp32(V, small_ref(), "small fp32c")
    Eref = oracle.walker_energies(small_ref(), wl.n_walkers, wl.n_elec)
    assert np.abs(E - Eref).max() <= FP32_WALKER


# ---------------------------------------------------------------------------
# p/d environments: ragged sizes, tile sizes, launch shapes
# ---------------------------------------------------------------------------
SHAPES = [dict(), dict(tile_size=64, pair_splits=1), dict(tile_size=256, pair_splits=3),
          dict(threads_per_block=256, positions_per_thread=2), dict(threads_per_block=64, positions_per_thread=4)]


@pytest.mark.parametrize("n_pos", [1, 31, 33, 257, 1000])
@pytest.mark.parametrize("shape", range(len(SHAPES)))
def test_pd_environment_ragged(n_pos, shape):
    wl = tiny_pd_environment(500 + n_pos, n_pairs=700, n_nuclei=40, n_pos=n_pos, exp_range=(0.1, 80.0),
                             spread=3.0, pos_radius=4.0)
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    kappa = oracle.abs_terms(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    kw = dict(SHAPES[shape])
    for prec in ("fp64", "fp32c"):
        with env_of(wl, prec, screen_tol=0.0, **kw) as env:
            V = env.eval(wl.positions)
        if prec == "fp64":
            check_fp64(V, ref, "fp64 n=%d %s" % (n_pos, kw))
        else:
            check_fp32(V, ref, "fp32c n=%d %s" % (n_pos, kw), kappa)


# ---------------------------------------------------------------------------
# realistic environment, reduced: every position
# ---------------------------------------------------------------------------
@functools.lru_cache(maxsize=None)
def realistic_small():
    wl = realistic_environment(seed=7711, n_atoms=200, n_walkers=8, n_elec=32)
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    return wl, ref


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_realistic_reduced_all_points(prec):
    wl, ref = realistic_small()
    with env_of(wl, prec) as env:
        info = env.info()
        assert info["n_by_L"][4] > 0 and info["n_by_L"][0] > 0
        V, E = env.eval_walkers(wl.positions, wl.n_walkers, wl.n_elec)
    Eref = oracle.walker_energies(ref, wl.n_walkers, wl.n_elec)
    if prec == "fp64":
        check_fp64(V, ref, "realistic-200 fp64")
        assert np.allclose(E, Eref, rtol=1e-10, atol=1e-9)
    else:
        check_fp32(V, ref, "realistic-200 fp32c")
        assert np.abs(E - Eref).max() <= FP32_WALKER


# ---------------------------------------------------------------------------
# realistic environment at full size (2,000 atoms, 131,072 positions), sampled
# ---------------------------------------------------------------------------
@functools.lru_cache(maxsize=None)
def realistic_full():
    return realistic_environment()


def test_realistic_full_size_sampled():
    wl = realistic_full()
    torch = pytest.importorskip("torch")
    # two whole walkers and the 32 positions closest to the environment
    r = np.linalg.norm(wl.positions, axis=1)
    outer = np.argsort(-r)[:32]
    wsel = [0, wl.n_walkers - 1]
    sample = np.concatenate([np.arange(w * wl.n_elec, (w + 1) * wl.n_elec) for w in wsel] + [outer])
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions[sample])
    pos = torch.from_numpy(wl.positions).cuda()
    out = {}
    for prec in ("fp32c", "fp64"):
        with env_of(wl, prec) as env:
            if prec == "fp64":
                V = env.eval(torch.from_numpy(wl.positions[sample]).cuda())
                env.synchronize()
                out[prec] = V.cpu().numpy()
            else:
                V, E = env.eval_walkers(pos, wl.n_walkers, wl.n_elec)
                env.synchronize()
                out[prec] = V.cpu().numpy()[sample]
                Ew = E.cpu().numpy()[wsel]
    check_fp64(out["fp64"], ref, "realistic-2000 fp64")
    check_fp32(out["fp32c"], ref, "realistic-2000 fp32c")
    Eref = oracle.walker_energies(ref[:2 * wl.n_elec], 2, wl.n_elec)
    assert np.abs(Ew - Eref).max() <= FP32_WALKER


# ---------------------------------------------------------------------------
# the paper's literal workload: point cells + nuclei, a few positions per call
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n_pos", [1, 7, 16, 17, 64, 128, 129])
def test_point_cells(n_pos):
    """The paper's cells (small charges, summed in compensated FP32 under
    FP32C) and nuclei (FP64): FP64 at 1e-10 relative, FP32C at 2e-6 Ha per
    point, through the few-position path (n <= 128) and the main path."""
    wl = point_cells_environment(1234 + n_pos, n_cells=20000, n_nuclei=36, n_positions=n_pos)
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    for prec in ("fp64", "fp32c"):
        with env_of(wl, prec) as env:
            V = env.eval(wl.positions)
            if prec == "fp64":
                check_fp64(V, ref, "cells fp64")
            else:
                check_fp32(V, ref, "cells fp32c")
    # every point charge in FP64 (threshold 0): the FP64 accuracy again
    with env_of(wl, "fp32c", point32_max_charge=0.0) as env:
        check_fp64(env.eval(wl.positions), ref, "cells, all FP64 points")


def test_point_cells_graph_replay():
    """The captured few-position call: replays equal direct calls, and new
    positions written into the buffer between replays are picked up."""
    torch = pytest.importorskip("torch")
    wl = point_cells_environment(4321, n_cells=50000, n_nuclei=36, n_positions=256)
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    stream = torch.cuda.current_stream()
    with env_of(wl, "fp32c", stream=stream.cuda_stream) as env:
        for n in (1, 16, 128):
            buf = torch.from_numpy(wl.positions[:n].copy()).cuda()
            out = torch.empty(n, dtype=torch.float64, device="cuda")
            with esp.Graph(env, buf, out) as g:
                g.launch()
                stream.synchronize()
                direct = env.eval(buf)
                stream.synchronize()
                assert torch.equal(out, direct)
                check_fp32(out.cpu().numpy(), ref[:n], "graph n=%d" % n)
                buf.copy_(torch.from_numpy(wl.positions[128:128 + n].copy()))
                g.launch()
                stream.synchronize()
                check_fp32(out.cpu().numpy(), ref[128:128 + n], "graph n=%d, second buffer" % n)


# ---------------------------------------------------------------------------
# few positions per call (<= 16: entries spread over threads, FP64 throughout)
# against the oracle, on every class of distribution; 17 takes the main path
# ---------------------------------------------------------------------------
@functools.lru_cache(maxsize=None)
def few_env():
    return realistic_environment(seed=2718, n_atoms=40, n_walkers=1, n_elec=17)


@pytest.mark.parametrize("n_pos", [1, 5, 16, 17])
def test_few_positions_all_classes(n_pos):
    wl = few_env()
    pos = wl.positions[:n_pos]
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, pos)
    for prec in ("fp64", "fp32c"):
        with env_of(wl, prec) as env:
            assert min(env.info()["n_by_L"]) > 0  # every L class present
            V = env.eval(pos)
            # (FP32C sums small point charges in compensated FP32 on every path)
            if prec == "fp64":
                check_fp64(V, ref, "few %d %s" % (n_pos, prec))
            else:
                check_fp32(V, ref, "few %d %s" % (n_pos, prec))
            # the same positions inside a larger call agree within the path's tolerance
            Vbig = env.eval(np.concatenate([pos, wl.positions[:1].repeat(40, 0)]))[:n_pos]
            assert np.abs(Vbig - V).max() <= (1e-10 * np.abs(ref).max() if prec == "fp64" else FP32_POINT)
            # walker energies through the same path
            Vw, Ew = env.eval_walkers(pos, 1, n_pos)
            assert np.array_equal(Vw, V)
            assert abs(Ew[0] + V.sum()) <= 1e-9 * max(1.0, np.abs(V).sum())


# ---------------------------------------------------------------------------
# FP32C calls of >= 4096 positions are staged in spatial order: results come
# back in input order, repeat bitwise, and follow a permutation of the input
# ---------------------------------------------------------------------------
def test_spatial_order_is_invisible():
    wl = few_env()
    rng = np.random.default_rng(31)
    pos = realistic_environment(seed=2718, n_atoms=40, n_walkers=160, n_elec=32).positions  # 5,120 positions
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, pos)
    with env_of(wl, "fp32c") as env:
        V = env.eval(pos)
        check_fp32(V, ref, "ordered fp32c")
        assert np.array_equal(env.eval(pos), V)
        p = rng.permutation(pos.shape[0])
        Vp = env.eval(pos[p])
        assert np.abs(Vp - V[p]).max() <= FP32_POINT
        Vw, Ew = env.eval_walkers(pos, 160, 32)
        assert np.array_equal(Vw, V)
        assert np.allclose(Ew, -V.reshape(160, 32).sum(1), rtol=1e-12, atol=1e-9)


# ---------------------------------------------------------------------------
# API behaviour on the device
# ---------------------------------------------------------------------------
def test_host_and_device_pointers_agree_and_repeat_bitwise():
    torch = pytest.importorskip("torch")
    wl = tiny_pd_environment(42, n_pairs=300, n_nuclei=20, n_pos=777, spread=3.0)  # bitwise checks only
    for prec in ("fp64", "fp32c"):
        with env_of(wl, prec) as env:
            Vh = env.eval(wl.positions)
            Vd = env.eval(torch.from_numpy(wl.positions).cuda())
            env.synchronize()
            Vh2 = env.eval(wl.positions)
        assert np.array_equal(Vh, Vd.cpu().numpy())
        assert np.array_equal(Vh, Vh2)


def test_empty_and_degenerate_inputs():
    wl = tiny_pd_environment(8, n_pairs=10, n_nuclei=3, n_pos=5)
    with env_of(wl, "fp32c") as env:
        assert env.eval(np.zeros((0, 3))).shape == (0,)
        V, E = env.eval_walkers(np.zeros((0, 3)), 4, 0)
        assert np.array_equal(E, np.zeros(4))
    # only point charges
    only_nuc = tiny_pd_environment(9, n_pairs=0, n_nuclei=5, n_pos=9)
    only_nuc.pairs = PairList.empty()
    ref = oracle.potential(only_nuc.nuclei_xyz, only_nuc.nuclei_Z, only_nuc.pairs, only_nuc.positions)
    with env_of(only_nuc, "fp32c") as env:
        check_fp64(env.eval(only_nuc.positions), ref, "only nuclei")
    # only pairs, and a position exactly at a Gaussian centre (finite potential)
    only_pairs = tiny_pd_environment(10, n_pairs=20, n_nuclei=0, n_pos=4)
    only_pairs.positions[0] = only_pairs.pairs.A[0]
    ref = oracle.potential(np.zeros((0, 3)), np.zeros(0), only_pairs.pairs, only_pairs.positions)
    with env_of(only_pairs, "fp64") as env:
        check_fp64(env.eval(only_pairs.positions), ref, "only pairs")
    # an environment with nothing in it
    with esp.Environment(np.zeros((0, 3)), np.zeros(0), PairList.empty()) as env:
        assert np.array_equal(env.eval(np.ones((3, 3))), np.zeros(3))


def test_memory_space_mismatch_rejected():
    torch = pytest.importorskip("torch")
    wl = tiny_pd_environment(11, n_pairs=5, n_nuclei=2, n_pos=4)
    kappa = oracle.abs_terms(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    with env_of(wl, "fp32c") as env:
        with pytest.raises(esp.EspError) as ei:
            env.eval(torch.from_numpy(wl.positions).cuda(), out=np.zeros(4))
        assert ei.value.status == esp.ESP_ERR_INVALID
        # the context stays usable
        ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
        check_fp32(env.eval(wl.positions), ref, "after error", kappa)


def test_precision_switch_and_timing():
    wl = tiny_pd_environment(12, n_pairs=200, n_nuclei=10, n_pos=300, spread=3.0)
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    kappa = oracle.abs_terms(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    with env_of(wl, "fp32c") as env:
        env.set_timing(True)
        check_fp32(env.eval(wl.positions), ref, "timing", kappa)
        k, t = env.last_timing()
        assert 0.0 < k <= t
        env.set_precision("fp64")
        check_fp64(env.eval(wl.positions), ref)


def test_fp64_near_path_when_enabled():
    """With a positive near_radius, (position, tile) blocks closer than it are
    evaluated in FP64 inside the FP32C kernel; the result stays within the FP32C
    bounds and moves toward the FP64 value."""
    wl, ref = realistic_small()
    with env_of(wl, "fp32c", near_radius=2.0) as env:
        V, E = env.eval_walkers(wl.positions, wl.n_walkers, wl.n_elec)
    check_fp32(V, ref, "near 2.0")
    assert np.abs(E - oracle.walker_energies(ref, wl.n_walkers, wl.n_elec)).max() <= FP32_WALKER


# ---------------------------------------------------------------------------
# the paper's coalescing study: both thread mappings compute the same sum
# ---------------------------------------------------------------------------
def test_coalescing_study_mappings_agree_with_oracle():
    wl = point_cells_environment(999, n_cells=30000, n_nuclei=36, n_positions=2)
    ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    with env_of(wl, "fp32c") as env:
        for k in range(2):
            for inco in (False, True):
                for soa in (False, True):
                    v64, ms = env.study_cell_sum(wl.positions[k], inco, True, n_loop=9, reps=2, soa=soa)
                    assert abs(v64 - ref[k]) <= FP64_REL * max(abs(ref[k]), 1.0) and ms > 0
                    v32, _ = env.study_cell_sum(wl.positions[k], inco, False, n_loop=9, reps=2, soa=soa)
                    assert abs(v32 - ref[k]) <= 1e-5  # plain FP32 terms, FP64 sums
