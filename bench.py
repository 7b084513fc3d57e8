"""Benchmark: Gaussian pair x point potential evaluations per second.

One step = one esp_eval_walkers call over one batch of walker positions (all
of the path: spatial ordering and staging, the potential kernel over every
distribution and point charge, the partial-sum reduction, the per-walker
energy reduction).

Workload (default): the realistic environment, 2,000 atoms on a jittered
2.8 bohr lattice outside the 6 bohr QM sphere with cc-pVDZ-shaped primitives
and a local PSD density (~1.1e6 Hermite distributions after screening at
1e-12) plus 2,000 nuclei, evaluated at 4,096 walkers x 32 electrons = 131,072
positions per GPU per step.  One eval = one distribution (or point charge) x
one position.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank evaluates its own walkers against the same
environment (weak scaling, no collective on the data path); rank 0 prints one
JSON line.  `--impl reference` times the FP64 CPU oracle on this host's cores
on a bounded sample of the same workload.

Besides the step, the line carries (rank 0): the FP64 rate on 256 walkers,
the accuracy of both precisions against the oracle on sampled positions, the
oracle's own rate (cpu_baseline), the batched leg (64 uneven systems in one
persistent graph-replayed batch vs separate calls), the few-positions-per-call
leg (the paper's 268,782 cells, one and 16 positions per call), and the
surrogate leg (training time, evaluation with fallback vs the exact sum,
network-only time and errors).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gaussian pair×point potential evals/s at ≤1e-5 Ha: FP64 vs FP32 vs surrogate"

# FP32 operations per evaluation by total angular momentum L (offset 3,
# |r|^2 3, scaled offset 3, T 1-3, Boys 2+2L, Hermite recursion and
# contraction, accumulate 1).  MUFU work (one rsqrt) is not counted.
OPS_PER_EVAL = {0: 10, 1: 26, 2: 52, 3: 95, 4: 170}
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def keep_heap():
    try:
        import ctypes
        libc = ctypes.CDLL("libc.so.6")
        libc.mallopt(-4, 0)
        libc.mallopt(-1, 1 << 30)
    except (OSError, AttributeError):
        pass


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("esp_potential.cuh", "esp_shape.cu", "esp_internal.h", "esp_eval_core.h"):
        with open(os.path.join(ROOT, "paper_1011_4687_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, n_pos: int):
    """DRAM bytes of one launch, from the committed ncu counters of a launch of
    this size; None if the size differs or the kernel source changed since
    the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        t = json.load(f)
    e = t.get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash() or e.get("positions") != n_pos:
        return None
    return e["dram_bytes"]


def workload_label(wl, large: bool = False, reduced: bool = False) -> str:
    """The workload as both arms of the benchmark name it."""
    return (("REDUCED (profiling) " if reduced else "") +
            ("large: 20,000 atoms" if large else "realistic: 2,000 atoms") +
            ", cc-pVDZ-shaped primitives, local PSD density, %d positions (%d walkers x %d electrons) per GPU"
            % (wl.n_walkers * wl.n_elec, wl.n_walkers, wl.n_elec))


def replica_positions(rank: int, n: int) -> np.ndarray:
    """The walkers of rank > 0 under torchrun: the same law, a seed of the rank's
    own (rank 0 keeps the workload's positions)."""
    from workloads import seed_for_config, qm_positions
    return qm_positions(np.random.default_rng(seed_for_config(2) * 1000 + rank), n)


def max_over_ranks(ms: float, world: int, device: str) -> float:
    """The slowest rank's step time (every rank returns it)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def build_workload(rank: int, walkers: int = 4096, large: bool = False):
    from workloads import realistic_environment, seed_for_config, qm_positions
    if large:
        # 20,000 atoms on a 28^3 lattice (same per-atom law), 16,384 walkers x 64 electrons
        wl = realistic_environment(seed=seed_for_config(5), n_atoms=20000, n_walkers=16384, n_elec=64, n_side=28)
    else:
        wl = realistic_environment(seed=seed_for_config(2))
    if rank > 0:
        wl.positions = replica_positions(rank, wl.n_walkers * wl.n_elec)
    if walkers != wl.n_walkers:
        wl.positions = wl.positions[: walkers * wl.n_elec].copy()
        wl.n_walkers = walkers
    return wl


def sample_indices(wl, n_walkers=2, n_outer=32):
    """Whole walkers (the first and the last) and the positions closest to the environment."""
    r = np.linalg.norm(wl.positions, axis=1)
    outer = np.argsort(-r)[:n_outer]
    ws = [0, wl.n_walkers - 1][:n_walkers]
    return ws, np.concatenate([np.arange(w * wl.n_elec, (w + 1) * wl.n_elec) for w in ws] + [outer])


def _gen_batched(n_sys):
    """The batched workload's systems, generated in a spawn-started process
    pool (numpy only; no CUDA in the workers)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from workloads import batched_specs, batched_system
    specs = batched_specs(n_sys=n_sys)
    order = sorted(range(len(specs)), key=lambda k: -specs[k]["n_atoms"])
    out = [None] * len(specs)
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        futs = {ex.submit(batched_system, specs[k]): k for k in order}
        for f in cf.as_completed(futs):
            out[futs[f]] = f.result()
    return out


def batch_leg(args, esp, torch, stream, flush, wls, oracle_mod=None):
    """Many uneven systems in one persistent, graph-replayed batch (tuned
    launch shape) against the same systems evaluated one esp_eval at a time."""
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=8) as ex:  # the pair builder runs outside the GIL
        envs = list(ex.map(lambda w: esp.Environment(w.nuclei_xyz, w.nuclei_Z, w.pairs, precision="fp32c",
                                                     stream=stream.cuda_stream), wls))
    pos = [torch.from_numpy(w.positions.reshape(-1, 3)).cuda() for w in wls]
    outs = [torch.empty(int(p.shape[0]), dtype=torch.float64, device="cuda") for p in pos]
    units = [e.info()["n_distributions"] + e.info()["n_point_charges"] for e in envs]
    evals = sum(u * int(p.shape[0]) for u, p in zip(units, pos))
    b = esp.Batch(envs, stream=stream.cuda_stream)
    tune = b.autotune(pos, outs)

    def timed(fn, k):
        ts = []
        for _ in range(k):
            flush.zero_()
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            fn()
            s1.record(stream)
            s1.synchronize()
            ts.append(s0.elapsed_time(s1))
        return statistics.mean(ts)

    def singles():
        for e, p, o in zip(envs, pos, outs):
            e.eval(p, out=o) if p.shape[0] else None

    for _ in range(max(1, args.warmup)):
        b.eval(pos, outs)
        singles()
    torch.cuda.synchronize()
    k = max(1, min(args.steps, 3))
    ms_b = timed(lambda: b.eval(pos, outs), k)
    ms_s = timed(singles, k)
    acc = None
    if oracle_mod is not None:
        # per-system error of the batched result against the FP64 oracle:
        # the first and the last position of every system
        b.eval(pos, outs)
        torch.cuda.synchronize()
        worst = 0.0
        for w, o in zip(wls, outs):
            if w.positions.shape[0] == 0:
                continue
            pick = np.array([0, w.positions.shape[0] - 1])
            ref = oracle_mod.potential(w.nuclei_xyz, w.nuclei_Z, w.pairs, w.positions.reshape(-1, 3)[pick])
            worst = max(worst, float(np.abs(o.cpu().numpy()[pick] - ref).max()))
        acc = {"sample": "first and last position of each of the %d systems vs the FP64 oracle" % len(wls),
               "max_point_err_ha": worst}
    res = {"workload": "%d systems, %d-%d distributions, %d-%d positions (log-uniform sizes)"
                       % (len(wls), min(units), max(units), min(int(p.shape[0]) for p in pos),
                          max(int(p.shape[0]) for p in pos)),
           "value": evals / (ms_b * 1e-3), "unit": "evals/s", "ms_per_step": ms_b,
           "evals_per_step": evals, "separate_evals_ms": ms_s, "speedup_vs_separate": ms_s / ms_b,
           "tuned_shape": {k2: tune[k2] for k2 in ("threads_per_block", "positions_per_thread", "split_scale")},
           "gpu_launches_per_step": 3}
    if acc is not None:
        res["accuracy"] = acc
    b.close()
    for e in envs:
        e.close()
    return res


def surrogate_leg(args, esp, torch, stream, flush, oracle_mod):
    """The learned surrogate with exact fallback on the small environment
    (200 nuclei + 2,000 s-charges), trained with the library defaults (2^22
    positions labelled by the exact kernel), evaluated at 131,072 positions per
    step, against the exact FP32C sum of the same positions."""
    from workloads import qm_positions, seed_for_config, small_environment
    wl = small_environment(seed=seed_for_config(1))
    env = esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision="fp32c", stream=stream.cuda_stream)
    units = env.info()["n_distributions"] + env.info()["n_point_charges"]
    t0 = time.perf_counter()
    sur = esp.Surrogate(env)
    t_train = time.perf_counter() - t0
    n = 131072
    pos_np = qm_positions(np.random.default_rng(seed_for_config(4)), n)
    pos = torch.from_numpy(pos_np).cuda()
    Vs = torch.empty(n, dtype=torch.float64, device="cuda")
    Vx = torch.empty(n, dtype=torch.float64, device="cuda")
    for _ in range(max(1, args.warmup)):
        sur.eval(pos, Vs)
        env.eval(pos, out=Vx)
    torch.cuda.synchronize()
    ts, tx, fb = [], [], []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        _, st = sur.eval(pos, Vs)
        ts.append(time.perf_counter() - t1)
        fb.append(st["n_fallback"])
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        env.eval(pos, out=Vx)
        torch.cuda.synchronize()
        tx.append(time.perf_counter() - t1)
    ms_s, ms_x = statistics.mean(ts) * 1e3, statistics.mean(tx) * 1e3
    # the network + baseline alone (no fallback): one fused tensor-core launch
    Vp = torch.empty(n, dtype=torch.float64, device="cuda")
    sur.predict(pos, Vp)
    tp = []
    for _ in range(args.steps):
        flush.zero_()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        sur.predict(pos, Vp)
        s1.record(stream)
        s1.synchronize()
        tp.append(s0.elapsed_time(s1))
    ms_p = statistics.mean(tp)
    info = sur.info()
    res = {"workload": "small environment (%d point charges + %d s-charges), %d positions per step"
                       % (wl.nuclei_Z.size, env.info()["n_distributions"], n),
           "value": units * n / (ms_s * 1e-3), "unit": "equivalent evals/s", "ms_per_step": ms_s,
           "exact_fp32c_ms": ms_x, "speedup_vs_exact_fp32c": ms_x / ms_s,
           "fallback_fraction": statistics.mean(fb) / n, "train_s": t_train,
           "valid_rms_err_ha": info["valid_rms_err"], "baseline_only_rms_err_ha": info["baseline_rms_err"],
           "trusted_voxel_fraction": info["trusted_fraction"],
           "predict_only_ms": ms_p, "predict_only_positions_per_s": n / (ms_p * 1e-3),
           "predict_only_tflops": n * 2.0 * (64 * 256 + 3 * 256 * 256 + 256) / (ms_p * 1e-3) / 1e12,
           "inference": "one fused tcgen05 kernel per call (BF16 x BF16 -> FP32 in TMEM); training GEMMs mma.sync"}
    if oracle_mod is not None:
        m = 64 * 32  # 64 whole walkers of 32 electrons
        ref = oracle_mod.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, pos_np[:m])
        got = Vs[:m].cpu().numpy()
        res["predict_only_rms_err_ha"] = float(np.sqrt(np.mean((Vp[:m].cpu().numpy() - ref) ** 2)))
        Eg = -got.reshape(64, 32).sum(1)
        Er = oracle_mod.walker_energies(ref, 64, 32)
        res["accuracy"] = {"sample": "64 walkers x 32 electrons vs the FP64 oracle",
                           "max_point_err_ha": float(np.abs(got - ref).max()),
                           "max_walker_err_ha": float(np.abs(Eg - Er).max())}
    sur.close()
    env.close()
    return res


def latency_leg(args, esp, torch, stream):
    """The paper's own call pattern: its cell count (268,782 point cells +
    36 nuclei) evaluated at one position per call (one Metropolis move), and at
    16 per call; microseconds per call on the device (CUDA events, device
    buffers) and through host buffers (wall clock, copies included)."""
    from workloads import point_cells_environment
    wl = point_cells_environment(seed=1011 * 100 + 6, n_cells=268782, n_nuclei=36, n_positions=16)
    env = esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision="fp32c", stream=stream.cuda_stream)
    units = env.info()["n_point_charges"]
    out = {"workload": "%d point charges (268,782 cells + 36 nuclei)" % units}
    reps = 200
    for npos in (1, 16):
        pos = torch.from_numpy(wl.positions[:npos].copy()).cuda()
        V = torch.empty(npos, dtype=torch.float64, device="cuda")
        for _ in range(10):
            env.eval(pos, out=V)
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(reps):
            env.eval(pos, out=V)
        s1.record(stream)
        s1.synchronize()
        us = s0.elapsed_time(s1) * 1e3 / reps
        hp = wl.positions[:npos].copy()
        hv = np.zeros(npos)
        t0 = time.perf_counter()
        for _ in range(reps):
            env.eval(hp, out=hv)
        us_host = (time.perf_counter() - t0) * 1e6 / reps
        out["positions_%d" % npos] = {"us_per_call": us, "us_per_call_host_buffers": us_host,
                                      "evals_per_s": units * npos / (us * 1e-6), "launches_per_call": 2}
    env.close()
    return out


def run_reference(args):
    """The oracle as it stands, on this host's cores, bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    wl = build_workload(0)
    n_units = (wl.meta["n_shell_pairs"] + wl.nuclei_Z.size)
    sample = np.arange(args.ref_positions)
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions[sample])
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    per = statistics.mean(times)
    val = n_units * sample.size / per
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_label(wl), "distributions": wl.meta["n_shell_pairs"],
                       "point_charges": int(wl.nuclei_Z.size), "oracle_positions_per_step": int(sample.size)},
            "cpu_baseline": {"value": val, "unit": "evals/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": "%d positions of the realistic workload per step (all distributions)"
                                       % sample.size},
            "e2e": {"value": val, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-walkers", type=int, default=256, help="walkers in the FP64 rate measurement")
    ap.add_argument("--ref-positions", type=int, default=32, help="positions per oracle step (reference arm)")
    ap.add_argument("--no-oracle", action="store_true", help="skip the accuracy check and CPU baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-systems leg")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate leg")
    ap.add_argument("--no-latency", action="store_true", help="skip the one-position-per-call leg")
    ap.add_argument("--batch-systems", type=int, default=64, help="systems in the batched leg")
    ap.add_argument("--walkers", type=int, default=4096,
                    help="walkers of 32 electrons per GPU (the benchmark workload is 4096; fewer only for profiling)")
    ap.add_argument("--large", action="store_true",
                    help="the large configuration instead: 20,000 atoms, 16,384 walkers x 64 electrons")
    args = ap.parse_args(argv)
    keep_heap()
    if args.impl == "reference":
        return run_reference(args)

    # the batched leg's systems come from a spawn-started pool, before any CUDA call
    batch_wls = None
    if not args.no_batch and int(os.environ.get("RANK", "0")) == 0:
        batch_wls = _gen_batched(args.batch_systems)

    import torch
    import torch.distributed as dist
    from paper_1011_4687_gb300 import build_lib, esp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        build_lib.build()
    if world > 1:
        dist.barrier()
    esp.load()

    if args.large:
        args.walkers = 16384
    wl = build_workload(rank, args.walkers, large=args.large)
    stream = torch.cuda.current_stream()
    env = esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision="fp32c", stream=stream.cuda_stream)
    info = env.info()
    n_pos = wl.n_positions
    units_per_pos = info["n_distributions"] + info["n_point_charges"]
    evals_per_step = units_per_pos * n_pos
    pos = torch.from_numpy(wl.positions).cuda()
    V = torch.empty(n_pos, dtype=torch.float64, device="cuda")
    E = torch.empty(wl.n_walkers, dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    env.set_timing(True)
    for _ in range(args.warmup):
        env.eval_walkers(pos, wl.n_walkers, wl.n_elec, V_out=V, E_out=E)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kern_ms = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            env.eval_walkers(pos, wl.n_walkers, wl.n_elec, V_out=V, E_out=E)
            ends[k].record(stream)
            kern_ms.append(env.last_timing()[0])
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = statistics.mean(step_ms)
    ms_max = max_over_ranks(ms, world, "cuda")
    value = evals_per_step * world / (ms_max * 1e-3)
    kern = statistics.mean(kern_ms)
    clocks = clk.summary()

    # end to end through the public API with pinned host buffers
    pin_pos = torch.from_numpy(wl.positions).pin_memory()
    pin_V = torch.empty(n_pos, dtype=torch.float64).pin_memory()
    pin_E = torch.empty(wl.n_walkers, dtype=torch.float64).pin_memory()
    hp, hv, he = pin_pos.numpy(), pin_V.numpy(), pin_E.numpy()
    env.eval_walkers(hp, wl.n_walkers, wl.n_elec, V_out=hv, E_out=he)
    e2e_t = []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        env.eval_walkers(hp, wl.n_walkers, wl.n_elec, V_out=hv, E_out=he)
        e2e_t.append(time.perf_counter() - t0)
    e2e_val = evals_per_step * world / statistics.mean(e2e_t)

    # FP64 rate on a subset of walkers (same environment, same kernels' FP64 variant)
    nw64 = min(args.fp64_walkers, wl.n_walkers)
    pos64 = pos[: nw64 * wl.n_elec].contiguous()
    env.set_precision("fp64")
    env.eval_walkers(pos64, nw64, wl.n_elec)
    torch.cuda.synchronize()
    f64 = []
    for _ in range(2):
        flush.zero_()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        env.eval_walkers(pos64, nw64, wl.n_elec)
        s1.record(stream)
        s1.synchronize()
        f64.append(s0.elapsed_time(s1))
    fp64_val = units_per_pos * nw64 * wl.n_elec / (statistics.mean(f64) * 1e-3)
    env.set_precision("fp32c")

    if rank != 0:
        env.close()
        if world > 1:
            dist.destroy_process_group()
        return 0

    # roofline of the potential kernel (FP32 issue bound)
    peaks, peak_src = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = SM_COUNT * FP32_LANES_PER_SM * sm_mhz * 1e6
    ops_launch = n_pos * sum(OPS_PER_EVAL[L] * info["n_by_L"][L] for L in range(5))
    achieved = ops_launch / (kern * 1e-3)
    traffic = profiled_traffic("potential_f32c_kernel", n_pos)

    out = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": workload_label(wl, args.large, not args.large and args.walkers != 4096),
                      "distributions": info["n_distributions"], "point_charges": info["n_point_charges"],
                      "precision": "FP32C (FP32 pair sum, compensated; nuclei and near blocks FP64)",
                      "distributions_by_L": info["n_by_L"], "evals_per_step_per_gpu": evals_per_step,
                      "l2": "flushed between timed steps (512 MB write)", "parallelism": "replicas" if world > 1 else "single"},
           # per step: spatial order (3 launches, FP32C calls of >= 4,096 positions), stage, potential,
           # reduce, walker energies
           "gpu_launches": (7 if n_pos >= 4096 else 4) * args.steps,
           "clocks": clocks,
           "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                        "unit": "Tops/s (FP32 lane ops)", "frac": achieved / peak_ops, "traffic": traffic,
                        "kernel": "potential_f32c_kernel", "kernel_ms": kern,
                        "peak_source": "152 SMs x 128 FP32 lanes x %.0f MHz (%s sm_max_mhz)" % (sm_mhz, peak_src)},
           "e2e": {"value": e2e_val, "unit": "evals/s", "h2d_bytes_per_step": int(n_pos * 24),
                   "d2h_bytes_per_step": int(n_pos * 8 + wl.n_walkers * 8)},
           "fp64": {"value": fp64_val, "unit": "evals/s", "positions_per_step": nw64 * wl.n_elec,
                    "ms_per_step": statistics.mean(f64)}}

    if not args.no_oracle:
        import oracle
        oracle.build()
        nws, nout = (1, 16) if args.large else (2, 32)
        ws, sample = sample_indices(wl, nws, nout)
        t0 = time.perf_counter()
        ref = oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions[sample])
        t_or = time.perf_counter() - t0
        Vs = V.cpu().numpy()[sample]
        Es = E.cpu().numpy()[ws]
        Eref = oracle.walker_energies(ref[: nws * wl.n_elec], nws, wl.n_elec)
        env.set_precision("fp64")
        V64 = env.eval(torch.from_numpy(wl.positions[sample]).cuda())
        torch.cuda.synchronize()
        V64 = V64.cpu().numpy()
        out["accuracy"] = {"sample": "%d whole walker(s) + %d outermost positions" % (nws, nout),
                           "fp32c_max_point_err_ha": float(np.abs(Vs - ref).max()),
                           "fp32c_max_walker_err_ha": float(np.abs(Es - Eref).max()),
                           "fp64_max_rel_err": float(np.max(np.abs(V64 - ref) / np.maximum(np.abs(ref), 1.0)))}
        out["cpu_baseline"] = {"value": units_per_pos * sample.size / t_or, "unit": "evals/s",
                               "cores": oracle.max_threads(), "kind": "oracle",
                               "sample": "%d positions x all %d distributions + point charges"
                                         % (sample.size, units_per_pos)}
    env.close()
    if batch_wls is not None:
        out["batch"] = batch_leg(args, esp, torch, stream, flush, batch_wls,
                                 None if args.no_oracle else __import__("oracle"))
        del batch_wls
    if not args.no_latency:
        out["few_positions_per_call"] = latency_leg(args, esp, torch, stream)
    if not args.no_surrogate:
        out["surrogate"] = surrogate_leg(args, esp, torch, stream, flush,
                                         None if args.no_oracle else __import__("oracle"))
    if not args.no_oracle:
        # the paper's framing, one CPU core (8 of the sampled positions); last,
        # because it leaves the oracle's OpenMP pool at one thread
        import oracle
        t1 = time.perf_counter()
        oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions[sample[:8]], threads=1)
        out["cpu_baseline"]["single_core_value"] = units_per_pos * 8 / (time.perf_counter() - t1)
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
