"""Benchmark: Gaussian pair x point potential evaluations per second.

One step = one esp_eval_walkers call over one batch of walker positions (all
of the path: spatial ordering and staging, the potential kernel over every
distribution and point charge, the partial-sum reduction, the per-walker
energy reduction).  One eval = one distribution (or point charge) x one
position; distributions are counted as the library builds them (after its
screening and merges), in both arms.

Workload (default `--config large`): the largest configuration, 20,000 atoms on
a jittered 2.8 bohr lattice (28^3 sites) outside the 6 bohr QM sphere with
cc-pVDZ-shaped primitives and a local PSD density (~2e7 Hermite
distributions after screening at 1e-12) plus 20,000 nuclei, evaluated at
16,384 walkers x 64 electrons = 1,048,576 positions per GPU per step.
`--config realistic` is the 2,000-atom, 131,072-position configuration, which
the default run also measures as a secondary leg.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank evaluates its own walkers against the same
environment (weak scaling, no collective on the data path); rank 0 prints one
JSON line.  `--impl reference` times the FP64 CPU oracle on this host's cores
on a bounded sample of the same workload.

Besides the step, the line carries (rank 0): the measured pipe peaks, the
census-based roofline of the FP32C kernel, the FP64 path on 16 whole walkers
with its own roofline, the accuracy of both precisions (against the oracle,
or for the large workload against the oracle-checked FP64 path), the oracle's
own rate (cpu_baseline), the realistic-configuration leg, the batched leg (64
uneven systems in one persistent graph-replayed batch vs separate calls), the
few-positions-per-call leg (the paper's 268,782 cells) and the surrogate leg.
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

# Algorithmic operation counts per term (one distribution x one position),
# written out for the McMurchie-Davidson evaluation of one term in plain
# arithmetic: no compensation (hi/lo words, Newton step, TwoSum), no loads.
# A multiply, add or fused multiply-add counts 1; the reciprocal square root
# (MUFU) counts 0 on the FP32 path and 1 on the FP64 path; erfc counts 1.
#   offset P - C                        3
#   L = 0: |d|^2 3, T = p |d|^2 1       4      (FP64: p = sqrt(p)^2, +1)
#   L > 0: x = sqrt(p) d 3, T = |x|^2 3  6
#   (FP32 asymptotic regime = multipole form on the unscaled offset: |d|^2 3 only)
#   Hermite recursion R(L), incl. the (-2)^n scaling of each level:
#                                        0, 4, 17, 46, 100 for L = 0..4
#   contraction sum G_tuv S_tuv          n_L = 1, 4, 10, 20, 35
#   accumulate                           1
# Boys F_0..F_L, by regime of T:
#   asymptotic (FP32: T >= 30, far/multipole form; FP64: T >= 45):
#       L = 0: 0 (FP32) / 1 (FP64: sqrt(pi)/2 * rsqrt);  L > 0: 1 + 2L (FP32) / 2 + 2L (FP64)
#       (h = 1/(2T), F_n = F_{n-1} (2n-1) h)
#   table (FP32: T < 30, 6 Taylor terms; FP64: T < 45, 9 terms):
#       row index and remainder 2; F_L by Horner 2 (K-1) + 1;
#       L > 0: exp(-T) by Horner 2 (K-1) + 1, 2T 1, downward recursion 2L
#   short-range remainder (monopole moved to a point charge): + 2 (erfc term)
HERMITE_REC = (0, 4, 17, 46, 100)
N_HERMITE = (1, 4, 10, 20, 35)


def term_ops(L: int, regime: str, fp64: bool, short: bool = False) -> int:
    """Operations of one term of total angular momentum L in the given Boys
    regime ("asym" or "table") on the FP32 (fp64=False) or FP64 path."""
    base = 3 + (4 + (1 if fp64 else 0) if L == 0 else 6) + HERMITE_REC[L] + N_HERMITE[L] + 1
    if regime == "asym":
        if not fp64:
            base -= 1 if L == 0 else 3  # multipole form: |d|^2 only, no T, no scaled offset
        boys = (1 if fp64 else 0) if L == 0 else (2 if fp64 else 1) + 2 * L
    else:
        K = 9 if fp64 else 6
        boys = 2 + 2 * (K - 1) + 1
        if L > 0:
            boys += 2 * (K - 1) + 1 + 1 + 2 * L
    return base + boys + (2 if short and regime == "table" else 0)


POINT_OPS_F64 = 8  # 3 sub, |d|^2 3, Z * rsqrt 1 (+ rsqrt 1 on the FP64 pipe), accumulate


def census_ops(census: dict, n_positions: int, fp64: bool):
    """(algorithmic ops of the distributions, ops of the point charges, terms)
    of one launch over n_positions, from a work census of a position sample
    (esp_work_census): FP32 takes the table below T = 30, FP64 below T = 45."""
    scale = n_positions / census["positions"]
    ops = 0.0
    terms = 0
    for s in (0, 1):
        for L in range(5):
            lt30, mid, ge45 = (census["T_lt_30"][s][L], census["T_30_45"][s][L], census["T_ge_45"][s][L])
            terms += lt30 + mid + ge45
            if fp64:
                ops += (lt30 + mid) * term_ops(L, "table", True, s == 1) + ge45 * term_ops(L, "asym", True, s == 1)
            else:
                ops += lt30 * term_ops(L, "table", False, s == 1) + (mid + ge45) * term_ops(L, "asym", False, s == 1)
    return ops * scale, census["point_terms"] * scale * POINT_OPS_F64, terms * scale


def keep_heap():
    try:
        import ctypes
        libc = ctypes.CDLL("libc.so.6")
        libc.mallopt(-4, 0)        # M_MMAP_MAX: serve large blocks from the heap
        libc.mallopt(-1, 1 << 30)  # M_TRIM_THRESHOLD: do not trim the heap
        libc.mallopt(-8, 1)        # M_ARENA_MAX: the generator's threads share one (non-trimming) arena
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


def profiled_traffic(kernel: str, n_pos: int, kind: str):
    """DRAM bytes of one launch, from the committed ncu counters of this
    workload; None if none were taken or the kernel source changed since the
    capture.  An entry holds either the bytes of a launch at this exact size
    ("positions", "dram_bytes") or, where the full launch is too long to
    capture, a line through captures at two reduced sizes ("fixed_bytes" +
    "bytes_per_position" x positions: the environment is read from DRAM about
    once, the positions' share grows with their number)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        t = json.load(f)
    e = t.get("%s/%s" % (kernel, kind))
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    if "bytes_per_position" in e:
        return e["fixed_bytes"] + e["bytes_per_position"] * n_pos
    if e.get("positions") != n_pos:
        return None
    return e["dram_bytes"]


WORKLOADS = {
    # the largest configuration: 20,000 atoms on a 28^3 lattice, 16,384 walkers x 64 electrons
    "large": dict(config=5, n_atoms=20000, n_walkers=16384, n_elec=64, n_side=28),
    # the realistic configuration: 2,000 atoms, 4,096 walkers x 32 electrons
    "realistic": dict(config=2, n_atoms=2000, n_walkers=4096, n_elec=32, n_side=None),
}


def workload_label(wl, kind: str, reduced: bool = False) -> str:
    """The workload as both arms of the benchmark name it."""
    return (("REDUCED (profiling) " if reduced else "") +
            "%s: %s atoms, cc-pVDZ-shaped primitives, local PSD density, %d positions (%d walkers x %d electrons) "
            "per GPU" % (kind, format(WORKLOADS[kind]["n_atoms"], ","), wl.n_walkers * wl.n_elec, wl.n_walkers,
                         wl.n_elec))


def replica_positions(rank: int, n: int, kind: str = "large") -> np.ndarray:
    """The walkers of rank > 0 under torchrun: the same law, a seed of the rank's
    own (rank 0 keeps the workload's positions)."""
    from workloads import seed_for_config, qm_positions
    return qm_positions(np.random.default_rng(seed_for_config(WORKLOADS[kind]["config"]) * 1000 + rank), n)


def max_over_ranks(ms: float, world: int, device: str) -> float:
    """The slowest rank's step time (every rank returns it)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def build_workload(kind: str, rank: int = 0, walkers: int = 0):
    from workloads import realistic_environment, seed_for_config
    w = WORKLOADS[kind]
    wl = realistic_environment(seed=seed_for_config(w["config"]), n_atoms=w["n_atoms"], n_walkers=w["n_walkers"],
                               n_elec=w["n_elec"], n_side=w["n_side"])
    if rank > 0:
        wl.positions = replica_positions(rank, wl.n_walkers * wl.n_elec, kind)
    if walkers and walkers != wl.n_walkers:
        wl.positions = wl.positions[: walkers * wl.n_elec].copy()
        wl.n_walkers = walkers
    return wl


def workload_config(wl, kind: str, units: dict, world: int, reduced: bool = False) -> dict:
    """config of the JSON line, identical in both arms: the workload and the
    library's unit count (Hermite distributions + point charges per position)."""
    n = wl.n_walkers * wl.n_elec
    return {"workload": workload_label(wl, kind, reduced), "distributions": int(units["n_distributions"]),
            "point_charges": int(units["n_point_charges"]), "positions_per_step": n,
            "evals_per_step_per_gpu": int((units["n_distributions"] + units["n_point_charges"]) * n),
            "l2": "inputs larger than L2 (records %s) and L2 flushed between timed steps (512 MB write)"
                  % ("~1.7 GB" if kind == "large" else "~90 MB"),
            "parallelism": "replicas (own walkers per GPU, same environment)" if world > 1 else "single GPU"}


def sample_indices(wl, n_walkers: int, n_outer: int, n_random: int, seed: int = 17):
    """Whole walkers (spread over the batch), the positions closest to the
    environment, and seeded random positions: (walker ids, position indices)."""
    r = np.linalg.norm(wl.positions, axis=1)
    outer = np.argsort(-r)[:n_outer]
    ws = np.unique(np.linspace(0, wl.n_walkers - 1, n_walkers).round().astype(int))
    walk = np.concatenate([np.arange(w * wl.n_elec, (w + 1) * wl.n_elec) for w in ws])
    rest = np.setdiff1d(np.arange(wl.n_positions), np.concatenate([walk, outer]))
    rnd = np.random.default_rng(seed).choice(rest, size=min(n_random, rest.size), replace=False)
    return ws, np.concatenate([walk, outer, np.sort(rnd)])


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


def surrogate_leg(args, env, wl, label, torch, stream, flush, exact_ms, V_exact=None, oracle_mod=None,
                  ref_fn=None, **cfg):
    """The surrogate with exact fallback on one workload: near tiles summed
    exactly, far tiles by FP64 interior expansion + BF16 network, fallback where
    untrusted, near point charges, or probed.  Timed (device, CUDA events on the
    library's stream) against the exact FP32C step of the same positions
    (exact_ms); its error against the library's FP64 path or the oracle on a
    sample (ref_fn(sample positions) -> reference values)."""
    units = env.info()["n_distributions"] + env.info()["n_point_charges"]
    n = wl.n_positions
    t0 = time.perf_counter()
    sur = esp_mod().Surrogate(env, **cfg)
    t_train = time.perf_counter() - t0
    pos = torch.from_numpy(wl.positions).cuda()
    Vs = torch.empty(n, dtype=torch.float64, device="cuda")
    for _ in range(max(1, min(args.warmup, 2))):
        sur.eval(pos, Vs)
    torch.cuda.synchronize()
    fb, ms = [], []
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        _, st = sur.eval(pos, Vs)
        s1.record(stream)
        s1.synchronize()
        ms.append(s0.elapsed_time(s1))
        fb.append(st["n_fallback"])
    ms_s = statistics.mean(ms)
    info = sur.info()
    Vp = sur.predict(pos)
    torch.cuda.synchronize()
    served = (Vs == Vp)
    res = {"workload": label, "value": units * n / (ms_s * 1e-3), "unit": "equivalent evals/s",
           "ms_per_step": ms_s, "exact_fp32c_ms_per_step": exact_ms, "speedup_vs_exact_fp32c": exact_ms / ms_s,
           "served_fraction": float(served.float().mean().item()), "fallback_fraction": statistics.mean(fb) / n,
           "near_entries": info["n_near_entries"], "far_entries": info["n_far_entries"],
           "near_share": info["n_near_entries"] / max(1, info["n_near_entries"] + info["n_far_entries"]),
           "train_s": t_train, "trusted_voxel_fraction": info["trusted_fraction"],
           "expansion_only_trusted_voxel_fraction": info["baseline_trusted_fraction"],
           "far_valid_rms_err_ha": info["valid_rms_err"], "far_valid_max_err_ha": info["valid_max_err"],
           "expansion_only_rms_err_ha": info["baseline_rms_err"],
           "expansion_only_max_err_ha": info["baseline_max_err"], "expansion_coefficients": info["n_baseline"],
           "steps": len(ms),
           "inference": "FP32C near-tile sum + FP64 solid-harmonic expansion + one fused tcgen05 network kernel; "
                        "training GEMMs on tcgen05"}
    if V_exact is not None:
        d = (Vs - V_exact).abs()
        res["max_point_diff_vs_exact_fp32c_ha"] = float(d.max().item())
    if ref_fn is not None:
        ws, sample = sample_indices(wl, 16, 256, 768)
        refv, what = ref_fn(wl.positions[sample])
        got = Vs.cpu().numpy()[sample]
        sv = served.cpu().numpy()[sample]
        nw = ws.size * wl.n_elec
        Eg = -got[:nw].reshape(ws.size, wl.n_elec).sum(1)
        Er = -refv[:nw].reshape(ws.size, wl.n_elec).sum(1)
        res["accuracy"] = {"against": what, "sample": "%d whole walkers + 256 outermost + 768 random positions"
                                                      % ws.size,
                           "max_point_err_ha": float(np.abs(got - refv).max()),
                           "max_served_point_err_ha": float(np.abs(got - refv)[sv].max()) if sv.any() else None,
                           "served_in_sample": int(sv.sum()),
                           "max_walker_err_ha": float(np.abs(Eg - Er).max())}
    sur.close()
    return res


def small_surrogate_leg(args, torch, stream, flush, oracle_mod):
    """The surrogate configuration's own environment (200 nuclei + 2,000
    s-charges in a 20 bohr cube) at 131,072 positions per step: every charge
    lies within 17 bohr of the centre, so most of the environment is near and
    summed exactly; reported for completeness."""
    from workloads import qm_positions, seed_for_config, small_environment
    wl = small_environment(seed=seed_for_config(1))
    wl.positions = qm_positions(np.random.default_rng(seed_for_config(4)), 131072)
    wl.n_walkers, wl.n_elec = 4096, 32
    env = esp_mod().Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision="fp32c", stream=stream.cuda_stream)
    pos = torch.from_numpy(wl.positions).cuda()
    Vx = torch.empty(wl.n_positions, dtype=torch.float64, device="cuda")
    exact_ms = timed_device(lambda: env.eval(pos, out=Vx), stream, flush, 3)
    ref_fn = None
    if oracle_mod is not None:
        ref_fn = lambda p: (oracle_mod.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, p), "FP64 oracle")
    res = surrogate_leg(args, env, wl, "small environment (%d point charges + %d s-charges), %d positions per step"
                        % (wl.nuclei_Z.size, len(wl.pairs), wl.n_positions), torch, stream, flush, exact_ms, Vx,
                        ref_fn=ref_fn)
    env.close()
    return res


def esp_mod():
    from paper_1011_4687_gb300 import esp
    return esp


def latency_leg(args, esp, torch, stream, oracle_mod=None):
    """The paper's own call pattern: its cell count (268,782 point cells +
    36 nuclei) evaluated at 1, 16 and 128 positions per call (one Metropolis
    move is one position): microseconds per call on the device (CUDA events,
    device buffers), replayed as a captured graph, and through host buffers
    (wall clock, copies included).  Cells are summed in compensated FP32,
    nuclei in FP64."""
    from workloads import point_cells_environment
    wl = point_cells_environment(seed=1011 * 100 + 6, n_cells=268782, n_nuclei=36, n_positions=128)
    env = esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision="fp32c", stream=stream.cuda_stream)
    units = env.info()["n_point_charges"]
    out = {"workload": "%d point charges (268,782 cells + 36 nuclei)" % units, "precision": "FP32C"}
    reps = 200
    ref = None
    if oracle_mod is not None:
        ref = oracle_mod.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions)
    for npos in (1, 16, 128):
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
        Vg = torch.empty(npos, dtype=torch.float64, device="cuda")
        with esp.Graph(env, pos, Vg) as g:
            for _ in range(10):
                g.launch()
            torch.cuda.synchronize()
            s0.record(stream)
            for _ in range(reps):
                g.launch()
            s1.record(stream)
            s1.synchronize()
            us_graph = s0.elapsed_time(s1) * 1e3 / reps
        hp = wl.positions[:npos].copy()
        hv = np.zeros(npos)
        t0 = time.perf_counter()
        for _ in range(reps):
            env.eval(hp, out=hv)
        us_host = (time.perf_counter() - t0) * 1e6 / reps
        leg = {"us_per_call": us, "us_per_call_graph_replay": us_graph, "us_per_call_host_buffers": us_host,
               "evals_per_s": units * npos / (us * 1e-6), "launches_per_call": 2}
        if ref is not None:
            leg["max_point_err_ha"] = float(np.abs(Vg.cpu().numpy() - ref[:npos]).max())
        out["positions_%d" % npos] = leg
    out["ratio_16_vs_1"] = out["positions_16"]["us_per_call"] / out["positions_1"]["us_per_call"]
    env.close()
    return out


def clients_leg(args, esp, torch, wl):
    """Several host threads sharing one GPU context through the library's
    server (the paper's proposal of several processes sharing one GPU): each
    client submits 64 walkers x 32 electrons per step; throughput for 1, 2 and
    4 clients against one, and one client overlapping host work (a fixed
    matrix product) with its request."""
    import threading
    env = esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision="fp32c")
    per = 64 * 32
    steps = 6
    rng = np.random.default_rng(11)
    pos = wl.positions[rng.choice(wl.n_positions, size=(4, steps, per))]
    res = {"workload": "realistic environment, %d positions (64 walkers x 32 electrons) per client per step" % per}
    base = None
    with esp.Server(env, 4 * per) as srv:
        outs = np.zeros((4, steps, per))
        srv.wait(srv.submit(pos[0, 0], outs[0, 0]))  # warm-up
        for nc in (1, 2, 4):
            def client(c):
                for k in range(steps):
                    srv.wait(srv.submit(pos[c, k], outs[c, k]))
            th = [threading.Thread(target=client, args=(c,)) for c in range(nc)]
            b0 = srv.stats()["batches"]
            t0 = time.perf_counter()
            for t in th:
                t.start()
            for t in th:
                t.join()
            dt = time.perf_counter() - t0
            rate = nc * steps * per / dt
            base = base or rate
            res["clients_%d" % nc] = {"positions_per_s": rate, "vs_one_client": rate / base,
                                      "batches": srv.stats()["batches"] - b0}
        # overlap: host work between submit and wait, against the two in sequence
        A = np.random.default_rng(12).normal(size=(600, 600))
        t0 = time.perf_counter()
        for k in range(steps):
            srv.wait(srv.submit(pos[0, k], outs[0, k]))
            A @ A
        seq = time.perf_counter() - t0
        t0 = time.perf_counter()
        for k in range(steps):
            t = srv.submit(pos[0, k], outs[0, k])
            A @ A
            srv.wait(t)
        ovl = time.perf_counter() - t0
        res["overlap"] = {"sequential_ms_per_step": seq * 1e3 / steps, "overlapped_ms_per_step": ovl * 1e3 / steps,
                          "host_work": "600 x 600 matrix product per step"}
    env.close()
    return res


def coalescing_leg(esp, reps=50):
    """The paper's coalescing study on its own workload shape (268,782 cells +
    36 nuclei, one position): its kernel structure (blocks of 256 threads, 9
    iterations each, shared-memory block sum) with the coalesced and the
    incoalesced thread-to-cell mapping, FP64 and FP32 arithmetic; kernel time
    per launch (CUDA events) and the incoalesced/coalesced ratio, next to the
    paper's 6.0x (kernel only, GTX 275)."""
    from workloads import point_cells_environment
    wl = point_cells_environment(seed=1011 * 100 + 6, n_cells=268782, n_nuclei=36, n_positions=1)
    env = esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision="fp32c")
    out = {"workload": "268,782 cells + 36 nuclei, one position; 256 threads x 9 iterations per block (the "
                       "paper's N_th and N_loop), %d blocks" % ((268818 + 256 * 9 - 1) // (256 * 9)),
           "paper_kernel_ratio": 6.0}
    for layout, soa in (("records32B", False), ("soa", True)):
        for prec, fp64 in (("fp64", True), ("fp32", False)):
            vc, tc = env.study_cell_sum(wl.positions[0], False, fp64, n_loop=9, reps=reps, soa=soa)
            vi, ti = env.study_cell_sum(wl.positions[0], True, fp64, n_loop=9, reps=reps, soa=soa)
            out["%s_%s" % (layout, prec)] = {"coalesced_us": tc * 1e3, "incoalesced_us": ti * 1e3,
                                             "incoalesced_over_coalesced": ti / tc, "abs_diff_ha": abs(vc - vi)}
    env.close()
    return out


def host_units(wl):
    """The library's unit count of the environment (distributions after its
    screening and merges + point charges), from a host-only build that touches
    no GPU."""
    from paper_1011_4687_gb300 import build_lib, esp
    build_lib.build()
    with esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, flags=esp.FLAG_HOST_ONLY) as env:
        return env.info()


def run_reference(args):
    """The oracle as it stands, on this host's cores, on a bounded sample of the
    headline workload per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    wl = build_workload(args.config, 0, args.walkers)
    units = host_units(wl)
    cfg = workload_config(wl, args.config, units, args.gpus, args.walkers not in (0, WORKLOADS[args.config]["n_walkers"]))
    per_pos = units["n_distributions"] + units["n_point_charges"]
    threads = oracle.max_threads()
    sample = np.arange(args.ref_positions if args.ref_positions > 0 else threads)
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions[sample])
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    per = statistics.mean(times)
    val = per_pos * sample.size / per
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": val, "unit": "evals/s", "cores": min(threads, sample.size), "kind": "oracle",
                             "sample": "%d positions of the workload per step x all %d distributions + point "
                                       "charges (the library's unit count)" % (sample.size, per_pos)},
            "e2e": {"value": val, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed_device(fn, stream, flush, k):
    """Mean device time (ms, CUDA events on `stream`) of k calls of fn, L2 flushed before each."""
    import torch
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


def accuracy_leg(wl, kind, env, V, E, torch, oracle_mod):
    """FP32C errors of the timed step's own outputs.  realistic: against the FP64
    oracle on 1,024 positions (512 closest to the environment, 512 random) and
    16 whole walkers.  large: against the library's FP64 path (itself checked
    against the oracle to 1e-10 in the tests) on the same sample shape, and the
    FP64 path against the oracle on 16 of those positions."""
    ws, sample = sample_indices(wl, 16, 512, 512)
    n_walk = ws.size * wl.n_elec
    Vs = V.cpu().numpy()[sample]
    Es = E.cpu().numpy()[ws]
    env.set_precision("fp64")
    V64 = env.eval(torch.from_numpy(wl.positions[sample]).cuda())
    torch.cuda.synchronize()
    V64 = V64.cpu().numpy()
    env.set_precision("fp32c")
    sub = sample if kind == "realistic" else sample[n_walk:n_walk + 16]
    t0 = time.perf_counter()
    ref = oracle_mod.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions[sub])
    t_or = time.perf_counter() - t0
    out = {"sample": "%d whole walkers (%d positions) + 512 outermost + 512 random positions" % (ws.size, n_walk)}
    if kind == "realistic":
        Eref = oracle_mod.walker_energies(ref[:n_walk], ws.size, wl.n_elec)
        out.update({"against": "FP64 oracle",
                    "fp32c_max_point_err_ha": float(np.abs(Vs - ref).max()),
                    "fp32c_max_walker_err_ha": float(np.abs(Es - Eref).max()),
                    "fp64_max_rel_err": float(np.max(np.abs(V64 - ref) / np.maximum(np.abs(ref), 1.0)))})
    else:
        E64 = -V64[:n_walk].reshape(ws.size, wl.n_elec).sum(1)
        k = slice(n_walk, n_walk + 16)
        out.update({"against": "the library's FP64 path (oracle on 16 of the positions)",
                    "fp32c_max_point_err_ha": float(np.abs(Vs - V64).max()),
                    "fp32c_max_walker_err_ha": float(np.abs(Es - E64).max()),
                    "fp32c_max_point_err_vs_oracle_ha": float(np.abs(Vs[k] - ref).max()),
                    "fp64_max_rel_err_vs_oracle": float(np.max(np.abs(V64[k] - ref) / np.maximum(np.abs(ref), 1.0)))})
    return out, sub.size, t_or


def fp32c_step_leg(args, wl, kind, env, esp, torch, stream, flush, world, local, peaks):
    """K timed steps of the whole path (esp_eval_walkers, FP32C) with clocks,
    kernel times, census-based roofline and the end-to-end rate."""
    info = env.info()
    n_pos = wl.n_positions
    units = info["n_distributions"] + info["n_point_charges"]
    evals = units * n_pos
    pos = torch.from_numpy(wl.positions).cuda()
    V = torch.empty(n_pos, dtype=torch.float64, device="cuda")
    E = torch.empty(wl.n_walkers, dtype=torch.float64, device="cuda")
    env.set_timing(True)
    for _ in range(args.warmup):
        env.eval_walkers(pos, wl.n_walkers, wl.n_elec, V_out=V, E_out=E)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kern_ms = []
    if world > 1:
        import torch.distributed as dist
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
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ms = statistics.mean(s.elapsed_time(e) for s, e in zip(starts, ends))
    ms_max = max_over_ranks(ms, world, "cuda")
    kern = statistics.mean(kern_ms)
    # end to end through the public API with pinned host buffers
    pin_pos = torch.from_numpy(wl.positions).pin_memory()
    hv = torch.empty(n_pos, dtype=torch.float64).pin_memory().numpy()
    he = torch.empty(wl.n_walkers, dtype=torch.float64).pin_memory().numpy()
    hp = pin_pos.numpy()
    e2e_t = []
    for _ in range(min(args.steps, args.e2e_steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        env.eval_walkers(hp, wl.n_walkers, wl.n_elec, V_out=hv, E_out=he)
        e2e_t.append(time.perf_counter() - t0)
    # roofline of the potential kernel: algorithmic FP32 ops from a census of
    # 512 of the step's positions, against the measured FFMA lane-op rate
    cs = env.work_census(wl.positions[np.linspace(0, n_pos - 1, 512).astype(int)])
    ops, pt_ops, terms = census_ops(cs, n_pos, fp64=False)
    achieved = ops / (kern * 1e-3)
    peak = peaks["fp32_fma_per_s"]
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tops/s (FP32 lane ops)",
            "frac": achieved / peak, "traffic": profiled_traffic("potential_f32c_kernel", n_pos, kind),
            "kernel": "potential_f32c_kernel", "kernel_ms": kern,
            "algorithmic_ops_per_launch": ops, "ops_per_distribution_term": ops / max(terms, 1.0),
            "peak_source": "measured FFMA lane-op rate (esp_measure_peaks, %d SMs read from the device) of measured"
                           % peaks["num_sms"],
            "census": cs}
    res = {"value": evals * world / (ms_max * 1e-3), "ms_per_step": ms_max, "kernel_ms": kern,
           "clocks": clk.summary(), "roofline": roof, "units": units, "evals": evals,
           "e2e": {"value": evals * world / statistics.mean(e2e_t), "unit": "evals/s",
                   "h2d_bytes_per_step": int(n_pos * 24), "d2h_bytes_per_step": int(n_pos * 8 + wl.n_walkers * 8),
                   "steps": len(e2e_t)},
           "gpu_launches_per_step": 7 if n_pos >= 4096 else 4, "info": info}
    return res, pos, V, E


def fp64_leg(args, wl, env, torch, stream, flush, peaks):
    """The FP64 path on 16 whole walkers of the workload (time and roofline
    against the measured DFMA lane-op rate)."""
    nw = min(16, wl.n_walkers)
    n = nw * wl.n_elec
    pos = torch.from_numpy(wl.positions[:n].copy()).cuda()
    info = env.info()
    units = info["n_distributions"] + info["n_point_charges"]
    env.set_precision("fp64")
    env.eval_walkers(pos, nw, wl.n_elec)
    torch.cuda.synchronize()

    def one():
        env.eval_walkers(pos, nw, wl.n_elec)

    ms = timed_device(one, stream, flush, 2)
    kms = env.last_timing()[0]  # potential kernel of the last timed call
    env.set_precision("fp32c")
    cs = env.work_census(wl.positions[:min(n, 512)])
    ops, pt_ops, terms = census_ops(cs, n, fp64=True)
    achieved = (ops + pt_ops) / (kms * 1e-3)
    return {"value": units * n / (ms * 1e-3), "unit": "evals/s", "positions_per_step": n,
            "sample": "%d whole walkers x %d electrons of the workload" % (nw, wl.n_elec), "ms_per_step": ms,
            "roofline": {"bound": "fp64", "achieved": achieved / 1e12, "peak": peaks["fp64_fma_per_s"] / 1e12,
                         "unit": "Tops/s (FP64 lane ops)", "frac": achieved / peaks["fp64_fma_per_s"],
                         "kernel": "potential_f64_kernel", "kernel_ms": kms,
                         "ops_per_distribution_term": ops / max(terms, 1.0),
                         "peak_source": "measured DFMA lane-op rate (esp_measure_peaks) of measured"}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="large", choices=sorted(WORKLOADS),
                    help="headline workload (default: the largest configuration)")
    ap.add_argument("--ref-positions", type=int, default=0,
                    help="positions per oracle step (reference arm); 0 = one per host thread")
    ap.add_argument("--e2e-steps", type=int, default=2, help="steps of the end-to-end (host buffer) measurement")
    ap.add_argument("--no-oracle", action="store_true", help="skip the accuracy check and CPU baseline")
    ap.add_argument("--no-secondary", action="store_true", help="skip the realistic-configuration leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-systems leg")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate leg")
    ap.add_argument("--no-latency", action="store_true", help="skip the one-position-per-call leg")
    ap.add_argument("--coalescing-study", action="store_true",
                    help="run only the paper's coalesced vs incoalesced study and print its JSON")
    ap.add_argument("--study-reps", type=int, default=50, help="timed launches per variant of the study")
    ap.add_argument("--batch-systems", type=int, default=64, help="systems in the batched leg")
    ap.add_argument("--walkers", type=int, default=0,
                    help="walkers per GPU of the headline workload (0: the configuration's own; fewer only for "
                         "profiling, and the line then says REDUCED)")
    args = ap.parse_args(argv)
    keep_heap()
    if args.impl == "reference":
        return run_reference(args)
    if args.coalescing_study:
        from paper_1011_4687_gb300 import build_lib, esp
        build_lib.build()
        print(json.dumps({"coalescing_study": coalescing_leg(esp, args.study_reps)}), flush=True)
        return 0
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    reduced = args.walkers not in (0, WORKLOADS[args.config]["n_walkers"])

    # workloads are generated before any CUDA call (the batched systems in a
    # spawn-started pool, the others on threads)
    batch_wls = None
    if not args.no_batch and rank == 0:
        batch_wls = _gen_batched(args.batch_systems)
    wl = build_workload(args.config, rank, args.walkers)
    wl2 = None
    if not args.no_secondary and rank == 0 and args.config != "realistic":
        wl2 = build_workload("realistic")

    import torch
    import torch.distributed as dist
    from paper_1011_4687_gb300 import build_lib, esp

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        build_lib.build()
    if world > 1:
        dist.barrier()
    esp.load()
    peaks = esp.measure_peaks(local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    env = esp.Environment(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, precision="fp32c", stream=stream.cuda_stream)
    head, pos, V, E = fp32c_step_leg(args, wl, args.config, env, esp, torch, stream, flush, world, local, peaks)
    f64 = fp64_leg(args, wl, env, torch, stream, flush, peaks)
    if rank != 0:
        env.close()
        if world > 1:
            dist.destroy_process_group()
        return 0

    out = {"metric": METRIC, "value": head["value"], "unit": "evals/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": workload_config(wl, args.config, head["info"], world, reduced),
           "path": {"precision": "FP32C (FP32 pair sum, compensated; nuclei and near blocks FP64)",
                    "distributions_by_L": head["info"]["n_by_L"],
                    "step": "esp_eval_walkers: spatial order (3 launches), stage, potential, reduce, walker energies"},
           "gpu_launches": head["gpu_launches_per_step"] * args.steps,
           "clocks": head["clocks"], "roofline": head["roofline"], "e2e": head["e2e"], "fp64": f64,
           "peaks_measured": peaks}
    oracle_mod = None
    if not args.no_oracle:
        import oracle
        oracle.build()
        oracle_mod = oracle
        acc, n_or, t_or = accuracy_leg(wl, args.config, env, V, E, torch, oracle)
        out["accuracy"] = acc
        per_pos = head["units"]
        out["cpu_baseline"] = {"value": per_pos * n_or / t_or, "unit": "evals/s",
                               "cores": min(oracle.max_threads(), n_or), "kind": "oracle",
                               "sample": "%d positions of the workload x all %d distributions + point charges"
                                         % (n_or, per_pos)}

    def fp64_ref(env_):
        def f(p):
            env_.set_precision("fp64")
            v = env_.eval(torch.from_numpy(np.ascontiguousarray(p)).cuda())
            torch.cuda.synchronize()
            env_.set_precision("fp32c")
            return v.cpu().numpy(), "the library's FP64 path (oracle-checked to 1e-10 in the tests)"
        return f

    sur_legs = {}
    if not args.no_surrogate and not reduced:
        sur_legs[args.config] = surrogate_leg(args, env, wl, workload_label(wl, args.config), torch, stream, flush,
                                              head["ms_per_step"], V, ref_fn=fp64_ref(env))
    del pos, V, E
    env.close()

    if wl2 is not None:
        env2 = esp.Environment(wl2.nuclei_xyz, wl2.nuclei_Z, wl2.pairs, precision="fp32c", stream=stream.cuda_stream)
        a2 = argparse.Namespace(**vars(args))
        h2, pos2, V2, E2 = fp32c_step_leg(a2, wl2, "realistic", env2, esp, torch, stream, flush, 1, local, peaks)
        leg = {"workload": workload_label(wl2, "realistic"), "value": h2["value"], "unit": "evals/s",
               "ms_per_step": h2["ms_per_step"], "steps": args.steps, "warmup": args.warmup,
               "clocks": h2["clocks"], "roofline": h2["roofline"], "e2e": h2["e2e"],
               "fp64": fp64_leg(args, wl2, env2, torch, stream, flush, peaks)}
        if oracle_mod is not None:
            leg["accuracy"], _, _ = accuracy_leg(wl2, "realistic", env2, V2, E2, torch, oracle_mod)
        out["realistic"] = leg
        out["clients"] = clients_leg(args, esp, torch, wl2)
        if not args.no_surrogate:
            sur_legs["realistic"] = surrogate_leg(args, env2, wl2, workload_label(wl2, "realistic"), torch, stream,
                                                  flush, h2["ms_per_step"], V2, ref_fn=fp64_ref(env2))
        del pos2, V2, E2
        env2.close()
    if batch_wls is not None:
        out["batch"] = batch_leg(args, esp, torch, stream, flush, batch_wls, oracle_mod)
        del batch_wls
    if not args.no_latency:
        out["few_positions_per_call"] = latency_leg(args, esp, torch, stream, oracle_mod)
        out["coalescing_study"] = coalescing_leg(esp)
    if not args.no_surrogate:
        sur_legs["small"] = small_surrogate_leg(args, torch, stream, flush, oracle_mod)
        out["surrogate"] = sur_legs
    if oracle_mod is not None:
        # the paper's framing, one CPU core (one position of the headline
        # workload); last, because it leaves the oracle's OpenMP pool at one thread
        t1 = time.perf_counter()
        oracle_mod.potential(wl.nuclei_xyz, wl.nuclei_Z, wl.pairs, wl.positions[:1], threads=1)
        out["cpu_baseline"]["single_core_value"] = head["units"] * 1 / (time.perf_counter() - t1)
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
