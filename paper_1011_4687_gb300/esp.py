"""ctypes binding of libesp_gb300.so (include/esp.h).

Argument marshalling only: every step of an evaluation runs in the library's
CUDA kernels.  There is no CPU fallback; if the compiled library is missing
the import of this module's functions raises.

Positions and outputs may be numpy arrays (host; the call is synchronous) or
torch CUDA tensors (device; the call is enqueued on the context's stream).
"""
from __future__ import annotations

import ctypes
import os
import weakref
from typing import Optional

import numpy as np

from . import build_lib

ESP_OK, ESP_ERR_INVALID, ESP_ERR_OOM, ESP_ERR_CUDA, ESP_ERR_TIMEOUT, ESP_ERR_STATE, ESP_ERR_UNSUPPORTED = range(7)
FP64, FP32C = 0, 1
FLAG_HOST_ONLY = 1  # esp_options.flags: build on the host only, touch no GPU
PRECISIONS = {"fp64": FP64, "fp32c": FP32C}

GAUSS_PAIR_DTYPE = np.dtype([("A", "<f8", (3,)), ("alpha", "<f8"), ("lmn_a", "<i4", (3,)), ("pad_a", "<i4"),
                             ("B", "<f8", (3,)), ("beta", "<f8"), ("lmn_b", "<i4", (3,)), ("pad_b", "<i4")])
POINT_CHARGE_DTYPE = np.dtype([("xyz", "<f8", (3,)), ("Z", "<f8")])
assert GAUSS_PAIR_DTYPE.itemsize == 96 and POINT_CHARGE_DTYPE.itemsize == 32


class EspError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("esp status %d: %s" % (status, message))
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("size", ctypes.c_int32), ("precision", ctypes.c_int32), ("screen_tol", ctypes.c_double),
                ("qm_center", ctypes.c_double * 3), ("cuda_stream", ctypes.c_void_p),
                ("device", ctypes.c_int32), ("tile_size", ctypes.c_int32),
                ("threads_per_block", ctypes.c_int32), ("positions_per_thread", ctypes.c_int32),
                ("pair_splits", ctypes.c_int32), ("flags", ctypes.c_int32), ("near_radius", ctypes.c_double),
                ("point32_max_charge", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("n_point_charges", ctypes.c_int64), ("n_pairs_in", ctypes.c_int64),
                ("n_distributions", ctypes.c_int64), ("n_screened", ctypes.c_int64),
                ("n_by_L", ctypes.c_int64 * 5), ("n_tiles", ctypes.c_int64), ("n_near_tiles", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64),
                ("precision", ctypes.c_int32), ("tile_size", ctypes.c_int32),
                ("threads_per_block", ctypes.c_int32), ("positions_per_thread", ctypes.c_int32),
                ("pair_splits", ctypes.c_int32), ("device", ctypes.c_int32)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["n_by_L"] = list(self.n_by_L)
        return d


class TuneReport(ctypes.Structure):
    _fields_ = [("threads_per_block", ctypes.c_int32), ("positions_per_thread", ctypes.c_int32),
                ("split_scale", ctypes.c_double), ("best_ms", ctypes.c_double), ("n_tried", ctypes.c_int32),
                ("tried_threads", ctypes.c_int32 * 16), ("tried_ppt", ctypes.c_int32 * 16),
                ("tried_scale", ctypes.c_double * 16), ("tried_ms", ctypes.c_double * 16)]

    def as_dict(self):
        n = self.n_tried
        return {"threads_per_block": self.threads_per_block, "positions_per_thread": self.positions_per_thread,
                "split_scale": self.split_scale, "best_ms": self.best_ms,
                "tried": [{"threads": self.tried_threads[i], "ppt": self.tried_ppt[i],
                           "split_scale": self.tried_scale[i], "ms": self.tried_ms[i]} for i in range(n)]}


class SurrogateCfg(ctypes.Structure):
    _fields_ = [("size", ctypes.c_int32), ("n_train", ctypes.c_int32), ("n_valid", ctypes.c_int32),
                ("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("degree", ctypes.c_int32),
                ("qm_radius", ctypes.c_double), ("position_sd", ctypes.c_double), ("fourier_sigma", ctypes.c_double),
                ("lr", ctypes.c_double), ("tol", ctypes.c_double), ("voxel", ctypes.c_double),
                ("nucleus_exclusion", ctypes.c_double), ("probe_stride", ctypes.c_int32),
                ("label_precision", ctypes.c_int32), ("seed", ctypes.c_uint64), ("far_radius", ctypes.c_double),
                ("far_penetration", ctypes.c_double)]


class SurrogateStats(ctypes.Structure):
    _fields_ = [("n_fallback", ctypes.c_int64), ("n_probe_fail", ctypes.c_int64), ("surrogate_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("train_loss", ctypes.c_double), ("valid_max_err", ctypes.c_double),
                ("trusted_fraction", ctypes.c_double), ("n_params", ctypes.c_int64), ("n_baseline", ctypes.c_int64),
                ("valid_rms_err", ctypes.c_double), ("baseline_max_err", ctypes.c_double),
                ("baseline_rms_err", ctypes.c_double), ("n_near_entries", ctypes.c_int64),
                ("n_far_entries", ctypes.c_int64), ("baseline_trusted_fraction", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Peaks(ctypes.Structure):
    _fields_ = [("fp32_fma_per_s", ctypes.c_double), ("fp32x2_fma_per_s", ctypes.c_double),
                ("fp64_fma_per_s", ctypes.c_double),
                ("mufu_rsqrt_per_s", ctypes.c_double), ("mufu_ex2_per_s", ctypes.c_double),
                ("fp32_ms", ctypes.c_double), ("fp32x2_ms", ctypes.c_double), ("fp64_ms", ctypes.c_double),
                ("rsqrt_ms", ctypes.c_double),
                ("ex2_ms", ctypes.c_double), ("num_sms", ctypes.c_int32), ("clock_khz", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


EXPORTED = ["esp_default_options", "esp_create", "esp_eval", "esp_eval_walkers", "esp_set_precision",
            "esp_get_info", "esp_synchronize", "esp_destroy", "esp_status_string", "esp_last_error",
            "esp_abi_version", "esp_debug_boys", "esp_debug_host_eval", "esp_set_timing", "esp_last_timing"]

_lib = None


def library_path() -> str:
    return build_lib.LIB


def load(build_if_missing: bool = False):
    """Load the compiled library (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = build_lib.LIB
    if build_if_missing and build_lib.is_stale():
        build_lib.build()
    if not os.path.exists(path):
        raise RuntimeError("libesp_gb300.so is not built (run paper_1011_4687_gb300.build_lib); "
                           "there is no CPU fallback")
    lib = ctypes.CDLL(path)
    P, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.esp_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.esp_default_options.restype = None
    lib.esp_create.argtypes = [P, i64, P, P, i64, ctypes.POINTER(Options), ctypes.POINTER(P)]
    lib.esp_create.restype = ctypes.c_int
    lib.esp_eval.argtypes = [P, P, i64, P]
    lib.esp_eval.restype = ctypes.c_int
    lib.esp_eval_walkers.argtypes = [P, P, i64, i64, P, P]
    lib.esp_eval_walkers.restype = ctypes.c_int
    lib.esp_set_precision.argtypes = [P, i32]
    lib.esp_set_precision.restype = ctypes.c_int
    lib.esp_get_info.argtypes = [P, ctypes.POINTER(Info)]
    lib.esp_get_info.restype = ctypes.c_int
    lib.esp_synchronize.argtypes = [P]
    lib.esp_synchronize.restype = ctypes.c_int
    lib.esp_destroy.argtypes = [P]
    lib.esp_destroy.restype = None
    lib.esp_status_string.argtypes = [ctypes.c_int]
    lib.esp_status_string.restype = ctypes.c_char_p
    lib.esp_last_error.argtypes = []
    lib.esp_last_error.restype = ctypes.c_char_p
    lib.esp_abi_version.restype = i32
    lib.esp_debug_boys.argtypes = [i32, i32, d, P]
    lib.esp_debug_boys.restype = ctypes.c_int
    lib.esp_debug_host_eval.argtypes = [P, P, i64, P]
    lib.esp_debug_host_eval.restype = ctypes.c_int
    PP = ctypes.POINTER(ctypes.c_void_p)
    lib.esp_batch_create.argtypes = [PP, i32, P, ctypes.POINTER(P)]
    lib.esp_batch_create.restype = ctypes.c_int
    lib.esp_batch_eval.argtypes = [P, PP, ctypes.POINTER(i64), PP]
    lib.esp_batch_eval.restype = ctypes.c_int
    lib.esp_batch_autotune.argtypes = [P, PP, ctypes.POINTER(i64), PP, ctypes.POINTER(TuneReport)]
    lib.esp_batch_autotune.restype = ctypes.c_int
    lib.esp_batch_set_shape.argtypes = [P, i32, i32, d]
    lib.esp_batch_set_shape.restype = ctypes.c_int
    lib.esp_batch_last_ms.argtypes = [P, ctypes.POINTER(d)]
    lib.esp_batch_last_ms.restype = ctypes.c_int
    lib.esp_batch_destroy.argtypes = [P]
    lib.esp_batch_destroy.restype = None
    lib.esp_surrogate_default_cfg.argtypes = [ctypes.POINTER(SurrogateCfg)]
    lib.esp_surrogate_default_cfg.restype = None
    lib.esp_surrogate_train.argtypes = [P, ctypes.POINTER(SurrogateCfg), ctypes.POINTER(P)]
    lib.esp_surrogate_train.restype = ctypes.c_int
    lib.esp_surrogate_eval.argtypes = [P, P, i64, P, ctypes.POINTER(SurrogateStats)]
    lib.esp_surrogate_eval.restype = ctypes.c_int
    lib.esp_surrogate_predict.argtypes = [P, P, i64, P]
    lib.esp_surrogate_predict.restype = ctypes.c_int
    lib.esp_surrogate_info.argtypes = [P, ctypes.POINTER(SurrogateStats)]
    lib.esp_surrogate_info.restype = ctypes.c_int
    lib.esp_surrogate_save.argtypes = [P, ctypes.c_char_p]
    lib.esp_surrogate_save.restype = ctypes.c_int
    lib.esp_surrogate_load.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(P)]
    lib.esp_surrogate_load.restype = ctypes.c_int
    lib.esp_surrogate_debug_step.argtypes = [P, P, P, i32, P, P, P]
    lib.esp_surrogate_debug_step.restype = ctypes.c_int
    lib.esp_surrogate_features.argtypes = [P, P, P]
    lib.esp_surrogate_features.restype = ctypes.c_int
    lib.esp_surrogate_set_wait_limit.argtypes = [P, i32]
    lib.esp_surrogate_set_wait_limit.restype = ctypes.c_int
    lib.esp_surrogate_debug_expansion.argtypes = [P, d, P, i32]
    lib.esp_surrogate_debug_expansion.restype = ctypes.c_int
    lib.esp_debug_fault_active.argtypes = [ctypes.c_char_p]
    lib.esp_debug_fault_active.restype = i32
    lib.esp_debug_solid_harmonics.argtypes = [i32, P, P]
    lib.esp_debug_solid_harmonics.restype = ctypes.c_int
    lib.esp_surrogate_debug_net.argtypes = [P, P, i32, P]
    lib.esp_surrogate_debug_net.restype = ctypes.c_int
    lib.esp_surrogate_destroy.argtypes = [P]
    lib.esp_surrogate_destroy.restype = None
    lib.esp_graph_create.argtypes = [P, P, i64, P, ctypes.POINTER(P)]
    lib.esp_graph_create.restype = ctypes.c_int
    lib.esp_graph_launch.argtypes = [P]
    lib.esp_graph_launch.restype = ctypes.c_int
    lib.esp_graph_destroy.argtypes = [P]
    lib.esp_graph_destroy.restype = None
    lib.esp_server_create.argtypes = [P, i64, ctypes.POINTER(P)]
    lib.esp_server_create.restype = ctypes.c_int
    lib.esp_server_submit.argtypes = [P, P, i64, P, ctypes.POINTER(i64)]
    lib.esp_server_submit.restype = ctypes.c_int
    lib.esp_server_wait.argtypes = [P, i64]
    lib.esp_server_wait.restype = ctypes.c_int
    lib.esp_server_stats.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.esp_server_stats.restype = ctypes.c_int
    lib.esp_server_destroy.argtypes = [P]
    lib.esp_server_destroy.restype = None
    lib.esp_study_cell_sum.argtypes = [P, P, i32, i32, i32, i32, i32, P, P]
    lib.esp_study_cell_sum.restype = ctypes.c_int
    lib.esp_work_census.argtypes = [P, P, i64, P]
    lib.esp_work_census.restype = ctypes.c_int
    lib.esp_measure_peaks.argtypes = [i32, ctypes.POINTER(Peaks)]
    lib.esp_measure_peaks.restype = ctypes.c_int
    lib.esp_set_timing.argtypes = [P, i32]
    lib.esp_set_timing.restype = ctypes.c_int
    lib.esp_last_timing.argtypes = [P, ctypes.POINTER(d), ctypes.POINTER(d)]
    lib.esp_last_timing.restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int):
    if status != ESP_OK:
        msg = _lib.esp_last_error().decode(errors="replace")
        raise EspError(status, msg or _lib.esp_status_string(status).decode())


def default_options() -> Options:
    o = Options()
    load().esp_default_options(ctypes.byref(o))
    return o


def pack_pairs(pairs) -> np.ndarray:
    """PairList (SoA) -> array of esp_gauss_pair."""
    n = len(pairs)
    a = np.zeros(n, GAUSS_PAIR_DTYPE)
    if n:
        a["A"], a["alpha"], a["lmn_a"] = pairs.A, pairs.alpha, pairs.la
        a["B"], a["beta"], a["lmn_b"] = pairs.B, pairs.beta, pairs.lb
    return a


def pack_charges(xyz, Z) -> np.ndarray:
    xyz = np.asarray(xyz, np.float64).reshape(-1, 3)
    a = np.zeros(xyz.shape[0], POINT_CHARGE_DTYPE)
    if xyz.shape[0]:
        a["xyz"], a["Z"] = xyz, np.asarray(Z, np.float64).reshape(-1)
    return a


def _ptr(x):
    """(pointer, is_device) of a numpy array or torch tensor."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous or x.dtype != np.float64:
            raise ValueError("host arrays must be C-contiguous float64")
        return ctypes.c_void_p(x.ctypes.data), False
    import torch  # noqa: F401  (only for device tensors)
    if x.dtype != torch.float64 or not x.is_contiguous():
        raise ValueError("tensors must be contiguous float64")
    return ctypes.c_void_p(x.data_ptr()), bool(x.is_cuda)


class Environment:
    """A built environment on one device (owns an esp_ctx)."""

    def __init__(self, nuclei_xyz, nuclei_Z, pairs, precision="fp32c", screen_tol=1e-12,
                 qm_center=(0.0, 0.0, 0.0), stream=None, device=-1, tile_size=0, threads_per_block=0,
                 positions_per_thread=0, pair_splits=0, near_radius=-1.0, flags=0, point32_max_charge=-1.0):
        lib = load()
        opt = default_options()
        opt.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        opt.screen_tol = float(screen_tol)
        opt.qm_center[:] = [float(v) for v in qm_center]
        opt.cuda_stream = ctypes.c_void_p(int(stream) if stream is not None else 0)
        opt.device = int(device)
        opt.tile_size = int(tile_size)
        opt.threads_per_block = int(threads_per_block)
        opt.positions_per_thread = int(positions_per_thread)
        opt.pair_splits = int(pair_splits)
        opt.near_radius = float(near_radius)
        opt.flags = int(flags)
        opt.point32_max_charge = float(point32_max_charge)
        ch = pack_charges(nuclei_xyz, nuclei_Z)
        pr = pack_pairs(pairs)
        w = np.ascontiguousarray(pairs.w, np.float64)
        ctx = ctypes.c_void_p()
        _check(lib.esp_create(ch.ctypes.data if ch.size else None, ch.size,
                              pr.ctypes.data if pr.size else None, w.ctypes.data if w.size else None,
                              pr.size, ctypes.byref(opt), ctypes.byref(ctx)))
        self._ctx = ctx
        self.stream = stream
        self._dependents = weakref.WeakSet()  # surrogates bound to this context

    # -- lifetime ------------------------------------------------------------
    def close(self):
        """Free the context (and first any surrogate still bound to it)."""
        for d in list(getattr(self, "_dependents", ())):
            d.close()
        if getattr(self, "_ctx", None) and self._ctx.value:
            load().esp_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls ---------------------------------------------------------------
    @property
    def handle(self) -> ctypes.c_void_p:
        return self._ctx

    def info(self) -> dict:
        inf = Info()
        _check(load().esp_get_info(self._ctx, ctypes.byref(inf)))
        return inf.as_dict()

    def set_precision(self, precision):
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _check(load().esp_set_precision(self._ctx, p))

    def set_timing(self, enable: bool = True):
        _check(load().esp_set_timing(self._ctx, int(bool(enable))))

    def last_timing(self):
        """(potential-kernel ms, device-pipeline ms) of the last evaluation."""
        k, t = ctypes.c_double(), ctypes.c_double()
        _check(load().esp_last_timing(self._ctx, ctypes.byref(k), ctypes.byref(t)))
        return k.value, t.value

    def synchronize(self):
        _check(load().esp_synchronize(self._ctx))

    def eval(self, positions, out=None):
        """V at each position.  numpy in -> numpy out; CUDA tensor in -> CUDA tensor out."""
        n = int(positions.shape[0]) if positions.ndim == 2 else int(positions.size // 3)
        if out is None:
            if isinstance(positions, np.ndarray):
                out = np.zeros(n, np.float64)
            else:
                import torch
                out = torch.empty(n, dtype=torch.float64, device=positions.device)
        pp, _ = _ptr(positions)
        po, _ = _ptr(out)
        _check(load().esp_eval(self._ctx, pp, n, po))
        return out

    def eval_walkers(self, positions, n_walkers, n_elec, V_out=None, E_out=None, want_V=True):
        """(V, E) with E[w] = -sum_e V[w, e]."""
        host = isinstance(positions, np.ndarray)
        if E_out is None:
            if host:
                E_out = np.zeros(n_walkers, np.float64)
            else:
                import torch
                E_out = torch.empty(n_walkers, dtype=torch.float64, device=positions.device)
        if V_out is None and want_V:
            if host:
                V_out = np.zeros(n_walkers * n_elec, np.float64)
            else:
                import torch
                V_out = torch.empty(n_walkers * n_elec, dtype=torch.float64, device=positions.device)
        pp, _ = _ptr(positions)
        pv, _ = _ptr(V_out)
        pe, _ = _ptr(E_out)
        _check(load().esp_eval_walkers(self._ctx, pp, int(n_walkers), int(n_elec), pv, pe))
        return V_out, E_out

    def work_census(self, positions: np.ndarray) -> dict:
        """Terms per (L, short-range, Boys band) at host positions (esp_work_census):
        {"far30": [5], "mid": [5], "far45": [5] ... } keyed as below, counts over all positions."""
        pos = np.ascontiguousarray(positions, np.float64).reshape(-1, 3)
        c = np.zeros(32, np.int64)
        _check(load().esp_work_census(self._ctx, pos.ctypes.data, pos.shape[0], c.ctypes.data))
        t = c[:30].reshape(2, 5, 3)  # [short][L][band]
        return {"positions": int(pos.shape[0]), "T_lt_30": t[:, :, 0].tolist(), "T_30_45": t[:, :, 1].tolist(),
                "T_ge_45": t[:, :, 2].tolist(), "point_terms": int(c[30]), "point32_terms": int(c[31])}

    def study_cell_sum(self, position, incoalesced: bool, fp64: bool, n_loop: int = 9, reps: int = 20,
                       soa: bool = False):
        """The paper's coalescing study on this context's point charges at one
        position: (V, ms per launch) of the coalesced or incoalesced mapping,
        over the 32-byte records or separate arrays (soa)."""
        p = np.ascontiguousarray(position, np.float64).reshape(3)
        v, ms = ctypes.c_double(), ctypes.c_double()
        _check(load().esp_study_cell_sum(self._ctx, p.ctypes.data, int(bool(incoalesced)), int(bool(fp64)),
                                         int(bool(soa)), int(n_loop), int(reps), ctypes.byref(v), ctypes.byref(ms)))
        return v.value, ms.value

    def debug_host_eval(self, positions: np.ndarray) -> np.ndarray:
        """Test hook: evaluate the built tiles on the host in FP64 (never used by eval)."""
        pos = np.ascontiguousarray(positions, np.float64).reshape(-1, 3)
        V = np.zeros(pos.shape[0])
        _check(load().esp_debug_host_eval(self._ctx, pos.ctypes.data, pos.shape[0], V.ctypes.data))
        return V


def measure_peaks(device: int = -1) -> dict:
    """Measured FFMA / DFMA / MUFU lane-op rates of the device (esp_measure_peaks)."""
    p = Peaks()
    _check(load().esp_measure_peaks(int(device), ctypes.byref(p)))
    return p.as_dict()


def debug_fault_active(what: str) -> bool:
    """Test hook: does the host-side fault injection (ESP_FAULT) name `what`?"""
    return bool(load().esp_debug_fault_active(what.encode()))


def debug_solid_harmonics(L: int, u) -> np.ndarray:
    """Test hook: the surrogate's real regular solid harmonics S_k(u), k < (L+1)^2, on the host."""
    u = np.ascontiguousarray(u, np.float64).reshape(3)
    out = np.zeros((L + 1) ** 2)
    _check(load().esp_debug_solid_harmonics(int(L), u.ctypes.data, out.ctypes.data))
    return out


def debug_boys(precision, nmax: int, T: float) -> np.ndarray:
    """Test hook: the device Boys algorithm of `precision`, run on the host."""
    F = np.zeros(nmax + 1)
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(load().esp_debug_boys(p, int(nmax), float(T), F.ctypes.data))
    return F


class Graph:
    """The few-position evaluation of a fixed device buffer, captured once and
    replayed per call (esp_graph_*).  positions [n, 3] and out [n] are CUDA
    float64 tensors that stay in place; write new positions into `positions`
    between launches."""

    def __init__(self, env, positions, out):
        self.env, self.positions, self.out = env, positions, out
        g = ctypes.c_void_p()
        _check(load().esp_graph_create(env.handle, ctypes.c_void_p(positions.data_ptr()), int(positions.shape[0]),
                                       ctypes.c_void_p(out.data_ptr()), ctypes.byref(g)))
        self._g = g
        env._dependents.add(self)

    def launch(self):
        _check(load().esp_graph_launch(self._g))
        return self.out

    def close(self):
        if getattr(self, "_g", None) and self._g.value:
            load().esp_graph_destroy(self._g)
            self._g = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """One context shared by several host threads (esp_server_*): submit()
    queues host positions and returns a ticket, wait() blocks until that
    request's potentials are in its output array."""

    def __init__(self, env, max_positions):
        self.env = env
        h = ctypes.c_void_p()
        _check(load().esp_server_create(env.handle, int(max_positions), ctypes.byref(h)))
        self._h = h
        self._keep = {}
        env._dependents.add(self)

    def submit(self, positions: np.ndarray, out: np.ndarray) -> int:
        pos = np.ascontiguousarray(positions, np.float64).reshape(-1, 3)
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.size != pos.shape[0]:
            raise ValueError("out must be a contiguous float64 array of one value per position")
        t = ctypes.c_int64()
        _check(load().esp_server_submit(self._h, pos.ctypes.data, pos.shape[0], out.ctypes.data, ctypes.byref(t)))
        self._keep[t.value] = (pos, out)  # keep the buffers alive until the wait
        return t.value

    def wait(self, ticket: int):
        try:
            _check(load().esp_server_wait(self._h, int(ticket)))
        finally:
            self._keep.pop(int(ticket), None)

    def stats(self):
        b, n = ctypes.c_int64(), ctypes.c_int64()
        _check(load().esp_server_stats(self._h, ctypes.byref(b), ctypes.byref(n)))
        return {"batches": b.value, "positions": n.value}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().esp_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many environments evaluated together (persistent kernel, CUDA graph).

    The environments must outlive the batch, share one device and one
    precision; positions and outputs are CUDA tensors (device memory)."""

    def __init__(self, envs, stream=None):
        lib = load()
        self.envs = list(envs)
        arr = (ctypes.c_void_p * len(self.envs))(*[e.handle.value for e in self.envs])
        b = ctypes.c_void_p()
        _check(lib.esp_batch_create(arr, len(self.envs), ctypes.c_void_p(int(stream) if stream is not None else 0),
                                    ctypes.byref(b)))
        self._b = b

    def _arrays(self, positions, outs):
        import torch
        n = len(self.envs)
        assert len(positions) == n
        if outs is None:
            outs = [torch.empty(int(p.shape[0]), dtype=torch.float64, device=p.device) for p in positions]
        P = (ctypes.c_void_p * n)(*[p.data_ptr() if p.numel() else 0 for p in positions])
        V = (ctypes.c_void_p * n)(*[v.data_ptr() if v.numel() else 0 for v in outs])
        N = (ctypes.c_int64 * n)(*[int(p.shape[0]) for p in positions])
        return P, N, V, outs

    def eval(self, positions, outs=None):
        P, N, V, outs = self._arrays(positions, outs)
        _check(load().esp_batch_eval(self._b, P, N, V))
        return outs

    def set_shape(self, threads, ppt, split_scale=1.0):
        _check(load().esp_batch_set_shape(self._b, int(threads), int(ppt), float(split_scale)))

    def last_ms(self) -> float:
        ms = ctypes.c_double()
        _check(load().esp_batch_last_ms(self._b, ctypes.byref(ms)))
        return ms.value

    def signature(self, positions) -> str:
        """Workload key for the autotune cache: environment sizes, position counts, device."""
        import hashlib
        import torch
        parts = [torch.cuda.get_device_name(), str(len(self.envs))]
        for e, p in zip(self.envs, positions):
            i = e.info()
            parts.append("%d:%d:%d:%d" % (i["n_distributions"], i["n_point_charges"], i["tile_size"], int(p.shape[0])))
        return hashlib.sha256("|".join(parts).encode()).hexdigest()[:24]

    def autotune(self, positions, outs=None, cache_path=None):
        """Time the built launch shapes x split multipliers and keep the best.
        With cache_path, a stored choice for the same workload key is reused."""
        import json
        import os
        key = self.signature(positions)
        cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
            if key in cache:
                c = cache[key]
                self.set_shape(c["threads_per_block"], c["positions_per_thread"], c["split_scale"])
                return dict(c, cached=True)
        P, N, V, outs = self._arrays(positions, outs)
        rep = TuneReport()
        _check(load().esp_batch_autotune(self._b, P, N, V, ctypes.byref(rep)))
        d = rep.as_dict()
        if cache_path:
            cache[key] = {k: d[k] for k in ("threads_per_block", "positions_per_thread", "split_scale", "best_ms")}
            tmp = cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(tmp, cache_path)
        return dict(d, cached=False)

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            load().esp_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


N_SURROGATE_PARAMS = 64 * 256 + 256 + 3 * (256 * 256 + 256) + 256 + 1


class Surrogate:
    """Learned surrogate of an Environment's potential over its QM sphere,
    with exact fallback (see include/esp.h)."""

    def __init__(self, env, _handle=None, **cfg):
        self.env = env
        if _handle is not None:
            self._s = _handle
            env._dependents.add(self)
            return
        lib = load()
        c = SurrogateCfg()
        lib.esp_surrogate_default_cfg(ctypes.byref(c))
        for k, v in cfg.items():
            setattr(c, k, v)
        h = ctypes.c_void_p()
        _check(lib.esp_surrogate_train(env.handle, ctypes.byref(c), ctypes.byref(h)))
        self._s = h
        env._dependents.add(self)

    @staticmethod
    def load(env, path):
        h = ctypes.c_void_p()
        _check(load().esp_surrogate_load(env.handle, path.encode(), ctypes.byref(h)))
        return Surrogate(env, _handle=h)

    def save(self, path):
        _check(load().esp_surrogate_save(self._s, path.encode()))

    def eval(self, positions, out=None):
        """(V, stats) for a CUDA tensor of positions [n, 3]."""
        import torch
        n = int(positions.shape[0])
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=positions.device)
        st = SurrogateStats()
        _check(load().esp_surrogate_eval(self._s, ctypes.c_void_p(positions.data_ptr()), n,
                                          ctypes.c_void_p(out.data_ptr()), ctypes.byref(st)))
        return out, st.as_dict()

    def predict(self, positions, out=None):
        import torch
        n = int(positions.shape[0])
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=positions.device)
        _check(load().esp_surrogate_predict(self._s, ctypes.c_void_p(positions.data_ptr()), n,
                                             ctypes.c_void_p(out.data_ptr())))
        return out

    def info(self) -> dict:
        st = SurrogateStats()
        _check(load().esp_surrogate_info(self._s, ctypes.byref(st)))
        return st.as_dict()

    def debug_step(self, positions: np.ndarray, targets: np.ndarray):
        """(params, grad, y) of one forward/backward pass on a host batch (no update)."""
        pos = np.ascontiguousarray(positions, np.float64).reshape(-1, 3)
        t = np.ascontiguousarray(targets, np.float32)
        params = np.zeros(N_SURROGATE_PARAMS, np.float32)
        grad = np.zeros(N_SURROGATE_PARAMS, np.float32)
        y = np.zeros(pos.shape[0], np.float32)
        _check(load().esp_surrogate_debug_step(self._s, pos.ctypes.data, t.ctypes.data, pos.shape[0],
                                                params.ctypes.data, grad.ctypes.data, y.ctypes.data))
        return params, grad, y

    def debug_net(self, positions: np.ndarray) -> np.ndarray:
        """Network outputs y of the fused tensor-core inference kernel at host positions."""
        pos = np.ascontiguousarray(positions, np.float64).reshape(-1, 3)
        y = np.zeros(pos.shape[0], np.float32)
        _check(load().esp_surrogate_debug_net(self._s, pos.ctypes.data, pos.shape[0], y.ctypes.data))
        return y

    def set_wait_limit(self, limit: int = -1):
        """Iterations of the network kernel's bounded waits (-1: the default)."""
        _check(load().esp_surrogate_set_wait_limit(self._s, int(limit)))

    def debug_expansion(self, dc: float = 0.0) -> np.ndarray:
        """Test hook: add dc to the expansion's constant coefficient; returns the coefficients."""
        n = self.info()["n_baseline"]
        c = np.zeros(max(n, 1))
        _check(load().esp_surrogate_debug_expansion(self._s, float(dc), c.ctypes.data, int(n)))
        return c[:n]

    def features(self):
        freq = np.zeros((32, 3), np.float32)
        ci = np.zeros(4)
        _check(load().esp_surrogate_features(self._s, freq.ctypes.data, ci.ctypes.data))
        return freq, ci[:3].copy(), float(ci[3])

    def close(self):
        if getattr(self, "_s", None) and self._s.value:
            load().esp_surrogate_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
