"""FP64 CPU oracle for the environment electrostatic potential.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark may use it; the library never does.  It shares no code with
the CUDA library (see esp_oracle.c for what it computes and how).

`build()` compiles esp_oracle.c with gcc into oracle/_build/liboracle.so.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "esp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, OpenMP, no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fno-fast-math", "-ffp-contract=off", "-std=c11",
           "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
            P = ctypes.c_void_p
            lib.oracle_boys.argtypes = [ctypes.c_int, d, P]
            lib.oracle_boys.restype = ctypes.c_int
            lib.oracle_pair_potential.argtypes = [P, d, P, P, d, P, P]
            lib.oracle_pair_potential.restype = d
            lib.oracle_potential.argtypes = [P, P, i64, P, P, P, P, P, P, P, i64, P, i64, P, ctypes.c_int]
            lib.oracle_potential.restype = ctypes.c_int
            lib.oracle_abs_terms.argtypes = lib.oracle_potential.argtypes
            lib.oracle_abs_terms.restype = ctypes.c_int
            lib.oracle_walker_energies.argtypes = [P, i64, i64, P]
            lib.oracle_walker_energies.restype = ctypes.c_int
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


def boys(nmax: int, T: float) -> np.ndarray:
    """[F_0(T), ..., F_nmax(T)]."""
    out = np.zeros(nmax + 1)
    if _load().oracle_boys(int(nmax), float(T), _ptr(out)) != 0:
        raise ValueError("bad Boys arguments")
    return out


def pair_potential(A, alpha, la, B, beta, lb, C) -> float:
    """int chi_a chi_b / |r - C| dr for one unnormalised Cartesian primitive pair."""
    A, B, C = _c(A, np.float64), _c(B, np.float64), _c(C, np.float64)
    la, lb = _c(la, np.int32), _c(lb, np.int32)
    return float(_load().oracle_pair_potential(_ptr(A), float(alpha), _ptr(la), _ptr(B),
                                               float(beta), _ptr(lb), _ptr(C)))


def potential(nuclei_xyz, nuclei_Z, pairs, positions, threads: int = 0) -> np.ndarray:
    """V[N] = sum_beta Z/|C-R| + sum_ab w_ab (a|1/r_C|b), FP64, Neumaier-summed."""
    nx = _c(nuclei_xyz, np.float64).reshape(-1, 3)
    nz = _c(nuclei_Z, np.float64).reshape(-1)
    pos = _c(positions, np.float64).reshape(-1, 3)
    A, al, la = _c(pairs.A, np.float64), _c(pairs.alpha, np.float64), _c(pairs.la, np.int32)
    B, be, lb = _c(pairs.B, np.float64), _c(pairs.beta, np.float64), _c(pairs.lb, np.int32)
    w = _c(pairs.w, np.float64)
    V = np.zeros(pos.shape[0])
    rc = _load().oracle_potential(_ptr(nx), _ptr(nz), nx.shape[0], _ptr(A), _ptr(al), _ptr(la),
                                  _ptr(B), _ptr(be), _ptr(lb), _ptr(w), w.shape[0],
                                  _ptr(pos), pos.shape[0], _ptr(V), int(threads))
    if rc != 0:
        raise ValueError("oracle rejected its input")
    return V


def abs_terms(nuclei_xyz, nuclei_Z, pairs, positions, threads: int = 0) -> np.ndarray:
    """K[N] = sum of |term| over every point charge and pair: the condition of V[N]."""
    nx = _c(nuclei_xyz, np.float64).reshape(-1, 3)
    nz = _c(nuclei_Z, np.float64).reshape(-1)
    pos = _c(positions, np.float64).reshape(-1, 3)
    A, al, la = _c(pairs.A, np.float64), _c(pairs.alpha, np.float64), _c(pairs.la, np.int32)
    B, be, lb = _c(pairs.B, np.float64), _c(pairs.beta, np.float64), _c(pairs.lb, np.int32)
    w = _c(pairs.w, np.float64)
    K = np.zeros(pos.shape[0])
    rc = _load().oracle_abs_terms(_ptr(nx), _ptr(nz), nx.shape[0], _ptr(A), _ptr(al), _ptr(la),
                                  _ptr(B), _ptr(be), _ptr(lb), _ptr(w), w.shape[0],
                                  _ptr(pos), pos.shape[0], _ptr(K), int(threads))
    if rc != 0:
        raise ValueError("oracle rejected its input")
    return K


def walker_energies(V, n_walkers: int, n_elec: int) -> np.ndarray:
    """E[w] = -sum_e V[w, e] (the walker's sum of U_ES over its electrons)."""
    V = _c(V, np.float64)
    assert V.size == n_walkers * n_elec
    E = np.zeros(n_walkers)
    if _load().oracle_walker_energies(_ptr(V), int(n_walkers), int(n_elec), _ptr(E)) != 0:
        raise ValueError("bad walker arguments")
    return E


def max_threads() -> int:
    return int(_load().oracle_max_threads())
