import ctypes
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _keep_heap():
    """Keep freed large numpy buffers in the process heap.

    Workload generation allocates many large temporaries; returning each to the
    kernel and faulting it back in dominates its run time on some hosts."""
    try:
        libc = ctypes.CDLL("libc.so.6")
        libc.mallopt(-4, 0)            # M_MMAP_MAX: serve large blocks from the heap
        libc.mallopt(-1, 1 << 30)      # M_TRIM_THRESHOLD: do not trim the heap
        libc.mallopt(-8, 1)            # M_ARENA_MAX: the generator's threads share that one arena
    except (OSError, AttributeError):
        pass


_keep_heap()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (run with -m gpu)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def pytest_terminal_summary(terminalreporter):
    """How many points of the kappa-bounded FP32C parity cases (synthetic p/d
    environments with positions inside large charges) needed more than the
    flat 2e-6 Ha bound."""
    mod = sys.modules.get("tests.test_gpu_parity") or sys.modules.get("test_gpu_parity")
    stats = getattr(mod, "KAPPA_STATS", None) if mod else None
    if stats and stats[0]:
        terminalreporter.write_line(
            "fp32c kappa-bounded cases: %d cases, %d points, %d beyond a flat 2e-6 Ha (worst %.3e Ha)"
            % tuple(stats))
