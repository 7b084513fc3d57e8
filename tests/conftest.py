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
    except (OSError, AttributeError):
        pass


_keep_heap()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (run with -m gpu)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")
