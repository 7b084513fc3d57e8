"""Host-side logic of bench.py (no GPU): the algorithmic operation count of a
work census and the DRAM-traffic lookup behind the bench line's roofline."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_term_ops_far_form_counts():
    """The far (multipole) form of an L = 0 term: offset 3, |d|^2 3, contraction
    1, accumulate 1; each higher L adds its Boys powers, recursion and
    contraction, so the count grows with L."""
    far = [bench.term_ops(L, "asym", False) for L in range(5)]
    assert far[0] == 8
    assert all(b > a for a, b in zip(far, far[1:]))
    # the table form always costs more than the far form of the same L
    assert all(bench.term_ops(L, "table", False) > far[L] for L in range(5))


def test_census_ops_scales_with_positions():
    census = {"positions": 512, "T_lt_30": [[10, 0, 0, 0, 0], [0] * 5], "T_30_45": [[0] * 5, [0] * 5],
              "T_ge_45": [[100, 0, 0, 0, 0], [0] * 5], "point_terms": 7, "point32_terms": 0}
    ops, pt, terms = bench.census_ops(census, 1024, fp64=False)
    # FP32: T < 30 takes the table, everything above the far form
    assert terms == 2 * 110
    assert ops == 2 * (10 * bench.term_ops(0, "table", False) + 100 * bench.term_ops(0, "asym", False))
    assert pt == 2 * 7 * bench.POINT_OPS_F64


def test_profiled_traffic_model_and_hash(tmp_path, monkeypatch):
    """Exact-size entries apply only at their size, line entries at any size,
    and nothing applies once the kernel source hash differs."""
    h = bench.kernel_source_hash()
    t = {"potential_f32c_kernel/realistic": {"source_hash": h, "positions": 100, "dram_bytes": 5000},
         "potential_f32c_kernel/large": {"source_hash": h, "fixed_bytes": 1000.0, "bytes_per_position": 2.0}}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps(t))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.profiled_traffic("potential_f32c_kernel", 100, "realistic") == 5000
    assert bench.profiled_traffic("potential_f32c_kernel", 200, "realistic") is None
    assert bench.profiled_traffic("potential_f32c_kernel", 500, "large") == pytest.approx(2000.0)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    assert bench.profiled_traffic("potential_f32c_kernel", 100, "realistic") is None
    assert bench.profiled_traffic("potential_f32c_kernel", 500, "large") is None

