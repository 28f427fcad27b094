"""Host logic of bench.py (no GPU): the per-entry error measure of reading
R10, the byte accounting behind the roofline, the instruction-issue roofline
of the refine pass, and the DRAM-traffic record that is used only while it
matches the pipeline sources."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_per_entry_error_scales_by_the_larger_diagonal():
    ref = np.array([[[2.0, 0.0], [0.0, 4.0]], [[1.0, 0.1], [0.1, 0.5]]])
    A = ref.copy()
    A[0, 0, 1] += 4e-9   # scale 4 -> 1e-9
    A[1, 1, 1] -= 3e-9   # scale 1 -> 3e-9
    e = bench.per_entry_error(A, ref)
    assert e["entries"] == ["a11", "a12", "a21", "a22"]
    np.testing.assert_allclose(e["max"], [0.0, 1e-9, 0.0, 3e-9], rtol=1e-6, atol=1e-18)
    np.testing.assert_allclose(e["mean"], [0.0, 0.5e-9, 0.0, 1.5e-9], rtol=1e-6, atol=1e-18)
    assert e["max_all"] == pytest.approx(3e-9, rel=1e-6)
    assert e["count"] == 2


def test_pipeline_bytes_per_node():
    """One CG step moves 88.125 B per node pair (stencil 48.125, update 24,
    column 16); a refinement step 128.125 (refine 40.125, update 72, column
    16).  The vectors are float2 pairs (both correctors), the cell bitmask
    1/8 B per node."""
    it = sum(v["iter"] for v in bench.BYTES_PER_NODE.values())
    rf = sum(v["refine"] for v in bench.BYTES_PER_NODE.values())
    assert it == pytest.approx(88.125)
    assert rf == pytest.approx(128.125)
    assert bench.BYTES_PER_NODE["stencil"]["iter"] == pytest.approx(6 * 8 + 1 / 8)


def test_refine_alu_counts_first_refinements_apart():
    prof = {"refine": {"ms": 10.0, "launches": 20}}
    nodes, reals, refines = 1000, 3, 12
    r = bench.refine_alu(prof, refines, reals, nodes, {"sm_mhz": 2000.0})
    work = nodes * (bench.REFINE_INST_PER_NODE * (refines - reals)
                    + bench.REFINE_FIRST_INST_PER_NODE * reals)
    assert r["achieved"] == pytest.approx(work / 0.010)
    assert r["peak"] == pytest.approx(152 * 4 * 32 * 2000e6)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert bench.refine_alu({"refine": {"ms": 1.0, "launches": 0}}, 4, 1, nodes, {}) is None


def test_traffic_record_only_for_matching_sources(monkeypatch):
    path = os.path.join(ROOT, "profiles", "dram_traffic_k_fused_S_U_C_plain_L32_batch128.json")
    rec = json.load(open(path))
    for k in ("stencil", "update_row", "column"):
        assert rec["bytes_per_node"][k] > 0
    monkeypatch.setattr(bench, "source_hash", lambda: rec["source_hash"])
    assert bench.ncu_traffic("stencil") == rec["bytes_per_node"]["stencil"]
    # a change to the pipeline sources makes the record stale: no traffic
    monkeypatch.setattr(bench, "source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic("stencil") is None
