"""The benchmark's host logic without a GPU: the reference arm's JSON line,
the CPU legs' view sequence, the committed-profile lookup, and the
algorithmic-byte formula."""
import json
import os
import sys
import types

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.fixture(scope="module")
def room():
    return bench.make_workload("room", 0)


def test_reference_arm_line(room):
    """The reference arm renders the view sequence of the CPU baseline with
    the oracle and prints the contract's keys; its e2e moves no bytes."""
    args = types.SimpleNamespace(steps=3, warmup=3, impl="reference")
    res = bench.run_reference(args, room)
    json.dumps(res)
    assert res["impl"] == "reference" and res["metric"] == bench.METRIC and res["unit"] == bench.UNIT
    assert res["value"] > 0 and res["steps"] == 3 and res["warmup"] == 3 and res["higher_is_better"] is True
    assert res["config"]["workload"] == room["name"]
    cb = res["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1) and cb["value"] == res["value"]
    assert res["e2e"] == {"value": res["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}


def test_reference_arm_of_gpu_only_workloads():
    args = types.SimpleNamespace(workload="transfer", seed=0, cpu_seconds=1.0)
    res = bench.run_reference_other(args)
    assert res["impl"] == "reference" and "unavailable" in res


def test_cpu_chunks_follow_the_views_in_order():
    """Chunks hold consecutive views of one scene, in order, wrapping around."""
    wk = {"soa": np.array([0, 0, 0, 1, 1, 0, 2, 2, 2, 2], np.uint32)}
    it = bench.cpu_chunks(wk, 3)
    got = [next(it) for _ in range(7)]
    assert got[:5] == [(0, [0, 1, 2]), (1, [3, 4]), (0, [5]), (2, [6, 7, 8]), (2, [9])]
    assert got[5] == (0, [0, 1, 2]) and got[6] == (1, [3, 4])
    for s, sel in got:
        assert all(int(wk["soa"][j]) == s for j in sel) and sel == list(range(sel[0], sel[0] + len(sel)))


def test_recorded_profile_needs_the_current_kernel_sources(tmp_path, monkeypatch):
    """A committed ncu figure is used only when its file names the hash of the
    kernel sources that are built now; comment lines are ignored."""
    (tmp_path / "profiles").mkdir()
    f = tmp_path / "profiles" / "raster_kernel_w.txt"
    f.write_text("# note: dram_bytes_per_launch: 1\nsource_sha256: abc\ndram_bytes_per_launch: 123\n"
                 "warp_instructions_per_launch: 456\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench.recorded_traffic("w") == 123.0
    assert bench.recorded_profile("w", "warp_instructions_per_launch") == 456.0
    assert bench.recorded_profile("w", "missing") is None
    assert bench.recorded_traffic("other") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "def")
    assert bench.recorded_traffic("w") is None


def test_committed_profiles_parse():
    """Every committed raster-stage summary carries a source hash and both
    per-launch figures as numbers."""
    d = os.path.join(bench.ROOT, "profiles")
    files = [x for x in os.listdir(d) if x.startswith("raster_kernel_") and x.endswith(".txt")]
    assert files
    for name in files:
        vals = {}
        with open(os.path.join(d, name)) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    vals[k.strip()] = v.strip()
        assert len(vals["source_sha256"]) == 16, name
        assert float(vals["dram_bytes_per_launch"]) > 0 and float(vals["warp_instructions_per_launch"]) > 0, name


def test_algorithmic_bytes_per_view(room):
    """The per-view algorithmic-byte formula on the vertex-coloured room (no atlas):
    12 B per triangle, 15 B per vertex, 7 B per pixel."""
    sc = room["scenes"][0]
    assert bench.algorithmic_bytes_per_view(sc, 128, 128, False) == 12.0 * sc.n_tris + 15.0 * sc.n_verts + 7.0 * 128 * 128
    assert bench.algorithmic_bytes_per_view(sc, 128, 128, True) - bench.algorithmic_bytes_per_view(sc, 128, 128, False) \
        == 4.0 * 128 * 128
