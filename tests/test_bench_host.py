"""Host arithmetic of the benchmark line (no GPU): the roofline's algorithmic bytes and the
ALU side computed from the work counters."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_algorithmic_bytes_per_launch():
    n, nnz, k = 10_000_000, 878_570_600, 16
    assert bench.algorithmic_bytes("knn", n, nnz, k) == 16 * n + 8 * n * k == 1_440_000_000
    assert bench.algorithmic_bytes("radius_fill", n, nnz, k) == 16 * n + 8 * (n + 1) + 4 * nnz
    assert bench.algorithmic_bytes("radius_count", n, nnz, k) == 16 * n
    assert bench.algorithmic_bytes("not_a_kernel", n, nnz, k) is None


def test_alu_side_against_the_fp32_lanes():
    counters = {"walks": 10, "expansions": 0, "box_tests": 0, "leaves": 0, "point_tests": 2_000_000_000,
                "needed_tests": 500_000_000, "passed": 0, "whole": 0, "inserts": 0}
    a = bench.alu_side(counters, "sphere", 4.0, 2070.0)
    assert a["tests_per_s"] == pytest.approx(5e11)
    assert a["needed_tests_per_s"] == pytest.approx(1.25e11)
    assert a["fp32_peak"] == pytest.approx(152 * 128 * 2070e6)
    assert a["fp32_frac"] == pytest.approx(5e11 * 9 / (152 * 128 * 2070e6))
    # without a clock sample there is no peak to divide by
    assert "fp32_frac" not in bench.alu_side(counters, "square", 4.0, None)


def test_every_search_kind_has_an_operation_count():
    assert set(bench.FP32_OPS_PER_TEST) == {"sphere", "circle", "cube", "square", "knn"}
    # sphere / kNN: 3 differences, 3 products, 2 sums and the comparison; the 2D and L-inf
    # kernels drop the z product or use maxima
    assert bench.FP32_OPS_PER_TEST["sphere"] == bench.FP32_OPS_PER_TEST["knn"] == 9
    assert bench.FP32_OPS_PER_TEST["square"] < bench.FP32_OPS_PER_TEST["circle"] < 9


def test_serving_trace_follows_its_recipe():
    """Poisson arrivals at the given rate, clouds drawn log-uniformly over the pool, half
    all-points and half 1 % subsets, half sphere and half kNN; seeded."""
    pool = [int(round(x)) for x in np.exp(np.linspace(np.log(50_000), np.log(20_000_000), 16))]
    trace = bench.serve_trace(10.0, 200.0, pool, 77)
    n = len(trace)
    assert abs(n - 2000) < 5 * 2000 ** 0.5  # Poisson count within five standard deviations
    t = [rq["t"] for rq in trace]
    assert t == sorted(t) and 0.0 <= t[0] and t[-1] < 10.0
    assert all(0 <= rq["cloud"] < len(pool) for rq in trace)
    assert 0.45 < sum(rq["subset"] for rq in trace) / n < 0.55
    radius = [rq for rq in trace if rq["search"] == "radius"]
    assert 0.45 < len(radius) / n < 0.55
    assert all(rq["kernel"] == "sphere" and rq["r"] in (0.5, 1.0, 2.0, 3.0) for rq in radius)
    assert all(rq["k"] in (8, 16, 32) for rq in trace if rq["search"] == "knn")
    assert bench.serve_trace(10.0, 200.0, pool, 77) == trace


def _profile_rows(name: str) -> dict:
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles", name)
    rows = {}
    with open(path) as f:
        for line in f:
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) >= 4 and cells[0].startswith("k_"):
                rows.setdefault(cells[0], []).append(cells[1:])
    return rows


def test_roofline_counters_match_the_committed_profile():
    """The DRAM traffic and instruction counts the bench line carries are the ones the
    committed ncu summary reports."""
    rows = _profile_rows("traffic_search_kernels_lidar_tile_10M.md")
    gb = lambda s: float(s.split()[0]) * 1e9  # noqa: E731
    traffic = {"knn": rows["k_knn_group<16>"][0], "radius_count": rows["k_radius_group count (records on)"][0],
               "radius_fill": rows["k_radius_group fill (replay)"][0]}
    for kernel, cells in traffic.items():
        assert bench.NCU_TRAFFIC[kernel]["bytes_per_launch"] == pytest.approx(gb(cells[1]) + gb(cells[2]), rel=0.01)
    inst = {"knn": rows["k_knn_group<16>"][1], "radius_count": rows["k_radius_group count"][0],
            "radius_fill": rows["k_radius_group fill"][0]}
    for kernel, cells in inst.items():
        per_group = float(cells[1].split()[0]) * 1e6 / 62500
        assert bench.NCU_INST_PER_GROUP[kernel]["warp_inst"] == pytest.approx(per_group, rel=0.01)


def test_reference_arm_line_is_measured_and_shares_the_config(capsys, monkeypatch):
    """The reference arm times whole oracle steps (no extrapolation): ms_per_step is the
    measured mean step and value = queries of one step / that time; its config object is
    the GPU arm's, key for key."""
    monkeypatch.setattr(bench, "ORACLE_TILE_POINTS", 3000)
    assert bench.main(["--impl", "reference", "--points", "5000", "--steps", "2", "--warmup", "1"]) == 0
    import json
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] == pytest.approx(2 * 3000 / (line["ms_per_step"] / 1e3))
    assert "extrapolat" not in json.dumps(line) or "nothing extrapolated" in line["cpu_baseline"]["sample"]
    cfg = dict(bench.WORKLOAD, radius={"kernel": "sphere", "r": 2.0})
    assert line["config"] == json.loads(json.dumps(bench.bench_config(cfg, 5000, 1)))
    assert line["cpu_baseline"]["value"] == line["value"] and line["e2e"]["value"] == line["value"]
