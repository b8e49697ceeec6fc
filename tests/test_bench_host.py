"""Host-side parts of bench.py (no GPU): which ncu traffic figure a tuned
configuration gets, the host topology used for the no-slip wall list, the
algorithmic byte counts, and the reference arm's JSON line (the CPU oracle on
a small lattice)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _tuned(**kw):
    tf = {"grid": [608, 152, 152], "block": [256, 1024, 1024], "l2_window": "vectors",
          "persistent": False, "cluster": False, "stream_single_reduction": False,
          "update_1red": [1, 152, 1024]}
    tf.update(kw)
    return tf


def test_traffic_is_reported_only_for_captured_configurations():
    textbook, gear, pgear = (t for _, t in bench.TRAFFIC_CAPTURES)
    assert bench.traffic_for(_tuned(), 1024) == textbook
    g = _tuned(stream_single_reduction=True, l2_window="vectors5")
    assert bench.traffic_for(g, 1024) == gear
    # rows per trip do not change the bytes a kernel moves
    assert bench.traffic_for(dict(g, update_1red=[2, 152, 1024]), 1024) == gear
    assert bench.traffic_for(dict(g, update_1red=[2, 608, 256]), 1024) is None
    assert bench.traffic_for(_tuned(persistent=True), 1024) is None
    assert bench.traffic_for(_tuned(persistent_single_reduction=True, persistent=True),
                             1024) is None            # r, p, q window only: not captured
    assert bench.traffic_for(_tuned(persistent_single_reduction=True, persistent=True,
                                    l2_window="vectors5"), 1024) == pgear
    assert bench.traffic_for(_tuned(l2_window="none"), 1024) is None
    assert bench.traffic_for(_tuned(), 512) is None


def test_byte_counts_of_the_fp64_loops():
    assert bench.BYTES_PER_CELL_ITER_METHOD == 108
    assert bench.BYTES_PER_CELL_ITER_FP64 == 117
    assert bench.BYTES_PER_CELL_ITER_FP64_1RED == 125
    assert sum(bench.BYTES_PER_CELL_CP2.values()) == 132 + 204 + 252


def test_roofline_headline_uses_the_method_bytes_whatever_loop_runs():
    nt, iters, secs, peak = 2_093_058, 13_144, 0.6254, 6782.4
    for tf, loop in ((_tuned(), 117), (_tuned(stream_single_reduction=True,
                                              l2_window="vectors5"), 125),
                     (_tuned(persistent=True, persistent_single_reduction=True), 125)):
        r = bench.roofline(tf, nt, iters, secs, peak, "measured", 1024)
        assert r["bytes_per_cell_iter"] == 108
        assert abs(r["achieved"] - 108 * nt * iters / secs / 1e9) < 1e-6
        assert abs(r["frac"] - r["achieved"] / peak) < 1e-12
        assert r["loop_bytes_per_cell_iter"] == loop
        assert abs(r["loop_frac"] / r["frac"] - loop / 108) < 1e-12
        assert r["traffic_source"].startswith("stored") == (r["traffic"] is not None)


@pytest.mark.parametrize("mesh", ["lattice", "graded"])
def test_side_neighbours_match_the_oracle_topology(mesh):
    if mesh == "graded":
        pytest.importorskip("scipy")
        m = synth.graded_mesh(10, seed=1)
    else:
        m = synth.lattice(12, seed=2)
    assert (bench.side_neighbours(m.tri) == oracle.topology(m.tri)).all()


def test_reference_arm_prints_its_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--n", "24", "--steps", "2", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "cell-iters/s"
    assert line["value"] > 0 and line["cpu_baseline"]["cores"] == oracle.omp_threads()
    assert line["cpu_baseline"]["kind"] == "oracle"
    # the same workload label as the GPU arm's line
    assert line["config"]["workload"] == bench.workload_label(24, 1e-10)
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_cpu_baseline_to_tolerance_reaches_rtol_and_gives_a_reference_solution():
    """The GPU line's CPU baseline: the oracle's OpenMP PCG timed to rtol on
    the whole workload, then continued to 1e-13; the reference solution it
    returns is the oracle's (checked against the single-threaded oracle)."""
    p = synth.channel_block_problem(24, seed=0)
    b = synth.rhs(p.mesh, seed=1)
    out, xr = bench.cpu_solve_to_tolerance(p, b, 1e-10)
    assert out["kind"] == "oracle" and out["cores"] == oracle.omp_threads()
    assert out["rel_res"] <= 1e-10 and out["iters"] > 0
    assert abs(out["value"] - p.mesh.nt * out["iters"] / out["time_to_rtol_s"]) < 1e-6 * out["value"]
    assert out["reference_solution"]["rel_res"] <= 1e-12
    xo, _, _ = oracle.solve_problem(p, b, rtol=1e-13)
    assert np.linalg.norm(xr - xo) / np.linalg.norm(xo) < 1e-9
