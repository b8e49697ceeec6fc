"""Host-side parts of bench.py (no GPU): which ncu traffic figure a tuned
configuration gets, the host topology used for the no-slip wall list, the
algorithmic byte counts, and the reference arm's JSON line (the CPU oracle on
a small lattice)."""
import json
import os
import subprocess
import sys

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
    assert bench.traffic_for(_tuned(), 1024) == bench.TRAFFIC_PER_ITER_N1024
    gear = _tuned(stream_single_reduction=True, l2_window="vectors5")
    assert bench.traffic_for(gear, 1024) == bench.TRAFFIC_PER_ITER_N1024_1RED
    # rows per trip do not change the bytes a kernel moves
    assert bench.traffic_for(dict(gear, update_1red=[2, 152, 1024]), 1024) == \
        bench.TRAFFIC_PER_ITER_N1024_1RED
    assert bench.traffic_for(dict(gear, update_1red=[2, 608, 256]), 1024) is None
    assert bench.traffic_for(_tuned(persistent=True), 1024) is None
    assert bench.traffic_for(_tuned(l2_window="none"), 1024) is None
    assert bench.traffic_for(_tuned(), 512) is None


def test_byte_counts_of_the_two_fp64_loops():
    assert bench.BYTES_PER_CELL_ITER_FP64 == 117
    assert bench.BYTES_PER_CELL_ITER_FP64_1RED == 125
    assert sum(bench.BYTES_PER_CELL_CP2.values()) == 132 + 204 + 252


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
                        "--n", "24", "--steps", "1", "--warmup", "0", "--cpu-iters", "20"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "cell-iters/s"
    assert line["value"] > 0 and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
