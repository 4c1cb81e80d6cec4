"""Host logic of bench.py (no GPU): the reference arm's JSON line on the small plates workload
follows the contract, and the algorithmic traffic models equal their documented formulas."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_json_contract():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "plates65", "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]
    # both arms print the same workload-only config, and the baseline names its host CPU
    assert set(line["config"]) == {"workload", "n_nodes", "n_cells", "rtol", "precision", "seed"}
    assert line["cpu_baseline"]["cpu_model"] and line["cpu_baseline"]["nproc"] >= 1


def test_traffic_models_match_their_formulas():
    N, nnz, it, solves = 1000, 7000, 10, 2
    info = {"n_nodes": N, "nnz": nnz, "pcg_kind": 2}
    b, f = bench.pcg_traffic_model(info, it, solves)
    assert b == it * (12 * nnz + 24 * N) + solves * (24 * nnz + 80 * N)
    assert f == it * (2 * nnz + 12 * N) + solves * (4 * nnz + 12 * N)
    # two smoothed levels and a dense coarsest level of 20 rows
    levels = [(N, nnz, 3000), (150, 1200, 400), (20, 300, 0)]
    b8, f8 = bench.amg_traffic_model(levels, nnz, N, it, solves, kind=8)
    vb = (48 * nnz + 24 * 3000) + (196 * N + 36 * 150) + (48 * 1200 + 24 * 400) + (196 * 150 + 36 * 20) \
        + (8 * 20 * 20 + 16 * 20)
    assert b8 == it * (12 * nnz + 116 * N + vb) + solves * (24 * nnz + 100 * N)
    vf = 2 * (4 * nnz + 2 * 3000) + 20 * N + 2 * (4 * 1200 + 2 * 400) + 20 * 150 + 2 * 20 * 20
    assert f8 == it * (2 * nnz + 12 * N + vf) + solves * (4 * nnz + 12 * N)
