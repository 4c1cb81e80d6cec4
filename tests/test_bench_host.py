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
    assert b == it * (12 * nnz + 24 * N) + solves * (24 * nnz + 96 * N)
    assert f == it * (2 * nnz + 12 * N) + solves * (4 * nnz + 12 * N)
    # two smoothed levels and a dense coarsest level of 20 rows: (n, A, P, Rf, U, Pf)
    levels = [(N, nnz, 3000, 9000, 7000, 9500), (150, 1200, 400, 1300, 1200, 1400), (20, 300, 0, 0, 0, 0)]
    b8, f8 = bench.amg_traffic_model(levels, nnz, N, it, solves, kind=8, sv=4)
    vb = (9000 * 8 + 4 * (4 * N + 150)) + ((7000 + 9500) * 8 + 4 * (2 * N + 150)) \
        + (1300 * 8 + 4 * (4 * 150 + 20)) + ((1200 + 1400) * 8 + 4 * (2 * 150 + 20)) \
        + 4 * (20 * 20 + 2 * 20)
    # finest down: + 4 N (second gathered copy) + 52 N (hook); up: + 12 N; w = A z: 12 nnz + 52 N
    per_it = vb + 4 * N + 52 * N + 12 * N + 12 * nnz + 8 * N + 24 * N + 20 * N
    assert b8 == it * per_it + solves * (24 * nnz + 116 * N)
    # FP32 hierarchy: only the CG's FP64 work counts as FP64 flops
    assert f8 == it * (2 * nnz + 14 * N) + solves * (4 * nnz + 12 * N)
    b64, f64 = bench.amg_traffic_model(levels, nnz, N, it, solves, kind=8, sv=8)
    vf = 2 * (9000 + 7000 + 9500) + 2 * N + 2 * (1300 + 1200 + 1400) + 2 * 150 + 2 * 20 * 20
    assert f64 == it * (vf + 2 * nnz + 14 * N) + solves * (4 * nnz + 12 * N)
