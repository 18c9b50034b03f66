"""The JSON line of bench.py's reference arm (the oracle on the host, no GPU) and the argument
defaults that the benchmark contract fixes."""
import contextlib
import io
import json
import sys

import bench


def test_defaults_keep_the_contract():
    sys_argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse()
    finally:
        sys.argv = sys_argv
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "ours"
    assert a.level is None and a.workload == "solve"


def test_reference_arm_prints_one_line_with_the_contract_keys():
    class Args:
        steps, warmup = 1, 0
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(Args, 0, 1, None)
    lines = [l for l in out.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference"
    assert j["metric"] == "MG Poisson DOF/s to 1e-8 (mixed vs FP64)" and j["unit"] == "DOF/s"
    assert j["higher_is_better"] is True and j["n_gpus"] == 1 and j["steps"] == 1
    assert j["config"]["workload"] == bench.WORKLOAD and j["config"]["dof"] == (2 ** 10 + 1) ** 2
    assert j["value"] > 0 and j["ms_per_step"] > 0
    e2e = j["e2e"]
    assert e2e["value"] == j["value"] and e2e["unit"] == j["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == j["value"] and cb["sample"]


def test_solve_roofline_counts_the_algorithmic_bytes_of_what_the_solve_ran():
    # 3 FP32 cycles of (4 sweeps + 1 defect at 48 B, restriction 5 B, prolongation 9 B) x 4/3,
    # three FP64 defects (two steps and the last check) at 96 B and two updates at 24 B
    r = bench.solve_roofline(1_000_000, 1.0, 1000.0, inner_cycles=3, outer_iters=2)
    per = 3 * (4 * 48 + 48 + 5 + 9) * 4 / 3 + 3 * 96 + 2 * 24
    assert abs(r["bytes_per_dof"] - per) < 1e-9
    assert abs(r["roofline_ms"] - per * 1e6 / 1e12 * 1e3) < 1e-12     # bytes / (GB/s), in ms
    assert abs(r["frac"] - r["roofline_ms"]) < 1e-12                    # measured 1 ms
    f = bench.solve_roofline(1_000_000, 2.0, 1000.0, fp64_cycles=2)     # FP64 MG: no outer steps
    assert abs(f["bytes_per_dof"] - 2 * (4 * 96 + 96 + 10 + 18) * 4 / 3) < 1e-9
    assert abs(f["frac"] - f["roofline_ms"] / 2.0) < 1e-12
