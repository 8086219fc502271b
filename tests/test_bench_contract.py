"""The benchmark's reference arm (the CPU oracle, no GPU) prints one JSON line with the
contract's keys, and the benchmark's operation counts match the implemented formulas."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-seconds", "1"], capture_output=True, text=True, check=True,
                         cwd=ROOT, timeout=600).stdout.strip().split("\n")
    d = json.loads(out[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "system-steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["dtype"] == "f64" and "workload" in d["config"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1


def test_flop_counts():
    # the per-system-step count of the star-relative Hermite step (n = 3: 633; two bodies:
    # one relative body, no pair of planets)
    sys.path.insert(0, ROOT)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_counts", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    f = bench.hermite_flops_per_system_step
    assert f(3) == 3 * (35 * 2 + 6 + 12 + 53) + 3 * 2 * 34 + 6 == 633
    assert f(2) == 3 * (35 + 6) + 3 * 34 + 6 == 231
    assert f(4) - f(3) > f(3) - f(2)  # pairs grow quadratically


def test_scope_table_counts():
    # the scope table's Hermite count, 3 P 58 + 3 n 34, against its own worked figures
    # (n = 3: ~830, n = 8: ~5.7 kflop, n = 15: ~19.8 kflop); the implemented Runge-Kutta
    # count at n = 3 (731) and the MVS count's parts
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_counts2", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    h = bench.scope_hermite_flops
    assert h(3) == 828 and abs(h(8) - 5700) < 50 and abs(h(15) - 19800) < 50
    assert bench.rkck_flops(3) == 731
    assert bench.scope_mvs_flops(8, 1.0, True) == 25 * 28 + 7 * 100 + 48
    assert bench.scope_mvs_flops(8, 2.0, False) == 25 * 21 + 7 * 130 + 48
