"""The bench's reference arm (the CPU oracle) on the CPU: one JSON line with
the contract's keys, for a solve workload, and an explicit line for a
workload that is not a solve."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                         cwd=ROOT, capture_output=True, text=True, timeout=600, check=True).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_line_has_the_contract_keys():
    d = _run("--steps", "2", "--warmup", "1", "--workload", "random_sparse_qp")
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["ms_per_step"] == 1e3 / d["value"]
    assert d["config"]["workload"].startswith("random_sparse_qp")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_non_solve_workload_says_so():
    d = _run("--steps", "1", "--warmup", "0", "--workload", "gemm")
    assert d["impl"] == "reference" and "unavailable" in d


def test_roofline_peak_source(tmp_path, monkeypatch):
    """The roofline denominator is the measured value when MEASURED_PEAKS.json
    holds it, else the profiling recipe's fallback, and says which."""
    sys.path.insert(0, ROOT)
    import bench
    f = tmp_path / "peaks.json"
    f.write_text(json.dumps({"hbm_gbs": 6543.2}))
    monkeypatch.setattr(bench, "PEAKS_JSON", str(f))
    assert bench.peak_of("hbm_gbs") == (6543.2, "MEASURED_PEAKS.json hbm_gbs (of measured)")
    v, src = bench.peak_of("bf16_tflops", "burst")
    assert v == 1900.0 and src.endswith("(burst, of fallback)")
    monkeypatch.setattr(bench, "PEAKS_JSON", str(tmp_path / "absent.json"))
    v, src = bench.peak_of("hbm_gbs")
    assert v == 6800.0 and "of fallback" in src


def test_oracle_agreement_against_the_stored_solve():
    """The bench's comparison with the oracle's stored n=1e6 solve: zero for
    the stored values themselves, the planted deviation otherwise."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    ref = json.load(open(bench.REF_JSON))
    x, y = np.zeros(1_000_000), np.zeros(500_000)
    x[ref["x_index"]] = ref["x_value"]
    y[ref["y_index"]] = ref["y_value"]
    a = bench.oracle_agreement(ref, x, y, ref["kkt"]["primal_obj"])
    assert a["obj_rel_err"] == 0 and a["x_max_rel_err"] == 0 and a["y_max_rel_err"] == 0
    k = ref["x_index"][5]
    x[k] += 1e-3 * (1 + abs(ref["x_value"][5]))
    a = bench.oracle_agreement(ref, x, y, ref["kkt"]["primal_obj"] * (1 + 1e-7))
    assert abs(a["x_max_rel_err"] - 1e-3) < 1e-12 and a["y_max_rel_err"] == 0
    assert 0 < a["obj_rel_err"] < 1e-7
