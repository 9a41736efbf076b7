"""The benchmark's reference arm on the CPU: `bench.py --impl reference` times
the CPU oracle on the 512x256 workload and prints one JSON line with the keys
of the benchmark contract (one step, no warm-up, to keep the suite short)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, check=True, capture_output=True, text=True, timeout=600)
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "ms" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["relres"] <= 1e-8  # the oracle's direct solve meets the benchmark's tolerance
    assert d["cpu_baseline"]["host"]["cores_available"] >= 1 and d["cpu_baseline"]["host"]["cpu_model"]


def test_benchmark_forms_use_known_options():
    # every form of the timed solve maps onto the library's options (the
    # binding rejects unknown names, which would otherwise surface only on a
    # GPU run of the benchmark)
    sys.path.insert(0, ROOT)
    import bench
    from paper_1501_06211_gb300 import ddel
    fields = {k for k, _ in ddel.ddel_options._fields_}
    names = [f[0] for f in bench.FORMS]
    assert len(set(names)) == len(names) and names[0] == "fp64"
    for name, prec, mode, dtype, desc, theta, extra in bench.FORMS:
        assert prec in (ddel.DDEL_FP64, ddel.DDEL_FP32, ddel.DDEL_MIXED) and mode in (0, 1, 2), name
        assert 0.0 <= theta <= 1.0 and set(extra) <= fields, name
        ddel._set_fields(ddel.ddel_default_options(), dict(precision=prec, schur_mode=mode, theta=theta, **extra))
