"""bench.py's JSON contract on the CPU: both arms describe the workload with
the same config, and the reference line carries the keys the contract asks
for (the oracle timing itself is stubbed here; it runs in the reference arm)."""
import importlib.util
import io
import json
import os
import sys
import types
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(b)
    finally:
        sys.argv = argv
    return b


def test_reference_line_and_shared_config(monkeypatch):
    b = load_bench()
    args = types.SimpleNamespace(workload="sphere65536_ks16_U", matvecs=20, form="mixed", steps=2,
                                 warmup=1, gpus=1)
    wl = b.WORKLOADS[args.workload]
    monkeypatch.setattr(b, "cpu_baseline", lambda wl: {"value": 7.0, "cores": 1, "sample": "stub"})
    buf = io.StringIO()
    with redirect_stdout(buf):
        b.run_reference(args, wl, 1, 0)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] == 7.0
    assert line["e2e"] == {"value": 7.0, "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"] == b.workload_config(args, wl, "mixed", 1)  # the GPU arm's config
    # other ranks print nothing and return
    buf = io.StringIO()
    with redirect_stdout(buf):
        b.run_reference(args, wl, 2, 1)
    assert buf.getvalue() == ""
