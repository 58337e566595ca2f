"""The reference arm of bench.py (the CPU oracle timed on the host cores) prints
one JSON line with the fields the benchmark contract asks for, on a small
workload and a short time budget (CPU only)."""
import io
import json
import types
from contextlib import redirect_stdout

import bench


def test_reference_arm_prints_one_contract_line(monkeypatch):
    real = bench.cpu_baseline
    monkeypatch.setattr(bench, "cpu_baseline", lambda prob, budget_s=12.0: real(prob, budget_s=0.3))
    args = types.SimpleNamespace(workload="cube_n3_p2", steps=2, warmup=1)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, rank=0, world=1)
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "GDOF/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GDOF/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "cube_n3_p2"


def test_reference_arm_is_silent_on_other_ranks(monkeypatch):
    monkeypatch.setattr(bench, "cpu_baseline", lambda *a, **k: (_ for _ in ()).throw(AssertionError))
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(types.SimpleNamespace(workload="cube_n3_p2", steps=1, warmup=0),
                            rank=1, world=2)
    assert buf.getvalue() == ""
