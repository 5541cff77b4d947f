"""The reference arm of bench.py on the CPU: the oracle, timed as it stands on
a bounded sample of the indentation recipe, prints one JSON line with the
keys the benchmark contract names.  The sample is shrunk here (depth 2 -> 3)
so the test takes seconds; the timed arithmetic is the same code path."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "CPU_SAMPLE", dict(depth_min=2, depth_max=3, dx_region=2.0 / 8,
                                                  points=dict(spacing=1.0 / 8, jitter=1.0 / 32)))
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2",
                                      "--warmup", "3", "--cpu-procs", "1"])
    assert bench.main() == 0
    out = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(out) == 1
    line = json.loads(out[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "Newton it/s"
    assert line["higher_is_better"] is True and line["steps"] == 2
    assert line["value"] > 0 and line["ms_per_step"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert cb["nproc"] >= 1 and cb["cpu_model"] and cb["dof"] > 0
    assert "depth 2->3" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
