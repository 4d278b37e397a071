"""The reference arm of bench.py prints one JSON line with the keys the driver reads, only on rank 0
(the oracle timing is replaced by a fixed sample so the test needs neither a GPU nor a minute)."""
import json
import types

import bench


def _args(**kw):
    base = dict(seed=1, config="C4", steps=2, warmup=1)
    base.update(kw)
    return types.SimpleNamespace(**base)


def test_reference_arm_line(monkeypatch, capsys):
    calls = []

    def fake_sample(seed, target="C4"):
        calls.append((seed, target))
        return 3.0, 24.0, 17, True

    monkeypatch.setattr(bench, "oracle_sample", fake_sample)
    bench.reference_arm(_args(), rank=0, world=1)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1 and len(calls) == 3                      # one warm-up, two timed steps
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "s"
    assert d["value"] == 24.0 and d["ms_per_step"] == 24000.0 and d["higher_is_better"] is False
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == 1 and "64^3" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": 24.0, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("C4")


def test_reference_arm_other_ranks_print_nothing(monkeypatch, capsys):
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: (_ for _ in ()).throw(AssertionError("ran")))
    bench.reference_arm(_args(), rank=1, world=2)
    assert capsys.readouterr().out == ""
