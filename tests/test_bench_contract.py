"""The reference arm of bench.py prints one JSON line with the keys the driver reads, only on rank 0.
It times complete oracle runs of the named workload itself (here the small 2D 64^2 system, so the
test needs neither a GPU nor a minute), on the host's threads."""
import json
import types

import bench


def _args(**kw):
    base = dict(seed=1, config="C1", steps=2, warmup=1)
    base.update(kw)
    return types.SimpleNamespace(**base)


def test_reference_arm_line(monkeypatch, capsys):
    calls = []
    real = bench.oracle_step

    def counted(system):
        calls.append(system.ndof)
        return real(system)

    monkeypatch.setattr(bench, "oracle_step", counted)
    bench.reference_arm(_args(), rank=0, world=1)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1 and calls == [20480] * 3                  # one warm-up, two timed steps
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "s"
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1e3 * d["value"]) < 1e-9 and d["higher_is_better"] is False
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == bench.oracle_threads() >= 1
    assert "C1 system per step" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the same workload description the GPU arm prints for this system
    import battery_system as bs
    assert d["config"]["workload"] == bench.workload_line("C1", bs.assemble("C1", seed=1), 1)


def test_reference_arm_other_ranks_print_nothing(monkeypatch, capsys):
    monkeypatch.setattr(bench, "oracle_step", lambda *a, **k: (_ for _ in ()).throw(AssertionError("ran")))
    bench.reference_arm(_args(), rank=1, world=2)
    assert capsys.readouterr().out == ""
