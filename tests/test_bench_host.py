"""CPU checks of bench.py's host-side legs (no GPU): the CPU baseline's JSON
fields, measured on a tiny sample."""
import importlib.util
import pathlib


def _bench():
    path = pathlib.Path(__file__).resolve().parents[1] / "bench.py"
    spec = importlib.util.spec_from_file_location("bench_under_test", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_cpu_baseline_fields():
    bench = _bench()
    line = bench.cpu_oracle_sample(0.2, 0.1)
    assert set(line) >= {"value", "unit", "cores", "kind", "sample", "single_thread"}
    assert line["kind"] == "oracle" and line["unit"] == bench.METRIC
    assert line["value"] > 0 and line["cores"] >= 1
    one = line["single_thread"]
    assert one["cores"] == 1 and one["value"] > 0 and one["unit"] == bench.METRIC
    assert "on 1 thread" in one["sample"] and "10^12" in line["sample"]
