"""bench.py --impl reference: the oracle timed on the host cores prints the
contract's JSON line (rank 0 only), with the CPU baseline of that run and an
end-to-end entry that moves no bytes to or from a device."""
import argparse
import json

import bench


def fake_baseline(seconds=12.0, all_core_seconds=6.0, y_check=None):
    return {"value": 2.5, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "gbs": 16.0,
            "sample": "stub", "all_cores": {"value": 20.0, "unit": "GFLOP/s", "cores": 8}}


def test_reference_line(monkeypatch, capsys):
    monkeypatch.setattr(bench, "cpu_baseline", fake_baseline)
    args = argparse.Namespace(gpus=1, steps=5, warmup=3)
    bench.run_reference(args, 1, 0)
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] == 2.5 and line["unit"] == "GFLOP/s" and line["higher_is_better"] is True
    assert line["e2e"] == {"value": 2.5, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == 2.5
    assert line["config"]["workload"] == bench.WORKLOAD
    # ms per step is one 192^3 product at that rate
    assert abs(line["ms_per_step"] - 2.0 * 189119224 / 2.5e9 * 1e3) < 1e-9


def test_reference_line_on_rank_0_only(monkeypatch, capsys):
    monkeypatch.setattr(bench, "cpu_baseline", fake_baseline)
    bench.run_reference(argparse.Namespace(gpus=2, steps=5, warmup=3), 2, 1)
    assert capsys.readouterr().out == ""
