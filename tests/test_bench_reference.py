"""The reference arm of bench.py (the oracle on the host cores) prints the line the benchmark
contract asks for; a tiny workload stands in for the paper-scale instance so that this runs in
seconds."""
import json

import bench
from paper_2107_01745_b300 import workloads as W


def test_reference_line_has_the_contract_keys(monkeypatch):
    monkeypatch.setattr(W, "paper_scale", lambda seed: W.tiny_fp64(0))

    class Args:
        warmup, steps = 3, 2

    line = bench.run_reference(Args)
    json.dumps(line)  # serialisable as one JSON line
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "ms" and line["higher_is_better"] is False
    assert line["steps"] == 2 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["value"] > 0 and line["ms_per_step"] == line["value"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == bench.WORKLOAD
