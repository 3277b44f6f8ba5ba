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
    assert line["steps_measured"] == 2 and "all 2" in line["steps_note"]
    # both arms print the same workload description
    p = W.tiny_fp64(0)
    n = p.tree.num_nonleaf * p.nu + (p.tree.num_nodes - 1) * p.nx
    assert line["config"] == bench._config(1, p.num_dual, n)


def test_reference_arm_stops_measuring_at_its_budget(monkeypatch):
    monkeypatch.setattr(W, "paper_scale", lambda seed: W.tiny_fp64(0))
    monkeypatch.setattr(bench, "REF_BUDGET_S", 0.0)

    class Args:
        warmup, steps = 3, 4

    line = bench.run_reference(Args)
    assert line["steps_measured"] == 1 and "budget" in line["steps_note"]
