"""The bench's reference arm (the FP64 oracle on the host cores) prints the
line the comparison needs: the same metric, unit, config and direction as the
GPU arm, and the cpu_baseline and e2e objects of the contract.  CPU only."""
import json

import bench


def test_reference_arm_line():
    class A:
        steps, warmup = 1, 3
        ref_budget_s = 1.0   # seconds of oracle work per step (the bench sizes it for minutes)
    r = bench.run_reference(A(), rank=0, world=1)
    json.dumps(r)   # serialisable as one JSON line
    assert r["impl"] == "reference"
    assert r["metric"] == bench.METRIC and r["unit"] == "element matrices/s"
    assert r["higher_is_better"] is True and r["n_gpus"] == 1
    assert r["config"] == bench.workload_config(1)
    assert r["value"] > 0 and r["ms_per_step"] > 0
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == r["value"] and cb["sample"]
    e = r["e2e"]
    assert e["value"] == r["value"] and e["unit"] == r["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
