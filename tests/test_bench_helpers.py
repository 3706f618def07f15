"""Host-side helpers of bench.py (no GPU): the DRAM-traffic record and the workload text."""
import hashlib
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_record_is_current_and_scales_with_factor_bytes():
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    sha = hashlib.sha256(open(os.path.join(ROOT, "paper_2103_05822_gb300", "csrc", "apply.cu"), "rb").read()).hexdigest()
    for kern in ("tucker_aggregate_kernel", "tucker_disaggregate_kernel"):
        ent = rec[kern]
        ratio = ent["dram_bytes_per_factor_byte"]
        assert abs(ratio - (ent["dram_read_sphere10"] + ent["dram_write_sphere10"]) / ent["factor_bytes_sphere10"]) < 1e-12
        # DRAM traffic of a streaming kernel: the factors once, a few percent on top
        assert 1.0 <= ratio < 1.1
        if ent["apply_cu_sha256"] == sha:
            assert bench.traffic_record(kern, 1_000_000) == round(ratio * 1_000_000)
        else:  # counters of another kernel source are not reported
            assert bench.traffic_record(kern, 1_000_000) is None
    assert bench.traffic_record("no_such_kernel", 10) is None


def test_whole_job_value_for_one_gpu():
    assert bench.whole_job_ms(200.0, 100, 1) == (200.0, 2.0)
