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


def test_default_run_keeps_the_timing_contract(monkeypatch):
    """No flags: one GPU, the 30-lambda sphere, at least three warm-up steps."""
    monkeypatch.setattr("sys.argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.workload == "sphere30" and a.impl == "ours"
    assert a.warmup >= 3 and a.steps >= 50


def test_workload_text_names_the_sizes():
    from paper_2103_05822_gb300.inputs import WORKLOADS
    txt = bench.workload_desc(WORKLOADS["sphere30"], 39, 40, 80, 1034)
    for part in ("30 lambda", "972000 RWGs", "40x80", "1034 groups", "1e-06"):
        assert part in txt, (part, txt)


def test_default_run_replays_a_cuda_graph():
    import sys
    old = sys.argv
    try:
        sys.argv = ["bench.py"]
        assert bench.parse().graph is True
        sys.argv = ["bench.py", "--no-graph"]
        assert bench.parse().graph is False
    finally:
        sys.argv = old


def test_size_quantile_groups_span_the_size_range():
    sizes = [50, 900, 10, 1786, 400, 940, 30]
    pick = bench.size_quantile_groups(sizes, 5)
    assert 2 in pick and 3 in pick  # the smallest and the largest group
    assert len(pick) == 5 and pick == sorted(pick)


def test_group_time_extrapolation_is_exact_for_an_affine_cost():
    """Per-group times t = a + b n_beta: the fit over a sample reproduces the total exactly,
    where plain scaling by the group count would be biased by the sample's sizes."""
    import numpy as np
    rng = np.random.default_rng(3)
    sizes = rng.integers(20, 1800, 500)
    a, b = 2e-4, 1e-6
    pick = bench.size_quantile_groups(sizes, 5)
    total = bench.scale_group_times(sizes[pick], a + b * sizes[pick], sizes)
    assert abs(total - float(np.sum(a + b * sizes))) <= 1e-9 * total
    # a degenerate sample (one size) falls back to the groups' share of RWGs
    assert abs(bench.scale_group_times([100, 100], [1.0, 1.0], [100, 300]) - 4.0) < 1e-12
