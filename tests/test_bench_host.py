"""Host logic of bench.py (no GPU): kernel names in the roofline, the committed DRAM capture
lookup, and the whole-job throughput arithmetic."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

SPLIT = {"rows_per_cta": 2, "threads_per_cta": 1024, "visit_order": 0, "split": 1, "up_block": 128,
         "up_threads": 512, "up_rows": 4}


def test_kernel_key_names_the_launched_kernels():
    assert bench.hv_kernel_key("fx64", SPLIT) == \
        "k_hv_fx_wb<2,2> (row pass) + k_hv_fx_up<4,2> (block 128, 512 threads)"
    assert bench.hv_kernel_key("f32", dict(SPLIT, rows_per_cta=4)).startswith("k_hv_f_wb<4> (row pass) + k_hv_up<4,float>")
    assert bench.hv_kernel_key("f64", SPLIT).startswith("k_hv<2,double,false> (row pass)")
    assert bench.hv_kernel_key("fx64", {"rows_per_cta": 2, "split": 0}) == "k_hv_fx<2,2,true>"


def test_traffic_lookup_is_keyed_to_kernel_and_source(monkeypatch):
    cap = json.load(open(os.path.join(ROOT, "profiles", "hv_dram_traffic.json")))
    monkeypatch.setattr(bench, "source_hash", lambda: cap["source_hash"])
    assert bench.ncu_traffic(cap["kernel"]) == cap["dram_bytes_per_launch"]
    assert bench.ncu_traffic(cap["kernel"] + " (another shape)") is None
    monkeypatch.setattr(bench, "source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic(cap["kernel"]) is None


def test_committed_capture_describes_the_default_shape():
    cap = json.load(open(os.path.join(ROOT, "profiles", "hv_dram_traffic.json")))
    assert cap["kernel"] == bench.hv_kernel_key("fx64", SPLIT)
    per = cap["per_kernel_dram_bytes"]
    assert sum(v["read"] + v["write"] for v in per.values()) == pytest.approx(cap["dram_bytes_per_launch"])


def test_job_throughput_is_whole_job():
    # 4 replicas of D = 1e9 states, 10 ms per step: 400 Gstates/s
    assert bench.job_throughput(10 ** 9, 4, 10.0) == pytest.approx(400.0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
