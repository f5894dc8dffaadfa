"""Host-side helpers of bench.py that shape the JSON line: the kernel names and
dtype label by launch shape, the count of this library's launches per step,
and the gating of the measured DRAM traffic by workload and kernel sources.
CPU only."""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

TC = {"threads": bench.SUBSET_TC, "pixels_per_thread": 1, "full_threads": 2}
GATHER = {"threads": bench.SUBSET_GATHER, "pixels_per_thread": 1, "full_threads": 2}
SFU = {"threads": 256, "pixels_per_thread": 4, "full_threads": 256}


def _args(**kw):
    d = dict(batch=64, P=1152, N=100, c=0.125, iters=30)
    d.update(kw)
    return argparse.Namespace(**d)


def test_kernel_names_follow_the_shape():
    assert bench.kernel_name(TC, "sub").startswith("iter_full_tcws_kernel")
    assert bench.kernel_name(GATHER, "sub").startswith("iter_subset_gather_kernel")
    assert bench.kernel_name(SFU, "sub").startswith("iter_subset_kernel<256, 4>")
    assert bench.kernel_name(TC, "full").startswith("iter_full_tcws_kernel")
    assert bench.kernel_name(SFU, "full") == "iter_full_kernel<256> (CUDA cores, separable)"


def test_dtype_label_says_what_runs():
    assert "split-bf16 x3" in bench.dtype_label(TC)
    assert bench.dtype_label(SFU) == "f32 (f64 e, u)"


def test_launches_per_step():
    # tensor cores: prep + constant tables; 4 per compressed iteration (mask
    # draws, R' tables, kernel, tails); 3 per full pass
    assert bench.launches_per_step(TC, 28, 3) == 1 + 1 + 28 * 4 + 3 * 3
    # gather kernel for the compressed iterations: mask draws, kernel, tails
    assert bench.launches_per_step(GATHER, 28, 3) == 1 + 1 + 28 * 3 + 3 * 3
    # CUDA cores throughout: one launch per iteration, no tables
    assert bench.launches_per_step(SFU, 28, 3) == 1 + 28 + 3


def test_traffic_is_reported_only_for_the_measured_workload_and_sources(monkeypatch):
    sub, full = bench.measured_traffic(_args(), TC)
    key_sub = bench.TRAFFIC_MEASURED[("sub", bench.SUBSET_TC)]
    key_full = bench.TRAFFIC_MEASURED[("full", 2)]
    current = bench.kernel_sha("full")
    assert sub == (key_sub["bytes"] if key_sub["sha"] == current else None)
    assert full == (key_full["bytes"] if key_full["sha"] == current else None)
    # another workload: nothing measured for it
    assert bench.measured_traffic(_args(batch=8), TC) == (None, None)
    assert bench.measured_traffic(_args(c=0.25), TC) == (None, None)
    # a kernel without a capture
    assert bench.measured_traffic(_args(), SFU) == (None, None)
    # sources changed since the capture
    monkeypatch.setattr(bench, "kernel_sha", lambda kind: "0" * 16)
    assert bench.measured_traffic(_args(), TC) == (None, None)
