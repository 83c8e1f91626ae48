"""Host logic of bench.py that needs no GPU: the measured-traffic table is
reported only while the kernel's sources are unchanged since the capture,
and the roofline flop counts grow with the mechanism as their derivations
say."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_is_reported_only_for_unchanged_kernel_sources(monkeypatch):
    files = ["kernels_sdc.cu", "chem.cuh"]
    table = {("k_demo", "fp64", "c4"): {"bytes_per_cell": 100.0, "files": files,
                                        "digest": bench._sources_digest(files)},
             ("k_stale", "fp64", "c4"): {"bytes_per_cell": 100.0, "files": files,
                                         "digest": "0000000000000000"}}
    monkeypatch.setattr(bench, "NCU_TRAFFIC", table)
    assert bench.ncu_traffic("k_demo", "fp64", "c4", 1000) == pytest.approx(1e5)
    assert bench.ncu_traffic("k_stale", "fp64", "c4", 1000) is None
    assert bench.ncu_traffic("k_demo", "mixed", "c4", 1000) is None


def test_traffic_table_names_existing_sources():
    for entry in bench.NCU_TRAFFIC.values():
        for f in entry["files"]:
            assert os.path.exists(os.path.join(ROOT, "paper_1309_7327_gb300", "csrc", f)), f
        assert entry["bytes_per_cell"] > 0


def test_flop_counts_grow_with_the_mechanism():
    """Per reaction 34 and per species 43 FP64 flops in the rates; the line
    kernel's count is affine in the species count."""
    assert bench.chem_flops_per_eval(21, 84, 0) - bench.chem_flops_per_eval(21, 83, 0) == 34.0
    assert bench.chem_flops_per_eval(21, 84, 0) - bench.chem_flops_per_eval(20, 84, 0) == 43.0
    # exponentials off the FP64 pipe: 14 flops less per reaction, species and cell
    assert bench.chem_flops_per_eval(21, 84, 0) - bench.chem_flops_per_eval(21, 84, 1) == 14.0 * 106
    a, b, c = (bench.march_flops_per_cell(n) for n in (3, 9, 15))
    assert b - a == c - b > 0
