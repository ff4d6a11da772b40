"""The stored FP32 floor (tests/golden/fp32_floor.json) behind the full-size gradient bars.

The file is written from the oracle alone by tests/golden/make_fp32_floor.py; these checks keep
it consistent with how it is used: both full-size workloads are present, an FP32 FFT (which rounds
at every butterfly level) is never more accurate than one rounding per transform output, and the
benchmark's parity bars are the GPU tests' bars.
"""
import json
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fp32_floor.json")


def _floor():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_floor_file_covers_the_full_size_workloads():
    fl = _floor()
    assert set(fl["workloads"]) >= {"multislice", "tomo", "farfield256"}
    for name, rec in fl["workloads"].items():
        for mode in ("rounded_transforms", "fp32_fft"):
            for k in ("loss", "gd", "gb", "gp", "gpos"):
                assert 0.0 < rec[mode][k] < 0.1, (name, mode, k)


@pytest.mark.parametrize("name", ["multislice", "tomo", "farfield256"])
def test_fp32_fft_floor_is_at_least_the_rounding_floor(name):
    rec = _floor()["workloads"][name]
    for k in ("gd", "gb", "gp", "gpos"):
        assert rec["fp32_fft"][k] >= rec["rounded_transforms"][k], k


@pytest.mark.parametrize("name", ["multislice", "tomo", "farfield256"])
def test_bench_parity_bars_are_the_gpu_test_bars(name):
    import bench
    from tests.test_gpu_parity import full_size_bars
    assert bench.parity_bars(name) == full_size_bars(name)
