"""Host-side arithmetic of the benchmark: the algorithmic work per unit that the roofline
fractions divide by, and the fused-kernel form named beside them."""
import math

import bench


def test_flops_per_unit_at_128():
    # 4 transforms of 128^2 at 5 N^2 log2 N^2 flops, plus 40 flops per pixel
    f = bench.flops_per_unit(128)
    assert f == 4 * 5 * 128 * 128 * 14 + 40 * 128 * 128
    assert abs(f / 1e6 - 5.24) < 0.01


def test_hbm_bytes_per_unit():
    N, cp = 128, 6
    assert bench.bytes_per_unit(N, 32, cp) == 24 * N * N + 16 * N * N / cp
    # two-pass far field: four transforms of two read+write passes, T gather, checkpoints
    assert bench.twopass_bytes_per_unit(N, 32, cp, 1, True) == 128 * N * N + 8 * N * N + 16 * N * N / cp
    # near field: per-call transforms shared by the n_dist holograms
    a = bench.twopass_bytes_per_unit(1024, 1, 1, 4, False)
    assert math.isclose(a, 64 * 1024 ** 2 / 4 + 64 * 1024 ** 2 + 4 * 1024 ** 2 + 24 * 1024 ** 2 / 4)


def test_launch_form_follows_the_batch():
    sms = 152
    assert bench.launch_form(64, 128, 12, sms) == "k_path_pipe"     # tomography batch
    assert bench.launch_form(76, 32, 6, sms) == "k_path_pipe"       # exactly half the SMs
    assert bench.launch_form(128, 32, 6, sms) == "k_path_help"      # multislice batch
    assert bench.launch_form(151, 32, 6, sms) == "k_path_help"
    assert bench.launch_form(152, 32, 6, sms) == "k_path"           # fills the device
    assert bench.launch_form(49, 1, 1, sms) == "k_path"             # one slice: no recompute
    assert bench.launch_form(100, 5, 1, sms) == "k_path"            # checkpoint every slice
