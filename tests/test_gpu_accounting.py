"""Accounting entry points: the library's kernel-launch counter and the measured FP32 FMA peak.

The counter must advance by exactly the kernels one call launches (the bench reports it as the
number of this library's kernels in the timed region), and the FMA throughput kernel must report
a figure of the order of the device's FP32 peak (SM count x 128 lanes x 2 flops x clock).
"""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


def test_launch_counter_counts_one_calls_kernels():
    import torch
    from paper_2012_12686_gb300.adorym import Engine, kernel_launches
    case = C.small_case(N=32, L=5, M=1, B=6, loss="poisson", seed=31)
    Im = C.measured(case).astype(np.float32)
    dev = torch.device("cuda:0")
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)
    d, b = t(case["delta"], np.float32), t(case["beta"], np.float32)
    probe, pos, meas = t(case["probe"], np.complex64), t(case["pos"], np.float32), t(Im, np.float32)
    eng = Engine(0)
    oid = eng.register_object(d, b)

    def call(grads):
        loss = torch.zeros((), dtype=torch.float64, device=dev)
        gd = torch.zeros_like(d) if "object" in grads else None
        gb = torch.zeros_like(b) if "object" in grads else None
        gp = torch.zeros_like(probe) if "probe" in grads else None
        n0 = kernel_launches()
        eng.loss_grad(case["problem"], oid, probe, pos, meas, loss, gd, gb, gp, None)
        torch.cuda.synchronize()
        return kernel_launches() - n0

    # bounding box + transmission + probe transform + fused kernel + probe-gradient transform,
    # + probe-gradient reduction with a probe gradient, + gradient add with an object gradient
    assert call(("object", "probe")) == 7
    assert call(("object",)) == 6
    assert call(()) == 5
    eng.unregister_object(oid)


def test_fp32_peak_is_of_the_order_of_the_device_peak():
    import torch
    from paper_2012_12686_gb300.adorym import fp32_peak
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12   # generous clock bound
    v = fp32_peak(0)
    assert 0.3 * nominal < v < 1.05 * nominal, (v, nominal)
