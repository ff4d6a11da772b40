"""Recompute helpers: a direct call whose batch leaves SMs idle (between half the SM count and the
SM count, one CTA per position) gives those SMs helper CTAs that recompute checkpoint segments.
Which CTA recomputed a segment must not change any result: the same request served (serving
never uses helpers) gives bitwise the same loss, probe and position gradients (no atomics on
those paths) and the same object gradient up to the order of the FP64 atomic additions.  Parity
of the helper path with the oracle is covered by the B = 80 case of test_gpu_parity.py.
"""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


def _batch():
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return max(sms // 2 + 8, min(sms - 40, 3 * sms // 4))   # 2 B > SMs > B: one CTA per position


@pytest.mark.parametrize("far,M,L", [(True, 1, 9), (True, 2, 10), (False, 1, 9)])
def test_helpers_do_not_change_results(far, M, L):
    import torch
    from paper_2012_12686_gb300.adorym import Engine, OK
    dev = torch.device("cuda:0")
    B = _batch()
    case = C.small_case(N=32, L=L, M=M, B=B, loss="poisson", far=far, seed=51 + M + L,
                        Ly=140 if far else None, Lx=150 if far else None)
    Im = C.measured(case)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)
    d, b = t(case["delta"], np.float32), t(case["beta"], np.float32)
    probe, pos, meas = t(case["probe"], np.complex64), t(case["pos"], np.float32), t(Im, np.float32)
    eng = Engine(0)
    oid = eng.register_object(d, b)

    def outs():
        return dict(loss=torch.zeros((), dtype=torch.float64, device=dev), gd=torch.zeros_like(d),
                    gb=torch.zeros_like(b), gp=torch.zeros_like(probe), gpos=torch.zeros_like(pos))

    direct = [outs() for _ in range(2)]
    for o in direct:
        eng.loss_grad(case["problem"], oid, probe, pos, meas, o["loss"], o["gd"], o["gb"], o["gp"], o["gpos"])
    torch.cuda.synchronize()
    served = outs()
    tk = eng.submit(case["problem"], oid, probe, pos, meas, served["loss"], served["gd"], served["gb"],
                    served["gp"], served["gpos"])
    assert eng.poll(tk, 30_000_000) == OK
    torch.cuda.synchronize()
    for o in direct + [served]:
        assert o["loss"].item() == direct[0]["loss"].item()
        for k in ("gp", "gpos"):
            np.testing.assert_array_equal(o[k].cpu().numpy(), direct[0][k].cpu().numpy(), err_msg=k)
        for k in ("gd", "gb"):
            assert C.rel(o[k].cpu().numpy(), direct[0][k].cpu().numpy()) <= 1e-6, k
    eng.close()
