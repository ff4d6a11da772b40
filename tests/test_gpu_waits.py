"""The bounded device-side waits and their fallback branches, made to run out on purpose.

Three waits are bounded, and each has a fallback (adorym_set_wait_limits shortens them):
* a position waiting for a segment a recompute helper holds recomputes it itself;
* a helper waiting for a position's checkpoint stops helping;
* a two-pass column kernel whose tile copy does not complete in time sets the call's status word
  (reported as ADORYM_EDATA) and leaves after waiting for its copies with the default limit.
With the first two limits at zero, the helper path must still give the plain path's results
(bitwise for loss, probe and positions, which have no atomics); with the tile-copy wait given up,
the call must report the timeout and a following call with the default limits must be unaffected.
Small cases only; no wait in these tests is unbounded.
"""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


@pytest.fixture
def limits():
    from paper_2012_12686_gb300.adorym import set_wait_limits, OK
    yield set_wait_limits
    assert set_wait_limits() == OK   # defaults


def _setup(case):
    import torch
    from paper_2012_12686_gb300.adorym import Engine
    dev = torch.device("cuda:0")
    Im = C.measured(case)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)
    d, b = t(case["delta"], np.float32), t(case["beta"], np.float32)
    eng = Engine(0)
    oid = eng.register_object(d, b)
    return eng, oid, d, b, t(case["probe"], np.complex64), t(case["pos"], np.float32), t(Im, np.float32)


def _outs(d, b, probe, pos):
    import torch
    return dict(loss=torch.zeros((), dtype=torch.float64, device=d.device), gd=torch.zeros_like(d),
                gb=torch.zeros_like(b), gp=torch.zeros_like(probe), gpos=torch.zeros_like(pos))


def test_helper_waits_run_out_and_results_do_not_change(limits):
    import torch
    from paper_2012_12686_gb300.adorym import OK
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    B = max(sms // 2 + 8, min(sms - 40, 3 * sms // 4))     # one CTA per position, helpers on idle SMs
    case = C.small_case(N=32, L=9, M=1, B=B, loss="poisson", seed=61, Ly=140, Lx=150)
    eng, oid, d, b, probe, pos, meas = _setup(case)
    served = _outs(d, b, probe, pos)                         # serving: the plain one-CTA path
    tk = eng.submit(case["problem"], oid, probe, pos, meas, served["loss"], served["gd"], served["gb"],
                    served["gp"], served["gpos"])
    assert eng.poll(tk, 30_000_000) == OK
    assert limits(0, 0) == OK
    runs = [_outs(d, b, probe, pos) for _ in range(3)]
    for o in runs:
        eng.loss_grad(case["problem"], oid, probe, pos, meas, o["loss"], o["gd"], o["gb"], o["gp"], o["gpos"])
    assert eng.check() == OK
    torch.cuda.synchronize()
    for o in runs:
        assert o["loss"].item() == served["loss"].item()
        for k in ("gp", "gpos"):
            np.testing.assert_array_equal(o[k].cpu().numpy(), served[k].cpu().numpy(), err_msg=k)
        for k in ("gd", "gb"):
            assert C.rel(o[k].cpu().numpy(), served[k].cpu().numpy()) <= 1e-6, k
    eng.close()


def test_tile_copy_timeout_reports_through_the_status_word(limits):
    import torch
    from paper_2012_12686_gb300.adorym import AdorymError, EDATA, OK, WAIT_DEFAULT, WAIT_GIVE_UP
    case = C.small_case(N=256, L=2, M=1, B=2, loss="lsq", seed=63)
    eng, oid, d, b, probe, pos, meas = _setup(case)
    ref = _outs(d, b, probe, pos)
    eng.loss_grad(case["problem"], oid, probe, pos, meas, ref["loss"], ref["gd"], ref["gb"], ref["gp"], ref["gpos"])
    assert eng.check() == OK
    assert limits(WAIT_DEFAULT, WAIT_DEFAULT, WAIT_GIVE_UP) == OK
    bad = _outs(d, b, probe, pos)
    eng.loss_grad(case["problem"], oid, probe, pos, meas, bad["loss"], bad["gd"], bad["gb"], bad["gp"], bad["gpos"])
    with pytest.raises(AdorymError) as ei:
        eng.check()
    assert ei.value.code == EDATA and "timed out" in str(ei.value)
    assert limits() == OK
    again = _outs(d, b, probe, pos)
    eng.loss_grad(case["problem"], oid, probe, pos, meas, again["loss"], again["gd"], again["gb"], again["gp"],
                  again["gpos"])
    assert eng.check() == OK
    torch.cuda.synchronize()
    assert again["loss"].item() == ref["loss"].item()
    for k in ("gp", "gpos"):
        np.testing.assert_array_equal(again[k].cpu().numpy(), ref[k].cpu().numpy(), err_msg=k)
    eng.close()

