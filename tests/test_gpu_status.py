"""Device status word: positions and hologram shifts live in device memory, so the host cannot
validate them; the kernels check them while the call runs and report a bad value through the
call's status word (ADORYM_EDATA) instead of trapping.  Patch corners are clamped, so such a
call touches no memory outside the object and the workspace; a following valid call is unaffected.
"""
import math

import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


def _setup(**kw):
    import torch
    from paper_2012_12686_gb300.adorym import Engine
    case = C.small_case(M=1, seed=21, **kw)
    Im = C.measured(case).astype(np.float32)
    dev = torch.device("cuda:0")
    eng = Engine(0)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)
    d, b = t(case["delta"], np.float32), t(case["beta"], np.float32)
    oid = eng.register_object(d, b)
    return eng, oid, case, d, b, t(case["probe"], np.complex64), t(case["pos"], np.float32), t(Im, np.float32)


def _call(eng, oid, case, d, b, probe, pos, Im, host_loss=False):
    import torch
    loss = torch.zeros((), dtype=torch.float64, device="cpu" if host_loss else d.device)
    gd, gb = torch.zeros_like(d), torch.zeros_like(b)
    eng.loss_grad(case["problem"], oid, probe, pos, Im, loss, gd, gb, torch.zeros_like(probe), torch.zeros_like(pos))
    return float(loss), gd


@pytest.mark.parametrize("kw", [dict(N=32, L=3, B=4), dict(N=256, L=2, B=2),
                                dict(N=32, L=2, B=2, far=False, n_dist=2, loss="lsq")])
def test_bad_positions_set_the_status_word(kw):
    import torch
    from paper_2012_12686_gb300.adorym import AdorymError, EDATA
    eng, oid, case, d, b, probe, pos, Im = _setup(**kw)
    ref_loss, ref_gd = _call(eng, oid, case, d, b, probe, pos, Im)
    assert eng.check() == 0
    flat = pos.view(-1)
    for bad in (math.nan, math.inf, 1e30):
        p_bad = pos.clone()
        p_bad.view(-1)[1] = bad
        _call(eng, oid, case, d, b, probe, p_bad, Im)            # asynchronous: returns at once
        with pytest.raises(AdorymError) as ei:
            eng.check()
        assert ei.value.code == EDATA
        with pytest.raises(AdorymError) as ei:                  # host output: the call reports it
            _call(eng, oid, case, d, b, probe, p_bad, Im, host_loss=True)
        assert ei.value.code == EDATA
    loss, gd = _call(eng, oid, case, d, b, probe, pos, Im)        # valid again, same results
    assert eng.check() == 0
    torch.cuda.synchronize()
    assert abs(loss - ref_loss) <= 1e-12 * abs(ref_loss)
    assert C.rel(gd.cpu().numpy(), ref_gd.cpu().numpy()) <= 1e-6
    assert flat.isfinite().all()
    eng.unregister_object(oid)


def test_serving_reports_bad_positions_at_poll():
    import torch
    from paper_2012_12686_gb300.adorym import AdorymError, EDATA, OK
    eng, oid, case, d, b, probe, pos, Im = _setup(N=64, L=3, B=5)
    p_bad = pos.clone()
    p_bad.view(-1)[0] = math.nan
    outs = [dict(loss=torch.zeros((), dtype=torch.float64, device=d.device), gd=torch.zeros_like(d),
                 gb=torch.zeros_like(b)) for _ in range(2)]
    t_bad = eng.submit(case["problem"], oid, probe, p_bad, Im, outs[0]["loss"], outs[0]["gd"], outs[0]["gb"])
    t_ok = eng.submit(case["problem"], oid, probe, pos, Im, outs[1]["loss"], outs[1]["gd"], outs[1]["gb"])
    with pytest.raises(AdorymError) as ei:
        eng.poll(t_bad, 30_000_000)
    assert ei.value.code == EDATA
    assert eng.poll(t_ok, 30_000_000) == OK
    eng.unregister_object(oid)
