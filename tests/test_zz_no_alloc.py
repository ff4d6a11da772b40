"""adorym_loss_grad_noalloc against adorym_loss_grad, through the C ABI.

The no-allocation entry point serves callers that cannot call cudaMalloc (under a host framework
that owns all device memory through its own pool, in loops that must not allocate): its workspace
is a fixed file-scope device array.  Its results must match the
regular entry point within the parity tolerances, on two calls in a row (the shared array keeps
the previous call's contents), and problems too large for the array must be refused cleanly.
This file is collected last so that a failure here cannot hide the other tests' results.
"""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


def _inputs(case, dev):
    import torch
    Im = C.measured(case)
    t = lambda a, dt=None: torch.from_numpy(np.ascontiguousarray(a if dt is None else a.astype(dt))).to(dev)
    return dict(d=t(case["delta"]), b=t(case["beta"]), probe=t(case["probe"], np.complex64),
                pos=t(case["pos"], np.float32), Im=t(Im, np.float32))


def _outs(x, want_I):
    import torch
    return dict(loss=torch.zeros((), dtype=torch.float64, device=x["d"].device),
                gd=torch.zeros_like(x["d"]), gb=torch.zeros_like(x["b"]), gp=torch.zeros_like(x["probe"]),
                gpos=torch.zeros_like(x["pos"]), I=torch.empty_like(x["Im"]) if want_I else None)


@pytest.mark.parametrize("kw", [dict(N=32, L=5, M=2, B=7, loss="poisson"),
                                dict(N=16, L=9, M=1, B=4, loss="lsq", tomo=True, theta=0.4, Ly=20, Lx=17),
                                dict(N=32, L=2, M=1, B=2, loss="lsq", far=False, n_dist=3)])
def test_noalloc_matches_loss_grad_twice(kw):
    import torch
    from paper_2012_12686_gb300.adorym import Engine, loss_grad_noalloc, OK
    dev = torch.device("cuda:0")
    case = C.small_case(seed=21, **kw)
    x = _inputs(case, dev)
    stream = torch.cuda.current_stream(dev)
    eng = Engine(0, stream.cuda_stream)
    oid = eng.register_object(x["d"], x["b"])
    ref = _outs(x, True)
    eng.loss_grad(case["problem"], oid, x["probe"], x["pos"], x["Im"], ref["loss"], ref["gd"], ref["gb"],
                  ref["gp"], ref["gpos"], ref["I"])
    for call in range(2):
        got = _outs(x, True)
        rc = loss_grad_noalloc(stream.cuda_stream, case["problem"], x["d"], x["b"], x["probe"], x["pos"], x["Im"],
                               got["loss"], got["gd"], got["gb"], got["gp"], got["gpos"], got["I"])
        assert rc == OK, rc
        torch.cuda.synchronize()
        assert abs(got["loss"].item() - ref["loss"].item()) <= C.TOL_I * abs(ref["loss"].item()), call
        assert C.rel(got["I"].cpu().numpy(), ref["I"].cpu().numpy()) <= C.TOL_I, call
        for k in ("gd", "gb", "gp", "gpos"):
            assert C.rel(got[k].cpu().numpy(), ref[k].cpu().numpy()) <= C.TOL_G, (call, k)
    eng.unregister_object(oid)
    eng.close()


def test_noalloc_refuses_problems_beyond_its_scratch():
    import torch
    from paper_2012_12686_gb300 import synth
    from paper_2012_12686_gb300.adorym import loss_grad_noalloc, ETOOBIG, EINVAL, workspace_bytes, \
        NOALLOC_SCRATCH_BYTES
    w = synth.workload("multislice", seed=0)
    assert workspace_bytes(w["problem"]) > NOALLOC_SCRATCH_BYTES
    dev = torch.device("cuda:0")
    p = w["problem"]
    small = lambda *s: torch.zeros(s, dtype=torch.float32, device=dev)
    d = small(p["Lz"], p["Ly"], p["Lx"])
    probe = torch.zeros((1, p["N"], p["N"]), dtype=torch.complex64, device=dev)
    pos = small(p["B"], 2)
    Im = small(p["B"], p["N"], p["N"])
    s = torch.cuda.current_stream(dev).cuda_stream
    assert loss_grad_noalloc(s, p, d, d, probe, pos, Im) == ETOOBIG
    # host pointers are refused (everything must already be on the device)
    assert loss_grad_noalloc(s, p, d, d, probe, pos.cpu(), Im) == EINVAL
    # variable slice spacing is not offered by this entry point
    assert loss_grad_noalloc(s, dict(p, B=2, N=32, gaps=[0.02] * (p["L"] - 1)), d, d, probe[:, :32, :32].contiguous(),
                             pos[:2].contiguous(), Im[:2, :32, :32].contiguous()) == EINVAL


def test_noalloc_reports_bad_positions_through_the_caller_status_word():
    """A non-finite position is seen only by the kernels: they set a bit in the caller's device
    status word (no trap, corners clamped); a valid call after it gives the regular results."""
    import math
    import torch
    from paper_2012_12686_gb300.adorym import Engine, loss_grad_noalloc, OK
    dev = torch.device("cuda:0")
    case = C.small_case(N=32, L=4, M=1, B=3, loss="poisson", seed=23)
    x = _inputs(case, dev)
    stream = torch.cuda.current_stream(dev)
    eng = Engine(0, stream.cuda_stream)
    oid = eng.register_object(x["d"], x["b"])
    ref = _outs(x, False)
    eng.loss_grad(case["problem"], oid, x["probe"], x["pos"], x["Im"], ref["loss"], ref["gd"], ref["gb"],
                  ref["gp"], ref["gpos"])
    status = torch.zeros((), dtype=torch.int32, device=dev)
    bad = x["pos"].clone()
    bad.view(-1)[1] = math.nan
    got = _outs(x, False)
    assert loss_grad_noalloc(stream.cuda_stream, case["problem"], x["d"], x["b"], x["probe"], bad, x["Im"],
                             got["loss"], got["gd"], got["gb"], got["gp"], got["gpos"], status=status) == OK
    torch.cuda.synchronize()
    assert int(status.item()) != 0
    status.zero_()
    got = _outs(x, False)
    assert loss_grad_noalloc(stream.cuda_stream, case["problem"], x["d"], x["b"], x["probe"], x["pos"], x["Im"],
                             got["loss"], got["gd"], got["gb"], got["gp"], got["gpos"], status=status) == OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert abs(got["loss"].item() - ref["loss"].item()) <= C.TOL_I * abs(ref["loss"].item())
    for k in ("gd", "gb", "gp", "gpos"):
        assert C.rel(got[k].cpu().numpy(), ref[k].cpu().numpy()) <= C.TOL_G, k
    eng.unregister_object(oid)
    eng.close()
