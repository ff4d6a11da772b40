"""torch.autograd.Function over the fused call: gradients equal the oracle's, and a directional
finite difference of the (FP32) loss agrees with <grad, v> through the autograd API."""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


def test_autograd_matches_oracle_and_finite_difference():
    import torch
    from paper_2012_12686_gb300.autograd import multislice_loss
    dev = torch.device("cuda:0")
    case = C.small_case(N=32, L=4, M=1, B=5, loss="lsq", seed=41)
    case["problem"]["eps"] = 1.0      # smooth amplitude loss, so an FP32 central difference resolves it
    Im = C.measured(case)
    L, gd, gb, gp, gpos = C.oracle_loss_grad(case, Im)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)
    d = t(case["delta"], np.float32).requires_grad_()
    b = t(case["beta"], np.float32).requires_grad_()
    probe = t(case["probe"], np.complex64).requires_grad_()
    pos = t(case["pos"], np.float32).requires_grad_()
    Imt = t(Im, np.float32)
    loss = multislice_loss(d, b, probe, pos, Imt, case["problem"])
    (2.0 * loss).backward()
    assert abs(loss.item() - L) / abs(L) < C.TOL_I
    assert C.rel(d.grad.cpu().numpy() / 2, gd) < C.TOL_G
    assert C.rel(b.grad.cpu().numpy() / 2, gb) < C.TOL_G
    assert C.rel(probe.grad.cpu().numpy() / 2, gp) < C.TOL_G
    assert C.rel(pos.grad.cpu().numpy() / 2, gpos) < C.TOL_G
    # directional derivative along a random delta perturbation (FP32 central difference; the step
    # keeps the loss difference far above FP32 rounding while O(h^2) stays below 1 %)
    g = np.random.default_rng(1)
    v = torch.from_numpy(g.uniform(-1, 1, case["delta"].shape).astype(np.float32)).to(dev)
    h = 5e-5
    with torch.no_grad():
        lp = multislice_loss(d + h * v, b, probe, pos, Imt, case["problem"]).item()
        lm = multislice_loss(d - h * v, b, probe, pos, Imt, case["problem"]).item()
    fd = (lp - lm) / (2 * h)
    an = float((d.grad / 2 * v).sum().item())
    assert abs(fd - an) <= 2e-2 * abs(an), (fd, an)


def test_autograd_only_requested_gradients():
    import torch
    from paper_2012_12686_gb300.autograd import multislice_loss
    dev = torch.device("cuda:0")
    case = C.small_case(N=16, L=2, M=1, B=3, loss="poisson", seed=43)
    Im = C.measured(case)
    d = torch.from_numpy(case["delta"]).to(dev)
    b = torch.from_numpy(case["beta"]).to(dev)
    probe = torch.from_numpy(case["probe"].astype(np.complex64)).to(dev).requires_grad_()
    pos = torch.from_numpy(case["pos"].astype(np.float32)).to(dev)
    loss = multislice_loss(d, b, probe, pos, torch.from_numpy(Im).to(dev), case["problem"])
    loss.backward()
    assert probe.grad is not None and d.grad is None and pos.grad is None
    ref = C.oracle_loss_grad(case, Im)
    assert C.rel(probe.grad.cpu().numpy(), ref[3]) < C.TOL_G
