"""The plain unfused torch GPU path that the benchmark compares against computes the same loss
and gradients as the FP64 oracle (so the comparison is like for like)."""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


def test_plain_path_matches_oracle():
    import torch
    import bench
    dev = torch.device("cuda:0")
    case = C.small_case(N=32, L=4, M=1, B=5, loss="poisson", seed=51)
    Im = C.measured(case)
    L, gd, gb, gp, gpos = C.oracle_loss_grad(case, Im)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)
    d = t(case["delta"], np.float32).requires_grad_()
    b = t(case["beta"], np.float32).requires_grad_()
    probe = t(case["probe"], np.complex64).requires_grad_()
    pos = t(case["pos"], np.float32).requires_grad_()
    loss, _ = bench.plain_loss(d, b, probe, pos, t(Im, np.float32), case["problem"])
    loss.backward()
    assert abs(loss.item() - L) / abs(L) < C.TOL_I
    for got, ref in ((d.grad, gd), (b.grad, gb), (probe.grad, gp), (pos.grad, gpos)):
        assert C.rel(got.cpu().numpy(), ref) < C.TOL_G
