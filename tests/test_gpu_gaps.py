"""Sparse / variable multislice (per-gap slice spacing) and the slice-gap gradient through
adorym_loss_grad_ext, against the FP64 oracle, on the shared-memory and the two-pass path."""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,L,M,B,far,cp", [(32, 5, 2, 4, True, 0), (64, 7, 1, 3, True, 3), (32, 3, 1, 2, False, 0),
                                           (256, 4, 1, 2, True, 0), (256, 3, 1, 1, False, 1)])
def test_variable_gaps(N, L, M, B, far, cp):
    import torch
    import oracle
    from paper_2012_12686_gb300.adorym import Engine
    case = C.small_case(N=N, L=L, M=M, B=B, loss="poisson" if far else "lsq", far=far, n_dist=2, cp=cp,
                        seed=71 + N + L)
    g = np.random.default_rng(L)
    case["problem"]["gaps"] = list(g.uniform(0.1, 3.0, L - 1))
    Im = C.measured(case)
    ref = oracle.loss_grad(case["problem"], case["delta"], case["beta"], case["probe"], case["pos"], Im,
                           want_gaps=True)
    dev = torch.device("cuda:0")
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)
    eng = Engine(0)
    d, b = t(case["delta"], np.float32), t(case["beta"], np.float32)
    oid = eng.register_object(d, b)
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    gd, gb = torch.zeros_like(d), torch.zeros_like(b)
    gpos = torch.zeros(case["pos"].shape, dtype=torch.float32, device=dev)
    ggap = torch.zeros(L - 1, dtype=torch.float32, device=dev)
    I_out = torch.empty(Im.shape, dtype=torch.float32, device=dev)
    eng.loss_grad_ext(case["problem"], oid, t(case["probe"], np.complex64), t(case["pos"], np.float32),
                      t(Im, np.float32), loss_out=loss, g_delta=gd, g_beta=gb, g_pos=gpos, g_gaps=ggap, I_out=I_out)
    torch.cuda.synchronize()
    I_ref = oracle.forward(case["problem"], case["delta"], case["beta"], case["probe"], case["pos"])
    assert C.rel(I_out.cpu().numpy(), I_ref) <= C.TOL_I
    assert abs(loss.item() - ref[0]) <= C.TOL_I * abs(ref[0])
    assert C.rel(gd.cpu().numpy(), ref[1]) <= C.TOL_G and C.rel(gb.cpu().numpy(), ref[2]) <= C.TOL_G
    assert C.rel(gpos.cpu().numpy(), ref[4]) <= C.TOL_G
    assert C.rel(ggap.cpu().numpy(), ref[-1]) <= C.TOL_G, (ggap.cpu().numpy(), ref[-1])
    eng.close()
