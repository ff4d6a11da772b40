"""Near-field free-propagation-distance gradient (dL/dN_F per problem and distance) through
adorym_loss_grad_ext, against the FP64 oracle, on both the shared-memory and the two-pass path."""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,L,B,nd", [(32, 1, 3, 4), (64, 2, 2, 3), (256, 1, 2, 4)])
def test_fresnel_number_gradient(N, L, B, nd):
    import torch
    import oracle
    from paper_2012_12686_gb300.adorym import Engine
    case = C.small_case(N=N, L=L, M=1, B=B, loss="lsq", far=False, n_dist=nd, seed=61 + N)
    Im = C.measured(case)
    ref = oracle.loss_grad(case["problem"], case["delta"], case["beta"], case["probe"], case["pos"], Im, want_nf=True)
    dev = torch.device("cuda:0")
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)
    eng = Engine(0)
    d, b = t(case["delta"], np.float32), t(case["beta"], np.float32)
    oid = eng.register_object(d, b)
    g_nf = torch.zeros((B, nd), dtype=torch.float32, device=dev)
    g_pos = torch.zeros((B, nd, 2), dtype=torch.float32, device=dev)
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    eng.loss_grad_ext(case["problem"], oid, t(case["probe"], np.complex64), t(case["pos"], np.float32),
                      t(Im, np.float32), loss_out=loss, g_pos=g_pos, g_nf=g_nf)
    torch.cuda.synchronize()
    assert abs(loss.item() - ref[0]) <= C.TOL_I * abs(ref[0])
    assert C.rel(g_pos.cpu().numpy(), ref[4]) <= C.TOL_G
    assert C.rel(g_nf.cpu().numpy(), ref[5]) <= C.TOL_G
    eng.close()
