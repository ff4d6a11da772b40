"""Regularizers (Table regularizers: l1, reweighted l1, TV) through the C ABI against the oracle."""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(5, 37, 29), (32, 64, 64)])
def test_regularize_matches_oracle(shape):
    import torch
    from oracle import regularizers as R
    from paper_2012_12686_gb300.adorym import Engine
    g = np.random.default_rng(shape[0])
    d = g.uniform(-1e-5, 1e-5, shape).astype(np.float32)
    b = (0.1 * g.uniform(-1e-5, 1e-5, shape)).astype(np.float32)
    snap_d = g.uniform(-1e-5, 1e-5, shape).astype(np.float32)
    snap_b = g.uniform(-1e-6, 1e-6, shape).astype(np.float32)
    dev = torch.device("cuda:0")
    eng = Engine(0)
    td, tb = torch.from_numpy(d).to(dev), torch.from_numpy(b).to(dev)
    oid = eng.register_object(td, tb)
    sid = eng.register_object(torch.from_numpy(snap_d).to(dev), torch.from_numpy(snap_b).to(dev))
    wd, wb = torch.empty_like(td), torch.empty_like(tb)
    eng.l1_weights(sid, 1e-7, wd, wb)
    rw_d, rw_b = R.l1_weights(snap_d, 1e-7), R.l1_weights(snap_b, 1e-7)
    assert C.rel(wd.cpu().numpy(), rw_d) < 1e-5 and C.rel(wb.cpu().numpy(), rw_b) < 1e-5
    kw = dict(alpha_delta=0.3, alpha_beta=2.0, gamma_tv=0.7)
    ref = R.regularize(d, b, w_delta=rw_d, w_beta=rw_b, **kw)
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    gd, gb = torch.zeros_like(td), torch.zeros_like(tb)
    eng.regularize(oid, w_delta=wd, w_beta=wb, loss_out=loss, g_delta=gd, g_beta=gb, **kw)
    torch.cuda.synchronize()
    assert abs(loss.item() - ref[0]) <= 1e-5 * abs(ref[0])
    assert C.rel(gd.cpu().numpy(), ref[1]) <= 1e-5
    assert C.rel(gb.cpu().numpy(), ref[2]) <= 1e-5
    host = np.zeros(1)
    eng.regularize(oid, loss_out=host, alpha_delta=1.0)            # plain l1, host loss, no gradient
    assert abs(host[0] - np.mean(np.abs(d.astype(np.float64)))) <= 1e-6 * host[0]
    eng.close()
