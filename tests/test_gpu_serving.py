"""Serving loop: requests of uneven tile size, slice count and batch run concurrently (slots,
footprint admission, captured graphs) and each result equals the same request run alone.

Also: a request larger than the footprint budget is refused at submit (ENOMEM), a budget too
small for all requests at once makes later requests wait for admission, and poll with a zero
timeout reports ETIMEDOUT for work still in flight without blocking.
"""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu

MIX = [dict(N=64, L=4, B=9, loss="poisson"), dict(N=128, L=8, B=5, loss="lsq"), dict(N=32, L=1, B=12, loss="lsq"),
       dict(N=256, L=4, B=3, loss="poisson"), dict(N=128, L=4, B=7, loss="poisson"), dict(N=64, L=8, B=11, loss="lsq"),
       dict(N=32, L=4, B=4, loss="poisson"), dict(N=128, L=1, B=16, loss="lsq")]


def _requests(dev):
    import torch
    reqs = []
    for i, kw in enumerate(MIX):
        case = C.small_case(M=1, seed=100 + i, Ly=300, Lx=290, **kw)
        Im = C.measured(case)
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)
        reqs.append(dict(case=case, d=t(case["delta"], np.float32), b=t(case["beta"], np.float32),
                         probe=t(case["probe"], np.complex64), pos=t(case["pos"], np.float32),
                         Im=t(Im, np.float32)))
    return reqs


def _outs(r):
    import torch
    return dict(loss=torch.zeros((), dtype=torch.float64, device=r["d"].device), gd=torch.zeros_like(r["d"]),
                gb=torch.zeros_like(r["b"]), gp=torch.zeros_like(r["probe"]), gpos=torch.zeros_like(r["pos"]))


def test_alone_equals_in_mix_and_admission():
    import torch
    from paper_2012_12686_gb300.adorym import Engine, ETIMEDOUT, OK, ENOMEM, AdorymError, workspace_bytes
    dev = torch.device("cuda:0")
    reqs = _requests(dev)
    eng = Engine(0)
    for r in reqs:
        r["oid"] = eng.register_object(r["d"], r["b"])
    # alone: direct calls, one at a time
    for r in reqs:
        r["alone"] = _outs(r)
        o = r["alone"]
        eng.loss_grad(r["case"]["problem"], r["oid"], r["probe"], r["pos"], r["Im"], o["loss"], o["gd"], o["gb"],
                      o["gp"], o["gpos"])
    torch.cuda.synchronize()
    # in the mix: a footprint budget that holds only part of the mix at once
    sizes = [workspace_bytes(r["case"]["problem"]) for r in reqs]
    budget = int(max(sizes) * 1.6)
    eng.serve_config(4, budget)
    with pytest.raises(AdorymError) as ei:          # larger than the whole budget: refused at submit
        big = dict(reqs[3]["case"]["problem"], B=64)
        eng.submit(big, reqs[3]["oid"], reqs[3]["probe"], torch.zeros((64, 2), device=dev),
                   torch.zeros((64, 256, 256), device=dev))
    assert ei.value.code == ENOMEM
    tickets = []
    for r in reqs:
        r["mix"] = _outs(r)
        o = r["mix"]
        tickets.append(eng.submit(r["case"]["problem"], r["oid"], r["probe"], r["pos"], r["Im"], o["loss"], o["gd"],
                                  o["gb"], o["gp"], o["gpos"]))
    first = [eng.poll(t, 0) for t in tickets]
    assert all(c in (OK, ETIMEDOUT) for c in first)
    assert ETIMEDOUT in first                         # the mix is still running right after submission
    for t, c in zip(tickets, first):
        if c == ETIMEDOUT:
            assert eng.poll(t, 30_000_000) == OK
    completed, waits = eng.serve_stats()
    assert completed == len(reqs)
    assert waits >= 1                                 # the budget forced admission waits
    for r in reqs:
        a, m = r["alone"], r["mix"]
        assert abs(a["loss"].item() - m["loss"].item()) <= 1e-12 * abs(a["loss"].item())
        for k in ("gd", "gb", "gp", "gpos"):
            assert C.rel(m[k].cpu().numpy(), a[k].cpu().numpy()) <= 1e-6, (r["case"]["problem"]["N"], k)
    eng.close()
