"""Serving loop: requests of uneven tile size, slice count and batch run concurrently (slots,
footprint admission, captured graphs); each result equals the same request run alone and matches
the FP64 oracle (1e-4 for intensities and loss, 1e-3 for gradients).

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
                gb=torch.zeros_like(r["b"]), gp=torch.zeros_like(r["probe"]), gpos=torch.zeros_like(r["pos"]),
                I=torch.empty_like(r["Im"]))


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
                                  o["gb"], o["gp"], o["gpos"], o["I"]))
    first = [eng.poll(t, 0) for t in tickets]
    assert all(c in (OK, ETIMEDOUT) for c in first)
    assert ETIMEDOUT in first                         # the mix is still running right after submission
    for t, c in zip(tickets, first):
        if c == ETIMEDOUT:
            assert eng.poll(t, 30_000_000) == OK
    completed, waits = eng.serve_stats()
    assert completed == len(reqs)
    assert waits >= 1                                 # the budget forced admission waits
    import oracle
    for r in reqs:
        a, m = r["alone"], r["mix"]
        assert abs(a["loss"].item() - m["loss"].item()) <= 1e-12 * abs(a["loss"].item())
        for k in ("gd", "gb", "gp", "gpos"):
            assert C.rel(m[k].cpu().numpy(), a[k].cpu().numpy()) <= 1e-6, (r["case"]["problem"]["N"], k)
        # the served result against the FP64 oracle on the same inputs
        case, Im = r["case"], r["Im"].cpu().numpy()
        I_ref = oracle.forward(case["problem"], case["delta"], case["beta"], case["probe"], case["pos"])
        L, gd, gb, gp, gpos = C.oracle_loss_grad(case, Im)
        errs = {"I": C.rel(m["I"].cpu().numpy(), I_ref), "loss": abs(m["loss"].item() - L) / abs(L),
                "gd": C.rel(m["gd"].cpu().numpy(), gd), "gb": C.rel(m["gb"].cpu().numpy(), gb),
                "gp": C.rel(m["gp"].cpu().numpy(), gp), "gpos": C.rel(m["gpos"].cpu().numpy(), gpos)}
        assert errs["I"] <= C.TOL_I and errs["loss"] <= C.TOL_I, (case["problem"]["N"], errs)
        assert max(errs["gd"], errs["gb"], errs["gp"], errs["gpos"]) <= C.TOL_G, (case["problem"]["N"], errs)
    eng.close()


def test_admission_lets_fitting_requests_overtake_a_waiting_one():
    """With the budget held by a long request, a second large request cannot be admitted; the small
    requests behind it fit and are admitted first (their admission waits are shorter), and the
    large one still completes.  poll_times reports the admission wait and the run time."""
    import torch
    from paper_2012_12686_gb300.adorym import Engine, OK, workspace_bytes
    dev = torch.device("cuda:0")
    big = C.small_case(N=128, L=64, M=1, B=128, loss="poisson", seed=200, Ly=300, Lx=290)
    small = C.small_case(N=32, L=2, M=1, B=4, loss="lsq", seed=201, Ly=300, Lx=290)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)
    eng = Engine(0)
    inputs = []
    for case in (big, small):
        d, b = t(case["delta"], np.float32), t(case["beta"], np.float32)
        inputs.append(dict(case=case, oid=eng.register_object(d, b), probe=t(case["probe"], np.complex64),
                           pos=t(case["pos"], np.float32), Im=t(C.measured(case), np.float32),
                           loss=torch.zeros((), dtype=torch.float64, device=dev)))
    wb = workspace_bytes(big["problem"])
    ws = workspace_bytes(small["problem"])
    eng.serve_config(4, int(wb * 1.5) + 4 * ws)     # one big request at a time, with room for small ones
    order = [0, 0, 1, 1, 1]                          # big, big (waits), three small ones behind it
    tickets = []
    for k in order:
        x = inputs[k]
        tickets.append(eng.submit(x["case"]["problem"], x["oid"], x["probe"], x["pos"], x["Im"], x["loss"]))
    times = []
    for tk in tickets:
        rc, queued, run, admitted = eng.poll_times(tk, 60_000_000)
        assert rc == OK
        assert queued >= 0.0 and run > 0.0 and admitted >= 0.0
        times.append((queued, run, admitted))
    # the second big request waited for the first one's memory; the small ones, submitted after it,
    # were admitted before it
    assert times[1][0] > times[0][0]
    assert max(a for _, _, a in times[2:]) < times[1][2], times
    eng.close()
