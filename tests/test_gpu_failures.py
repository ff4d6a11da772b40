"""Host-side failure handling: an injected workspace-allocation failure and request cancellation.

An allocation failure is made on the host (the library refuses the next workspace growth before
it touches the device): the call reports ENOMEM and enqueues nothing, the context keeps its
workspace and later calls give the same results as on a context that never failed.  A serving
request cancelled while it waits for admission is never run (its outputs stay untouched and poll
reports ECANCELED); the requests around it complete with their normal results.
"""
import numpy as np
import pytest

from tests import _cases as C

pytestmark = pytest.mark.gpu


def _tensors(case, dev):
    import torch
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)
    return dict(d=t(case["delta"], np.float32), b=t(case["beta"], np.float32), probe=t(case["probe"], np.complex64),
                pos=t(case["pos"], np.float32), Im=t(C.measured(case), np.float32))


def _same(got, want):
    assert abs(got[0] - want[0]) <= 1e-12 * abs(want[0])
    assert C.rel(got[1], want[1]) <= 1e-6 and C.rel(got[2], want[2]) <= 1e-6


def _run(eng, problem, oid, x):
    import torch
    loss = torch.zeros((), dtype=torch.float64, device=x["d"].device)
    gd, gb = torch.zeros_like(x["d"]), torch.zeros_like(x["b"])
    eng.loss_grad(problem, oid, x["probe"], x["pos"], x["Im"], loss, gd, gb, None, None)
    torch.cuda.synchronize()
    return loss.item(), gd.cpu().numpy(), gb.cpu().numpy()


def test_injected_allocation_failure_leaves_context_usable():
    import torch
    from paper_2012_12686_gb300.adorym import Engine, AdorymError, ENOMEM
    dev = torch.device("cuda:0")
    small = C.small_case(N=32, L=4, M=1, B=4, loss="lsq", seed=41, Ly=120, Lx=110)
    large = C.small_case(N=64, L=4, M=1, B=12, loss="lsq", seed=42, Ly=120, Lx=110)
    xs, xl = _tensors(small, dev), _tensors(large, dev)

    ref = Engine(0)                                   # a context that never fails
    r_oid = ref.register_object(xs["d"], xs["b"])
    l_oid = ref.register_object(xl["d"], xl["b"])
    want_s = _run(ref, small["problem"], r_oid, xs)
    want_l = _run(ref, large["problem"], l_oid, xl)
    ref.close()

    eng = Engine(0)
    so, lo = eng.register_object(xs["d"], xs["b"]), eng.register_object(xl["d"], xl["b"])
    eng.inject_alloc_failures(1)
    with pytest.raises(AdorymError) as ei:            # first call needs a workspace: refused
        _run(eng, small["problem"], so, xs)
    assert ei.value.code == ENOMEM and "injected" in str(ei.value)
    _same(_run(eng, small["problem"], so, xs), want_s)   # the injection is spent: the retry runs

    eng.inject_alloc_failures(1)
    _same(_run(eng, small["problem"], so, xs), want_s)   # fits the workspace: no growth, no failure
    with pytest.raises(AdorymError) as ei:            # needs a larger workspace: refused
        _run(eng, large["problem"], lo, xl)
    assert ei.value.code == ENOMEM
    _same(_run(eng, small["problem"], so, xs), want_s)   # the old workspace was kept
    _same(_run(eng, large["problem"], lo, xl), want_l)
    eng.close()


def test_cancel_queued_requests():
    import torch
    from paper_2012_12686_gb300.adorym import Engine, AdorymError, ECANCELED, EINVAL, ENOENT, OK
    dev = torch.device("cuda:0")
    case = C.small_case(N=64, L=8, M=1, B=8, loss="poisson", seed=43, Ly=160, Lx=150)
    x = _tensors(case, dev)
    eng = Engine(0)
    oid = eng.register_object(x["d"], x["b"])
    want = _run(eng, case["problem"], oid, x)

    eng.serve_config(1)                               # one slot: requests run one after another
    n = 8
    outs, tickets = [], []
    for _ in range(n):
        o = dict(loss=torch.full((), -1.0, dtype=torch.float64, device=dev), gd=torch.zeros_like(x["d"]),
                 gb=torch.zeros_like(x["b"]))
        outs.append(o)
        tickets.append(eng.submit(case["problem"], oid, x["probe"], x["pos"], x["Im"], o["loss"], o["gd"], o["gb"]))
    cancelled = []
    for t in reversed(tickets):                       # the last ones are still waiting for admission
        try:
            eng.cancel(t)
            cancelled.append(t)
        except AdorymError as e:
            assert e.code == EINVAL                   # already admitted: runs to completion
    assert tickets[-1] in cancelled
    with pytest.raises(AdorymError) as ei:
        eng.cancel(tickets[-1] + 1000)
    assert ei.value.code == ENOENT
    for t, o in zip(tickets, outs):
        if t in cancelled:
            with pytest.raises(AdorymError) as ei:
                eng.poll(t, 30_000_000)
            assert ei.value.code == ECANCELED
        else:
            assert eng.poll(t, 30_000_000) == OK
    torch.cuda.synchronize()
    for t, o in zip(tickets, outs):
        if t in cancelled:                            # never ran: outputs untouched
            assert o["loss"].item() == -1.0
            assert not o["gd"].any().item()
        else:
            _same((o["loss"].item(), o["gd"].cpu().numpy(), o["gb"].cpu().numpy()), want)
    completed, _ = eng.serve_stats()
    assert completed == n - len(cancelled)
    with pytest.raises(AdorymError) as ei:            # a polled ticket is gone
        eng.cancel(tickets[0])
    assert ei.value.code == ENOENT
    eng.close()
