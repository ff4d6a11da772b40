"""The C ABI library builds, loads without a GPU and exports every function include/adorym.h declares;
argument validation that needs no device is exercised through adorym_workspace_bytes."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "adorym.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(adorym_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2012_12686_gb300 import build
    build.build()
    from paper_2012_12686_gb300 import adorym
    return adorym.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    from paper_2012_12686_gb300 import adorym
    assert set(adorym.EXPORTS) == set(names)


def _problem(**kw):
    from paper_2012_12686_gb300.adorym import Problem
    d = dict(N=128, L=32, M=1, B=128, Ly=512, Lx=512, Lz=32, kdz=253.35, lambda_dz_over_px2=0.0248,
             farfield=1, nf=[], loss="poisson", eps=1e-6)
    d.update(kw)
    return Problem.of(d)


def test_workspace_planning_and_validation(lib):
    from paper_2012_12686_gb300.adorym import workspace_bytes, AdorymError
    ws = workspace_bytes(_problem())
    # checkpoints (6) + segment (6) + park + far field + probe partials: ~15 fields of 128 KB per
    # position, plus the complex64 transmission volume (512 x 512 x 32) and the two FP64
    # object-gradient accumulators
    T = 512 * 512 * 32 * (8 + 16)
    assert T + 128 * 14 * 128 * 1024 < ws < T + 128 * 20 * 128 * 1024
    ws1 = workspace_bytes(_problem(checkpoint_every=1))
    assert ws1 > ws
    for bad in (dict(N=100), dict(N=2048), dict(Lz=31), dict(B=0), dict(M=0), dict(loss=7), dict(eps=-1.0),
                dict(checkpoint_every=33), dict(farfield=0, nf=[0.1], Ly=128, Lx=128, Lz=128 * 32 + 1),
                dict(farfield=0, nf=[], Ly=128, Lx=128, Lz=128 * 32), dict(tomo=1, theta=float("nan"))):
        with pytest.raises(AdorymError):
            workspace_bytes(_problem(**bad))
    near = workspace_bytes(_problem(farfield=0, nf=[1e-3, 2e-3], Ly=128, Lx=128, Lz=128 * 32))
    assert near > 0


def test_null_context_is_rejected(lib):
    assert lib.adorym_forward(None, None, 0, None, None, None) != 0
    assert lib.adorym_poll(None, 1, 0) != 0
    from paper_2012_12686_gb300.adorym import EINVAL
    assert lib.adorym_cancel(None, 1) == EINVAL
    assert lib.adorym_inject_alloc_failures(None, 1) == EINVAL
    assert lib.adorym_check(None) == EINVAL
    assert lib.adorym_last_error(None) == b"null context"


def test_wait_limits_are_validated(lib):
    """adorym_set_wait_limits (test hook of the bounded device waits) checks its arguments on the host."""
    from paper_2012_12686_gb300.adorym import set_wait_limits, EINVAL, OK, WAIT_DEFAULT, WAIT_GIVE_UP
    assert set_wait_limits(-3, WAIT_DEFAULT, WAIT_DEFAULT) == EINVAL
    assert set_wait_limits(WAIT_DEFAULT, -3, WAIT_DEFAULT) == EINVAL
    assert set_wait_limits(WAIT_DEFAULT, WAIT_DEFAULT, -3) == EINVAL
    assert set_wait_limits(0, 0, WAIT_GIVE_UP) == OK
    assert set_wait_limits() == OK
