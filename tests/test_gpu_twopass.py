"""GPU parity of the two-pass path (tiles of 256, 512 and 1024 pixels) against the FP64 oracle.

Far-field multislice ptychography at 256 (several slices with ragged checkpoint segments, two
probe modes, patches that leave the volume, both losses) and near-field multi-distance
holography at 256 / 512 / 1024, up to the full 8-problem, 4-distance 1024x1024 workload.
"""
import os

import numpy as np
import pytest

from tests import _cases as C
from tests.test_gpu_parity import _compare

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,L,M,B,loss,cp", [
    (256, 3, 1, 2, "poisson", 0),    # segments (2, 1)
    (256, 4, 2, 3, "lsq", 3),        # two modes, segments (3, 1)
    (512, 2, 1, 1, "lsq", 0),
])
def test_twopass_farfield_parity(N, L, M, B, loss, cp):
    case = C.small_case(N=N, L=L, M=M, B=B, loss=loss, cp=cp, seed=N + L + M)
    _compare(case)


@pytest.mark.parametrize("N,L,M,B,nd,loss", [(256, 1, 1, 2, 3, "lsq"), (256, 3, 2, 1, 2, "lsq"),
                                             (512, 2, 1, 1, 4, "lsq"), (256, 2, 1, 2, 2, "poisson")])
def test_twopass_nearfield_parity(N, L, M, B, nd, loss):
    case = C.small_case(N=N, L=L, M=M, B=B, loss=loss, far=False, n_dist=nd, seed=3 + N + L)
    _compare(case)


def test_holography_full_workload():
    """8 problems of 1024x1024, one slice, Fresnel numbers 1e-3..8e-3, per-hologram shifts of
    +-5 px plus a sub-pixel part, LSQ; gradients for the object and the shifts."""
    from paper_2012_12686_gb300 import synth
    w = synth.workload("holo", seed=0)
    workers = min(os.cpu_count() or 1, w["problem"]["B"])
    Im = C.measured_par(w, workers)
    I_ref = C.oracle_forward(w, "", workers)
    ref = C.oracle_loss_grad(w, Im, workers)
    r = C.cuda_run(w, Im, want=(True, False, True))
    errs = {"I": C.rel(r["I"], I_ref), "loss": abs(r["loss"] - ref[0]) / abs(ref[0]),
            "gd": C.rel(r["gd"], ref[1]), "gb": C.rel(r["gb"], ref[2]), "gpos": C.rel(r["gpos"], ref[4])}
    assert errs["I"] <= C.TOL_I and errs["loss"] <= C.TOL_I, errs
    assert max(errs["gd"], errs["gb"], errs["gpos"]) <= C.TOL_G, errs
