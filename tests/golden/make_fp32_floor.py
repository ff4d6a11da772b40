"""Write tests/golden/fp32_floor.json: the FP32 error floor of the full-size parity workloads.

At full size some gradients of the multislice model are ill-conditioned with respect to FP32
rounding of the wavefields: a far-field pixel that the model predicts dark but that holds a
count gets a large adjoint seed (Eq. poisson_loss, Eq. lsq_loss with eps added), and the value
of a dark pixel is set by the rounding noise of every transform before it.  This script measures
that floor with the oracle alone: it evaluates the oracle's model (oracle.model.loss_grad) with
the three DFT functions the model uses replaced by

  rounded_transforms  the oracle's FP64 DFT, rounded once to complex64 at each transform output
  fp32_fft            an FFT computed in single precision (scipy.fft on complex64 input)

and everything else unchanged in FP64, and stores the relative L2 error of the loss and of every
gradient against the plain FP64 oracle.  The GPU parity bar of a full-size gradient is
max(1e-3, fp32_fft floor): a path that computes every step in FP32 is held to the accuracy of an
FP32 FFT evaluation of the same model.  Inputs are the seeded workloads of
paper_2012_12686_gb300.synth, measured intensities the oracle's forward of the second object plus
Poisson noise, exactly as tests/_cases.py builds them for the GPU parity tests.

    python tests/golden/make_fp32_floor.py [--workers N]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

OUT = os.path.join(HERE, "fp32_floor.json")
WORKLOADS = ("multislice", "tomo", "farfield256")


def _transforms(mode):
    """(dft_minus, dft_plus, idft_minus) for an error model; None: the oracle's own."""
    import oracle.dft as D
    if mode == "rounded_transforms":
        r = lambda f: (lambda x: np.asarray(f(x), np.complex64).astype(np.complex128))
        return r(D.dft_minus), r(D.dft_plus), r(D.idft_minus)
    if mode == "fp32_fft":
        import scipy.fft as sf
        c = lambda x: np.asarray(x, np.complex64)
        return (lambda x: sf.fft2(c(x)).astype(np.complex128),                  # sum x e^{-2 pi i}
                lambda x: sf.ifft2(c(x), norm="forward").astype(np.complex128),  # sum x e^{+2 pi i}
                lambda x: sf.ifft2(c(x)).astype(np.complex128))                  # inverse of dft_minus
    return None


def _job(args):
    mode, problem, d, b, probe, pos, Im = args
    from unittest import mock
    import oracle.model as model
    t = _transforms(mode)
    if t is None:
        return model.loss_grad(problem, d, b, probe, pos, Im)
    with mock.patch.object(model, "dft_minus", t[0]), mock.patch.object(model, "dft_plus", t[1]), \
            mock.patch.object(model, "idft_minus", t[2]):
        return model.loss_grad(problem, d, b, probe, pos, Im)


def _run(pool, mode, w, Im, workers):
    """Oracle loss and gradients over the batch, split by positions (every term is a batch mean)."""
    p = w["problem"]
    B = p["B"]
    chunks = [c for c in np.array_split(np.arange(B), min(workers, B)) if len(c)]
    res = pool.map(_job, [(mode, dict(p, B=len(c)), w["delta"], w["beta"], w["probe"], w["pos"][c], Im[c])
                          for c in chunks])
    wt = [len(c) / B for c in chunks]
    return (sum(x * r[0] for x, r in zip(wt, res)), sum(x * r[1] for x, r in zip(wt, res)),
            sum(x * r[2] for x, r in zip(wt, res)), sum(x * r[3] for x, r in zip(wt, res)),
            np.concatenate([x * r[4] for x, r in zip(wt, res)], 0))


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    import multiprocessing as mp
    import scipy
    from paper_2012_12686_gb300 import synth
    from tests import _cases as C
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    out = {"how": __doc__.split("\n\n")[1].replace("\n", " "),
           "versions": {"numpy": np.__version__, "scipy": scipy.__version__}, "workloads": {}}
    with mp.get_context("spawn").Pool(args.workers) as pool:
        for name in WORKLOADS:
            t0 = time.time()
            w = synth.workload(name, seed=0)
            Im = C.measured_par(w, args.workers)       # oracle forward of the second object + Poisson
            ref = _run(pool, None, w, Im, args.workers)
            rec = {"B": w["problem"]["B"], "N": w["problem"]["N"], "L": w["problem"]["L"],
                   "loss": w["problem"]["loss"], "eps": w["problem"]["eps"]}
            for mode in ("rounded_transforms", "fp32_fft"):
                r = _run(pool, mode, w, Im, args.workers)
                rec[mode] = {"loss": abs(r[0] - ref[0]) / abs(ref[0]), "gd": _rel(r[1], ref[1]),
                             "gb": _rel(r[2], ref[2]), "gp": _rel(r[3], ref[3]), "gpos": _rel(r[4], ref[4])}
            rec["seconds"] = round(time.time() - t0, 1)
            out["workloads"][name] = rec
            print(name, json.dumps(rec), flush=True)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
