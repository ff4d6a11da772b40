"""Parity-test cases: seeded inputs, FP64 oracle results, CUDA results, error metrics.

Inputs come from ``paper_2012_12686_gb300.synth`` (no method arithmetic); measured intensities
are simulated by the ORACLE's forward model on a second object plus Poisson noise, so no
expected value ever comes from the CUDA path.
"""
from __future__ import annotations

import math
import multiprocessing as mp

import numpy as np

from paper_2012_12686_gb300 import synth

# relative-L2 bars against the FP64 oracle
TOL_I = 1e-4       # intensities and loss
TOL_G = 1e-3       # gradients


def rel(a, b):
    a = np.asarray(a, np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, a.dtype)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))


def small_case(N=32, L=5, M=2, B=7, loss="poisson", far=True, tomo=False, theta=0.0, cp=0, seed=0,
               Ly=None, Lx=None, n_dist=3, outside=True):
    """A small far-field / tomography / near-field problem with ragged edges."""
    g = np.random.default_rng(seed)
    if far:
        Ly = Ly or N + 24
        Lx = Lx or N + 17
        Lz = L
        p = dict(N=N, L=L, M=M, B=B, Lz=Lz, Ly=Ly, Lx=Lx, kdz=synth.KDZ_10NM,
                 lambda_dz_over_px2=0.37, farfield=1, nf=[], loss=loss, eps=1e-6, tomo=int(tomo),
                 theta=theta, checkpoint_every=cp)
        d = synth.ellipsoid_volume((Lz, Ly, Lx), 12, (3, N / 2), (1, max(2, L / 2)), (1e-4, 3e-4), 5e-4, seed + 1)
        b = (d / 8.0).astype(np.float32)
        dm = synth.ellipsoid_volume((Lz, Ly, Lx), 12, (3, N / 2), (1, max(2, L / 2)), (1e-4, 3e-4), 5e-4, seed + 2)
        bm = (dm / 8.0).astype(np.float32)
        probe = synth.probe_phase_screen(N, N / 6.0, 2.0, 1.0, 1e4, seed + 3, M)
        pos = np.stack([g.uniform(-4 if outside else 0, Ly - N + (4 if outside else 0), B),
                        g.uniform(-4 if outside else 0, Lx - N + (4 if outside else 0), B)], 1)
        # keep residuals away from +-1/2 (the rounding boundary of the patch corner)
        fr = pos - np.floor(pos)
        pos = np.where(np.abs(fr - 0.5) < 0.05, pos + 0.1, pos).astype(np.float32)
    else:
        Ly = Lx = N
        Lz = B * L
        nf = [0.02, 0.05, 0.11, 0.3][:n_dist]
        p = dict(N=N, L=L, M=M, B=B, Lz=Lz, Ly=Ly, Lx=Lx, kdz=20.0, lambda_dz_over_px2=0.3,
                 farfield=0, nf=nf, loss=loss, eps=1e-6, tomo=0, theta=0.0, checkpoint_every=cp)
        d = (synth.smooth_field((Lz, N, N), 2.0, 0.0, 0.08, seed + 1))
        b = (synth.smooth_field((Lz, N, N), 2.0, 0.0, 0.004, seed + 2))
        dm = (synth.smooth_field((Lz, N, N), 2.0, 0.0, 0.08, seed + 4))
        bm = b.copy()
        probe = (np.ones((M, N, N)) + 0.05 * (g.standard_normal((M, N, N)) + 1j * g.standard_normal((M, N, N))))
        probe = probe.astype(np.complex64)
        pos = synth.hologram_shifts(B, n_dist, 3, seed + 5)
    return dict(problem=p, delta=d, beta=b, delta_meas=dm, beta_meas=bm, probe=probe, pos=pos,
                photons=1e4 if not far else 1.0)


def measured(case, seed=99):
    """I_meas = Poisson(oracle forward of the second object) (scaled photons for near field)."""
    import oracle
    I = oracle.forward(case["problem"], case["delta_meas"], case["beta_meas"], case["probe"], case["pos"])
    return synth.poisson(I, seed, case.get("photons", 1.0))


def _oracle_chunk(args):
    import oracle
    kind, problem, d, b, probe, pos, Im = args
    if kind == "forward":
        return oracle.forward(problem, d, b, probe, pos)
    return oracle.loss_grad(problem, d, b, probe, pos, Im)


def _chunks(case, workers):
    """Split a batch into per-worker sub-problems.  Far field: positions (whole object each).
    Near field: problems, each chunk with its own slab of the volume."""
    p = dict(case["problem"])
    B = p["B"]
    idx = np.array_split(np.arange(B), min(workers, B))
    out = []
    for c in idx:
        q = dict(p, B=len(c))
        if p["farfield"]:
            out.append((q, case["delta"], case["beta"], case["pos"][c], c))
        else:
            L = p["L"]
            q["Lz"] = len(c) * L
            sl = slice(c[0] * L, (c[-1] + 1) * L)
            out.append((q, case["delta"][sl], case["beta"][sl], case["pos"][c], c))
    return out


def _pool_map(jobs):
    """Spawn pool of single-threaded workers (one BLAS thread each, so they do not oversubscribe)."""
    import os
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(len(jobs)) as pool:
            return pool.map(_oracle_chunk, jobs)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def oracle_forward(case, which="", workers=1):
    """Oracle intensities of the case's object (which="") or of its second object (which="_meas")."""
    import oracle
    d, b = case["delta" + which], case["beta" + which]
    if workers <= 1 or case["problem"]["B"] < 2:
        return oracle.forward(case["problem"], d, b, case["probe"], case["pos"])
    c2 = dict(case, delta=d, beta=b)
    ch = _chunks(c2, workers)
    res = _pool_map([("forward", q, dd, bb, case["probe"], pp, None) for q, dd, bb, pp, _ in ch])
    return np.concatenate(res, 0)


def measured_par(case, workers, seed=99):
    return synth.poisson(oracle_forward(case, "_meas", workers), seed, case.get("photons", 1.0))


def oracle_loss_grad(case, I_meas, workers=1):
    """Oracle loss and gradients; with workers > 1 the batch is split over a spawn pool and the
    per-chunk results are re-weighted (every term is a mean over the batch's pixels)."""
    import oracle
    p = dict(case["problem"])
    B = p["B"]
    if workers <= 1 or B < 2:
        return oracle.loss_grad(p, case["delta"], case["beta"], case["probe"], case["pos"], I_meas)
    ch = _chunks(case, workers)
    res = _pool_map([("loss_grad", q, dd, bb, case["probe"], pp, I_meas[c]) for q, dd, bb, pp, c in ch])
    w = [len(c) / B for *_, c in ch]
    L = sum(wi * r[0] for wi, r in zip(w, res))
    gp = sum(wi * r[3] for wi, r in zip(w, res))
    gpos = np.concatenate([wi * r[4] for wi, r in zip(w, res)], 0)
    if p["farfield"]:
        gd = sum(wi * r[1] for wi, r in zip(w, res))
        gb = sum(wi * r[2] for wi, r in zip(w, res))
    else:   # disjoint slabs
        gd = np.concatenate([wi * r[1] for wi, r in zip(w, res)], 0)
        gb = np.concatenate([wi * r[2] for wi, r in zip(w, res)], 0)
    return L, gd, gb, gp, gpos


def cuda_run(case, I_meas, want=(True, True, True), engine=None):
    """Run forward and loss_grad through the C ABI; returns numpy results."""
    import torch
    from paper_2012_12686_gb300.adorym import Engine
    dev = torch.device("cuda:0")
    eng = engine or Engine(0)
    p = case["problem"]
    d = torch.from_numpy(np.ascontiguousarray(case["delta"])).to(dev)
    b = torch.from_numpy(np.ascontiguousarray(case["beta"])).to(dev)
    probe = torch.from_numpy(np.ascontiguousarray(case["probe"]).astype(np.complex64)).to(dev)
    pos = torch.from_numpy(np.ascontiguousarray(case["pos"]).astype(np.float32)).to(dev)
    Im = torch.from_numpy(np.ascontiguousarray(I_meas).astype(np.float32)).to(dev)
    oid = eng.register_object(d, b)
    I_out = torch.empty(Im.shape, dtype=torch.float32, device=dev)
    eng.forward(p, oid, probe, pos, I_out)
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    gd = torch.zeros_like(d) if want[0] else None
    gb = torch.zeros_like(b) if want[0] else None
    gp = torch.zeros_like(probe) if want[1] else None
    gpos = torch.zeros_like(pos) if want[2] else None
    I2 = torch.empty_like(I_out)
    eng.loss_grad(p, oid, probe, pos, Im, loss, gd, gb, gp, gpos, I2)
    torch.cuda.synchronize()
    eng.unregister_object(oid)
    f = lambda t: None if t is None else t.cpu().numpy()
    return dict(I=f(I_out), I2=f(I2), loss=float(loss.item()), gd=f(gd), gb=f(gb), gp=f(gp), gpos=f(gpos))
