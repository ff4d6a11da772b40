"""Benchmark: multislice ptychography loss + gradient (forward + adjoint) throughput on GB300.

Workload (one step = one minibatch): 512x512x32 object of random ellipsoids, 128x128 probe
with a random phase screen, 32x32 raster at 12 px with +-0.5 px jitter (1024 positions,
minibatches of 128), 0.248 nm / 10 nm voxels, Poisson loss, gradients w.r.t. delta, beta,
probe and positions, sqrt(L) checkpointing.  Unit of work: one (position, slice) forward +
adjoint evaluation; one step is 128 x 32 = 4096 units.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Multi-GPU (torchrun): every rank evaluates its own minibatches
(the positions of an epoch are independent units), no collective on the data path, weak
scaling; the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "position·slice fwd+adjoint evals/s vs plain GPU path at ≤1e-4 rel err; p50/p99"
UNIT = "position·slice/s"
WORKLOAD = "multislice"
WORKLOAD_DESC = ("3D multislice far-field ptychography: object 512x512x32 (ellipsoids, delta<=5e-6, beta=delta/10), "
                 "probe 128x128 with phase screen, 32x32 raster step 12 px +-0.5 px jitter, minibatch 128, "
                 "Poisson loss, grads delta/beta/probe/positions, sqrt-checkpointing (every 6 of 32 slices)")
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def flops_per_unit(N: int) -> float:
    """Algorithmic FP32 flops per (position, slice): 4 FFTs of N^2 (5 N^2 log2 N^2 each: forward
    propagation 2, adjoint 2; checkpoint recompute not credited) + ~40 flops/pixel elementwise."""
    return 4 * 5 * N * N * math.log2(N * N) + 40 * N * N


def bytes_per_unit(N: int, L: int, cp: int) -> float:
    """Algorithmic HBM bytes per (position, slice): delta+beta patch read (8 N^2), object-gradient
    read-modify-write (16 N^2), checkpoint write+read (16 N^2 / cp)."""
    return 8 * N * N + 16 * N * N + 16 * N * N / cp


def launch_form(B: int, L: int, cp: int, sms: int) -> str:
    """Fused-kernel form the library launches for a direct loss_grad call with uniform slice
    spacing (N <= 128): two-CTA clusters for batches of at most half the SM count, recompute
    helpers on the idle SMs for batches below the SM count, else one CTA per position; the two
    recompute forms only when the sweep has more than one checkpoint segment of several slices."""
    ncp = -(-L // cp)
    if ncp > 1 and cp > 1 and 2 * B <= sms:
        return "k_path_pipe"
    if ncp > 1 and cp > 1 and B < sms:
        return "k_path_help"
    return "k_path"


def twopass_bytes_per_unit(N: int, L: int, cp: int, nd: int, far: bool) -> float:
    """Algorithmic HBM bytes per unit of the two-pass structure: every 2-D transform of an N x N
    complex64 field in HBM needs two read+write passes (32 N^2 bytes).  Far field per (position,
    slice): forward + adjoint propagation (4 transforms) + T gather (8 N^2) + checkpoint (16 N^2 /
    cp).  Near field per hologram: the exit-wave transform and the final inverse shared by nd
    holograms, one inverse and one forward transform per hologram, I_meas read (4 N^2), T and the
    object-gradient update per slice shared by nd."""
    if far:
        return 4 * 32 * N * N + 8 * N * N + 16 * N * N / cp
    return (2 * 32 * N * N) / nd + 2 * 32 * N * N + 4 * N * N + L * (8 + 16) * N * N / nd


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="adorym_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={SMI_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            try:
                os.remove(self.path)
            except OSError:
                pass
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            with open(self.path) as fh:
                for line in fh:
                    f = [t.strip() for t in line.split(",")]
                    if len(f) >= 9 and f[1].replace(".", "").isdigit():
                        rows.append(f)
            os.remove(self.path)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


# ----------------------------------------------------------------------------- oracle timing
def _oracle_one(args):
    import oracle
    problem, d, b, probe, pos, Im = args
    t = time.perf_counter()
    oracle.loss_grad(problem, d, b, probe, pos, Im)
    return time.perf_counter() - t


def _oracle_one_kept(args):
    """The oracle's outputs for one task: (0, (intensities, (loss, gd, gb, gp, gpos)))."""
    import oracle
    problem, d, b, probe, pos, Im = args
    r = oracle.loss_grad(problem, d, b, probe, pos, Im)
    return 0.0, (oracle.forward(problem, d, b, probe, pos), r)


def _oracle_fwd(args):
    import oracle
    problem, d, b, probe, pos = args
    return oracle.forward(problem, d, b, probe, pos)


def oracle_measured(w, n_pos: int, workers: int, seed: int = 99, pool=None):
    """Measured intensities of the first n_pos positions made by the oracle alone: its forward
    model of the workload's second object (delta_meas, beta_meas) plus Poisson noise, one
    position per task on its patch.  [n_pos, N, N] float32."""
    import numpy as np
    from paper_2012_12686_gb300 import synth
    N = w["problem"]["N"]
    p = dict(w["problem"], B=1, Ly=N, Lx=N)
    jobs = []
    for i in range(n_pos):
        pos = np.asarray(w["pos"][i:i + 1], np.float64)
        c = np.floor(pos[0] + 0.5).astype(int)
        jobs.append((p, _crop(w["delta_meas"], c, N), _crop(w["beta_meas"], c, N), w["probe"], pos - c))
    own = pool is None
    if own:
        pool = oracle_pool(workers)
    try:
        I = np.concatenate(pool.map(_oracle_fwd, jobs), 0)
    finally:
        if own:
            pool.close()
            pool.join()
    return synth.poisson(I, seed, w.get("photons", 1.0)).astype(np.float32)


def _crop(vol, c, N):
    """vol[:, c0:c0+N, c1:c1+N] with zeros outside the volume (the patch the oracle reads)."""
    import numpy as np
    out = np.zeros((vol.shape[0], N, N), vol.dtype)
    ya, yb = max(c[0], 0), min(c[0] + N, vol.shape[1])
    xa, xb = max(c[1], 0), min(c[1] + N, vol.shape[2])
    if ya < yb and xa < xb:
        out[:, ya - c[0]:yb - c[0], xa - c[1]:xb - c[1]] = vol[:, ya:yb, xa:xb]
    return out


def oracle_pool(workers: int):
    """Spawn pool of single-threaded oracle workers (one BLAS thread each)."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    return mp.get_context("spawn").Pool(workers)


def oracle_sample(w, I_meas_np, n_pos: int, workers: int, pool=None, keep=False):
    """Time the FP64 oracle (as it stands) on n_pos positions of the minibatch, one position per
    task, over a spawn pool of `workers` single-threaded processes.  Returns (wall s, positions),
    and with keep=True also the per-position outputs [(corner, I, (loss, gd, gb, gp, gpos))]: each
    task is the one-position problem on its patch (patch frame, loss normalised by N^2)."""
    import numpy as np
    N = w["problem"]["N"]
    p = dict(w["problem"], B=1, Ly=N, Lx=N)
    jobs, corners = [], []
    for i in range(n_pos):
        # each task gets only its patch of the volume (the oracle reads nothing else for it)
        pos = np.asarray(w["pos"][i:i + 1], np.float64)
        c = np.floor(pos[0] + 0.5).astype(int)
        crop = []
        for vol in (w["delta"], w["beta"]):
            out = np.zeros((vol.shape[0], N, N), vol.dtype)
            ya, yb = max(c[0], 0), min(c[0] + N, vol.shape[1])
            xa, xb = max(c[1], 0), min(c[1] + N, vol.shape[2])
            out[:, ya - c[0]:yb - c[0], xa - c[1]:xb - c[1]] = vol[:, ya:yb, xa:xb]
            crop.append(out)
        jobs.append((p, crop[0], crop[1], w["probe"], pos - c, I_meas_np[i:i + 1]))
        corners.append(c)
    own = pool is None
    if own:
        pool = oracle_pool(workers)
    try:
        pool.map(_oracle_one, jobs[:workers])          # warm: imports, DFT matrices
        t = time.perf_counter()
        pool.map(_oracle_one, jobs)
        wall = time.perf_counter() - t
        # outputs for the parity check: a second, untimed pass that also returns them
        res = pool.map(_oracle_one_kept, jobs) if keep else None
    finally:
        if own:
            pool.close()
            pool.join()
    if not keep:
        return wall, n_pos
    return wall, n_pos, [(c, r[1][0], r[1][1]) for c, r in zip(corners, res)]


def oracle_batch_parity(kept, shape, B, I_gpu, loss_gpu, gd_gpu, gb_gpu, gp_gpu, gpos_gpu):
    """Relative L2 errors of one GPU loss_grad call on a minibatch against the oracle's outputs
    for the same B positions (from oracle_sample(keep=True)), assembled into the batch's frame: the
    per-position losses and probe / position gradients are rescaled from a one-position mean to
    the batch mean (1/B), the patch gradients are added into the volume at each position's corner
    (pixels outside the volume dropped)."""
    import numpy as np
    import oracle
    Lz, Ly, Lx = shape
    gd = np.zeros(shape)
    gb = np.zeros(shape)
    I = np.stack([k[1][0] for k in kept])
    loss = sum(k[2][0] for k in kept) / B
    gp = sum(k[2][3] for k in kept) / B
    gpos = np.concatenate([k[2][4] for k in kept], 0) / B
    for c, _, r in kept:
        oracle.model.put_chunk_T(gd, c, r[1] / B)
        oracle.model.put_chunk_T(gb, c, r[2] / B)

    def rel(a, b):
        a = np.asarray(a)
        return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))
    return {"I": rel(I_gpu, I), "loss": abs(loss_gpu - loss) / abs(loss), "gd": rel(gd_gpu, gd),
            "gb": rel(gb_gpu, gb), "gp": rel(gp_gpu, gp), "gpos": rel(gpos_gpu, gpos)}


# ----------------------------------------------------------------------------- multi-rank host logic
def rank_batches(rank: int, world: int, start: int, count: int, nb: int):
    """Minibatch indices a rank evaluates at steps start..start+count-1: at every step the ranks
    take distinct minibatches of the epoch (positions are independent units, no collective)."""
    return [(rank + (start + k) * world) % nb for k in range(count)]


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank number over the process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- plain GPU path
def plain_loss(delta, beta, probe, pos, I_meas, p):
    """The plain, unfused GPU formulation the fused engine is compared with: the same far-field
    multislice model written with torch.fft and elementwise tensor ops, differentiated by torch
    autograd (every slice's intermediates kept), one request at a time.  Measurement baseline
    only; it is not part of the engine."""
    import torch
    N, L, kdz, c = p["N"], p["L"], p["kdz"], p["lambda_dz_over_px2"]
    dev = delta.device
    p0 = torch.floor(pos.detach() + 0.5)
    dr = pos - p0
    f = torch.fft.fftfreq(N, device=dev)
    ramp = torch.exp(-2j * math.pi * (dr[:, 0, None, None] * f[None, :, None] + dr[:, 1, None, None] * f[None, None, :]))
    psi = torch.fft.ifft2(torch.fft.fft2(probe)[None] * ramp[:, None])            # [B, M, N, N]
    if p.get("tomo"):
        delta, beta = plain_rotate(delta, p["theta"]), plain_rotate(beta, p["theta"])
    pad = N
    dp = torch.nn.functional.pad(delta, (pad, pad, pad, pad))
    bp = torch.nn.functional.pad(beta, (pad, pad, pad, pad))
    iy = (p0[:, 0].long() + pad)[:, None] + torch.arange(N, device=dev)[None]
    ix = (p0[:, 1].long() + pad)[:, None] + torch.arange(N, device=dev)[None]
    H = torch.exp(1j * math.pi * c * (f[:, None] ** 2 + f[None, :] ** 2))
    for j in range(L):
        od = dp[j][iy[:, :, None], ix[:, None, :]]
        ob = bp[j][iy[:, :, None], ix[:, None, :]]
        phi = psi * torch.exp(-kdz * ob + 1j * kdz * od)[:, None]
        if j < L - 1:
            psi = torch.fft.ifft2(torch.fft.fft2(phi) * H)
    Psi = torch.fft.ifft2(phi) * N
    I = (Psi.real ** 2 + Psi.imag ** 2).sum(1)
    eps = p["eps"]
    if p["loss"] == "lsq":
        terms = (torch.sqrt(I + eps) - torch.sqrt(I_meas + eps)) ** 2
    else:
        terms = I - I_meas * torch.log(I + eps)
    return terms.mean(), I


def plain_rotate(vol, theta):
    """Bilinear rotation about y in the x-z plane with torch indexing (differentiable by autograd)."""
    import torch
    Lz, Ly, Lx = vol.shape
    dev = vol.device
    zt, xt = torch.meshgrid(torch.arange(Lz, device=dev, dtype=torch.float64),
                            torch.arange(Lx, device=dev, dtype=torch.float64), indexing="ij")
    cz, cx = (Lz - 1) / 2.0, (Lx - 1) / 2.0
    c, s = math.cos(theta), math.sin(theta)
    x0 = c * (xt - cx) - s * (zt - cz) + cx
    z0 = s * (xt - cx) + c * (zt - cz) + cz
    fx, fz = torch.floor(x0), torch.floor(z0)
    ax, az = (x0 - fx).float(), (z0 - fz).float()
    out = torch.zeros_like(vol)
    for dz, wz in ((0, 1 - az), (1, az)):
        for dx, wx in ((0, 1 - ax), (1, ax)):
            zi, xi = (fz + dz).long(), (fx + dx).long()
            ok = (zi >= 0) & (zi < Lz) & (xi >= 0) & (xi < Lx)
            g = vol[zi.clamp(0, Lz - 1), :, xi.clamp(0, Lx - 1)]            # [Lz, Lx, Ly]
            out = out + (g * (wz * wx * ok)[:, :, None]).permute(0, 2, 1)
    return out


def time_plain(w, dev, pos_b, I_meas_b, steps, warmup):
    """Per-step device time of the plain path (loss + autograd backward) on the same minibatches."""
    import torch
    p = w["problem"]
    want = set(w.get("grads", ("object", "probe", "positions")))
    d = torch.from_numpy(w["delta"]).to(dev).requires_grad_()
    b = torch.from_numpy(w["beta"]).to(dev).requires_grad_()
    probe = torch.from_numpy(w["probe"]).to(dev).requires_grad_("probe" in want)
    nb = len(pos_b)
    times = []
    for k in range(warmup + steps):
        pos = pos_b[k % nb].clone().requires_grad_("positions" in want)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        loss, _ = plain_loss(d, b, probe, pos, I_meas_b[k % nb], p)
        loss.backward()
        e.record()
        torch.cuda.synchronize(dev)
        if k >= warmup:
            times.append(s.elapsed_time(e))
        d.grad = b.grad = probe.grad = None
    return times


def time_regularize(eng, oid, d, b, stream, flush, hbm_peak, reps=20):
    """adorym_regularize on the workload's object (reweighted l1 + TV, value and gradient): kernel
    time with CUDA events on the library's stream, L2 flushed before every call.  Algorithmic bytes
    per voxel: delta, beta and the two weight arrays read (16 B) and the two gradients read and
    written (16 B); neighbour reads of the TV stencil come from cache and are not counted."""
    import torch
    with torch.cuda.stream(stream):
        wd = torch.ones_like(d)
        wb = torch.ones_like(b)
        eng.l1_weights(oid, 1e-8, wd, wb)
        gd, gb = torch.zeros_like(d), torch.zeros_like(b)
        loss = torch.zeros((), dtype=torch.float64, device=d.device)
        kw = dict(alpha_delta=1e-3, alpha_beta=1e-3, gamma_tv=1e-2, w_delta=wd, w_beta=wb, loss_out=loss,
                  g_delta=gd, g_beta=gb)
        for _ in range(3):
            eng.regularize(oid, **kw)
        # back to back on the stream (the host's call overhead overlaps the previous call's
        # kernels); the volume's arrays (delta, beta, weights, gradients) exceed L2, so every call
        # streams them from HBM
        ms = []
        for k in range(3):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                eng.regularize(oid, **kw)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1) / reps)
    n = d.numel()
    t = min(ms)
    gbs = 32 * n / (t * 1e-3) / 1e9
    return {"ms": t, "voxels": n, "bytes_per_voxel": 32, "achieved_gbs": gbs, "peak_gbs": hbm_peak,
            "frac": gbs / hbm_peak, "case": f"reweighted l1 + TV, value and gradient, {reps} calls back to back, "
                                            "best of 3 runs (arrays larger than L2)"}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank):
    if rank != 0:
        return
    import numpy as np
    from paper_2012_12686_gb300 import synth
    w = synth.workload(WORKLOAD, seed=0)
    L = w["problem"]["L"]
    # measured data for the sampled positions come from the oracle itself (no GPU on this arm)
    import oracle
    cores = os.cpu_count() or 1
    n_pos = cores
    sample_pos = w["pos"][:n_pos]
    Im = synth.poisson(oracle.forward(dict(w["problem"], B=n_pos), w["delta_meas"], w["beta_meas"], w["probe"],
                                      sample_pos), 7)
    ws = dict(w, pos=sample_pos)
    budget_s = 150.0
    times = []
    t_all = time.perf_counter()
    steps_run = 0
    pool = oracle_pool(cores)
    try:
        for k in range(args.warmup + args.steps):
            wall, npos = oracle_sample(ws, Im, n_pos, cores, pool=pool)
            if k >= args.warmup:
                times.append(wall)
                steps_run += 1
            if time.perf_counter() - t_all > budget_s and steps_run >= 1:
                break
    finally:
        pool.close()
        pool.join()
    mean_s = statistics.mean(times)
    value = n_pos * L / mean_s
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": steps_run,
            "warmup": args.warmup, "ms_per_step": mean_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD_DESC, "sample": f"{n_pos} positions x {L} slices per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n_pos} positions x {L} slices of one minibatch per step, "
                                       f"one position per single-threaded process"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2012_12686_gb300 import synth
    from paper_2012_12686_gb300.adorym import Engine, Problem, fp32_peak, kernel_launches

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    w = synth.workload(args.workload, seed=0, **({"B": args.batch} if args.batch else {}))
    p = w["problem"]
    N, L, B, M = p["N"], p["L"], p["B"], p["M"]
    far = bool(p["farfield"])
    nd = 1 if far else len(p["nf"])
    cp = p["checkpoint_every"] or int(math.ceil(math.sqrt(L)))
    all_pos = w.get("all_pos", w["pos"])
    nb = max(1, len(all_pos) // B)
    units = B * L * M if far else B * nd          # near field: one hologram distance is one unit
    with torch.cuda.stream(stream):
        d = torch.from_numpy(w["delta"]).to(dev)
        b = torch.from_numpy(w["beta"]).to(dev)
        dm = torch.from_numpy(w["delta_meas"]).to(dev)
        bm = torch.from_numpy(w["beta_meas"]).to(dev)
        probe = torch.from_numpy(w["probe"]).to(dev)
        pos_all = torch.from_numpy(all_pos).to(dev)
        eng = Engine(local_rank, stream.cuda_stream)
        oid = eng.register_object(d, b)
        oid_m = eng.register_object(dm, bm)
        prob = Problem.of(p)
        # measured data of the epoch: forward model of the second object + Poisson noise
        shape = (nb, B, N, N) if far else (nb, B, nd, N, N)
        I_meas = torch.empty(shape, dtype=torch.float32, device=dev)
        for k in range(nb):
            eng.forward(prob, oid_m, probe, pos_all[k * B:(k + 1) * B].contiguous(), I_meas[k])
        gen = torch.Generator(device=dev)
        gen.manual_seed(1234)
        ph = float(w.get("photons", 1.0))
        I_meas = torch.poisson(I_meas * ph, generator=gen) / ph
        pos_b = [pos_all[k * B:(k + 1) * B].contiguous() for k in range(nb)]
        loss = torch.zeros((), dtype=torch.float64, device=dev)
        gd, gb = torch.zeros_like(d), torch.zeros_like(b)
        want = set(w.get("grads", ("object", "probe", "positions")))
        gp = torch.zeros_like(probe) if "probe" in want else None
        gpos = torch.zeros(tuple(pos_all[:B].shape), dtype=torch.float32, device=dev) if "positions" in want else None
        flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
        eng.enable_kernel_timing(True)

        def step(k):
            eng.loss_grad(prob, oid, probe, pos_b[k % nb], I_meas[k % nb], loss, gd, gb, gp, gpos)

        for k in rank_batches(rank, world, 0, args.warmup, nb):
            step(k)
        stream.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    path_ms = []
    with ClockSampler(local_rank) as clk, torch.cuda.stream(stream):
        torch.cuda.synchronize(dev)
        launches0 = kernel_launches()
        t0 = time.perf_counter()
        for k, bi in enumerate(rank_batches(rank, world, args.warmup, args.steps, nb)):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            step(bi)
            ev[k][1].record(stream)
            path_ms.append(eng.kernel_ms())
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        n_launches = kernel_launches() - launches0   # this library's kernels in the timed region
        # latency sample: at least 200 more steps, each timed on its own (L2 flushed before each),
        # so that p99 is a percentile and not the maximum of a short run
        n_lat = max(200, args.steps)
        lat_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_lat)]
        for k, bi in enumerate(rank_batches(rank, world, args.warmup + args.steps, n_lat, nb)):
            flush.fill_(float(k))
            lat_ev[k][0].record(stream)
            step(bi)
            lat_ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
    step_ms = [a.elapsed_time(bq) for a, bq in ev]
    t_ours = max_over_ranks(sum(step_ms) / 1e3, dev)
    value = units * args.steps * world / t_ours
    ms_sorted = sorted(a.elapsed_time(bq) for a, bq in lat_ev)
    p50 = ms_sorted[len(ms_sorted) // 2]
    p99 = ms_sorted[min(len(ms_sorted) - 1, int(math.ceil(0.99 * len(ms_sorted))) - 1)]

    # ---- the plain unfused GPU path on the same minibatches (comparison arm of the metric)
    plain = None
    if not args.no_plain and far:
        pt = time_plain(w, dev, pos_b, I_meas, steps=min(args.steps, 20), warmup=3)
        ps = sorted(pt)
        plain = {"value": units / (statistics.mean(pt) / 1e3), "unit": UNIT, "ms_per_step": statistics.mean(pt),
                 "p50_ms": ps[len(ps) // 2], "p99_ms": ps[min(len(ps) - 1, int(math.ceil(0.99 * len(ps))) - 1)],
                 "steps": len(pt), "impl": "torch.fft + elementwise + torch autograd, one request at a time"}

    # ---- end to end through the public C ABI with pinned host buffers
    n_e2e = max(3, min(args.steps, 50))
    h_meas = [I_meas[k].cpu().pin_memory() for k in range(nb)]
    h_pos = [pb.cpu().pin_memory() for pb in pos_b]
    h_probe = probe.cpu().pin_memory()
    h_loss = np.zeros(1, np.float64)
    h_gp = torch.zeros(probe.shape, dtype=torch.complex64).pin_memory() if gp is not None else None
    h_gpos = torch.zeros(tuple(pos_all[:B].shape), dtype=torch.float32).pin_memory() if gpos is not None else None
    eng.enable_kernel_timing(False)
    with torch.cuda.stream(stream):
        for k in range(2):
            eng.loss_grad(prob, oid, h_probe, h_pos[k % nb], h_meas[k % nb], h_loss, gd, gb, h_gp, h_gpos)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for k in range(n_e2e):
            eng.loss_grad(prob, oid, h_probe, h_pos[k % nb], h_meas[k % nb], h_loss, gd, gb, h_gp, h_gpos)
        t_e2e = time.perf_counter() - t0
    e2e_val = units * world * n_e2e / max_over_ranks(t_e2e, dev)
    nel = (lambda t: 0 if t is None else t.numel())
    h2d = h_meas[0].numel() * 4 + h_pos[0].numel() * 4 + h_probe.numel() * 8 + nel(h_gp) * 8
    d2h = 8 + nel(h_gp) * 8 + nel(h_gpos) * 4

    if rank != 0:
        return
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = (peaks.get("sm_max_mhz") or 2070.0)
    fp32_peak_derived = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    k_ms = statistics.mean(path_ms)
    if far and N <= 128:
        achieved = units * flops_per_unit(N) / (k_ms * 1e-3) / 1e12
        form = launch_form(B, L, cp, props.multi_processor_count)
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak_derived, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak_derived, "kernel": f"{form}<{N},far>"}
        try:   # the same fraction against an FFMA throughput kernel measured now, on this GPU
            measured = fp32_peak(local_rank)
            roof.update(peak_measured_ffma=measured, frac_of_measured_ffma=achieved / measured)
        except Exception as exc:
            roof.update(peak_measured_ffma=None, peak_measured_note=str(exc))
    else:
        # two-pass / near field: HBM-bound; algorithmic bytes of the minimal pass structure
        bpu = twopass_bytes_per_unit(N, L, cp, nd, far)
        achieved = units * bpu / (k_ms * 1e-3) / 1e9
        hpk = peaks.get("hbm_gbs", 6795.5)
        roof = {"bound": "hbm", "achieved": achieved, "peak": hpk, "unit": "GB/s", "frac": achieved / hpk,
                "kernel": ("k_row/k_col two-pass sequence" if N >= 256
                           else f"{launch_form(B, L, cp, props.multi_processor_count)}<{N},near>"),
                "bytes_per_unit": bpu}
    hbm_ach = units * bytes_per_unit(N, L, cp) / (k_ms * 1e-3) / 1e9
    # the regularizer on the metric's 512 x 512 x 32 object, whose six volume arrays (268 MB) exceed L2
    reg = (time_regularize(eng, oid, d, b, stream, flush, peaks.get("hbm_gbs", 6795.5))
           if args.workload == WORKLOAD else None)
    src = kernel_source_bytes()
    traffic = profiled_traffic(hashlib.sha256(src).hexdigest()[:16])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "global_batch": B * world, "slices": L, "tile": N,
                       "parallelism": f"replica{world}" if world > 1 else "single", "l2": "flushed between steps"},
            "latency_ms": {"p50": p50, "p99": p99, "samples": len(ms_sorted),
                           "how": "per-step device time of separately timed steps after the timed region"},
            "gpu_launches": n_launches,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": dict(roof, traffic=traffic if args.workload == WORKLOAD else None, kernel_ms=k_ms,
                             peak_note=(f"FP32 FMA peak derived: {props.multi_processor_count} SMs x 128 lanes x 2 "
                                        f"x {sm_max:.0f} MHz" if roof["bound"] == "alu" else
                                        "measured copy bandwidth (MEASURED_PEAKS.json)"),
                             hbm_algorithmic_gbs=hbm_ach, hbm_peak_gbs=peaks.get("hbm_gbs", 6795.5)),
            "clocks": clk.summary(), "wall_s_timed": wall}
    if plain is not None:
        plain["speedup_of_fused"] = value / plain["value"]
        line["plain_gpu"] = plain
    if reg is not None:
        line["regularize"] = reg
    if args.workload != WORKLOAD:
        line["config"]["workload"] = args.workload
    if args.batch:
        line["config"]["workload"] = f"{args.workload} with batch {args.batch}"
    if not args.no_cpu_baseline and world == 1 and args.workload == WORKLOAD:
        # the oracle on the first minibatch (B positions x all slices): timed as it stands for the
        # CPU baseline, then its outputs compared with one untimed GPU call on the same inputs.
        # The measured intensities of this check come from the oracle (forward of the second
        # object + Poisson noise), so no oracle input comes from the CUDA path.
        cores = os.cpu_count() or 1
        w0 = dict(w, pos=all_pos[:B])
        pool = oracle_pool(cores)
        try:
            Im0 = oracle_measured(w0, B, cores, pool=pool)
            wall_c, npos, kept = oracle_sample(w0, Im0, B, cores, pool=pool, keep=True)
        finally:
            pool.close()
            pool.join()
        line["cpu_baseline"] = {"value": npos * L / wall_c, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"the {npos} positions x {L} slices of the first minibatch, one "
                                          f"position per single-threaded process ({wall_c:.1f} s wall)"}
        with torch.cuda.stream(stream):
            Im0_d = torch.from_numpy(Im0).to(dev)
            l0 = torch.zeros((), dtype=torch.float64, device=dev)
            gd0, gb0 = torch.zeros_like(d), torch.zeros_like(b)
            gp0 = torch.zeros_like(probe)
            gpos0 = torch.zeros((B, 2), dtype=torch.float32, device=dev)
            I0 = torch.empty((B, N, N), dtype=torch.float32, device=dev)
            eng.loss_grad(prob, oid, probe, pos_b[0], Im0_d, l0, gd0, gb0, gp0, gpos0, I0)
            stream.synchronize()
        errs = oracle_batch_parity(kept, tuple(w["delta"].shape), B, I0.cpu().numpy(), float(l0.item()),
                                   gd0.cpu().numpy(), gb0.cpu().numpy(), gp0.cpu().numpy(), gpos0.cpu().numpy())
        line["parity"] = dict(errs, vs="FP64 oracle, first minibatch, same launch configuration as the timed steps",
                              bars=parity_bars(args.workload))
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Serving mix: Poisson arrivals of loss+gradient requests of uneven tile size, slice count
    and batch over resident volumes, through adorym_submit / adorym_poll (slots, footprint
    admission, captured graphs).  Latency = completion - arrival on the host clock.  The plain
    torch path is timed once per request template and replayed one request at a time on the same
    arrival schedule (a single server: start = max(arrival, previous finish))."""
    import threading
    import numpy as np
    import torch
    from paper_2012_12686_gb300 import synth
    from paper_2012_12686_gb300.adorym import Engine, Problem, OK
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    g = np.random.default_rng(7)
    Ls, Ns = (1, 8, 32, 64), (64, 128, 256)
    side = args.serve_side
    eng = Engine(0)
    vols = {}
    for L in Ls:   # resident volumes side x side x L (ellipsoids, beta = delta / 10)
        d = synth.ellipsoid_volume((L, side, side), 96, (16, 96), (1, max(1, L // 2)), (1e-6, 3e-6), 5e-6, 50 + L)
        td = torch.from_numpy(d).to(dev)
        tb = (td / 10.0).contiguous()
        vols[L] = (td, tb, eng.register_object(td, tb))
    probes = {N: torch.from_numpy(synth.probe_phase_screen(N, N / 8.0, 4.0, 1.0, 1e6, 60 + N)).to(dev) for N in Ns}
    # request templates with their own positions and measured data (forward of a perturbed object)
    templates = []
    for k in range(args.serve_templates):
        N, L = int(g.choice(Ns)), int(g.choice(Ls))
        B = int(g.integers(8, 257))
        pos = torch.from_numpy(g.uniform(0, side - N, (B, 2)).astype(np.float32)).to(dev)
        p = dict(N=N, L=L, M=1, B=B, Lz=L, Ly=side, Lx=side, kdz=synth.KDZ_10NM,
                 lambda_dz_over_px2=synth.LAMBDA_DZ_OVER_PX2_10NM, farfield=1, nf=[], loss="poisson", eps=1e-3)
        td, tb, oid = vols[L]
        I = torch.empty((B, N, N), dtype=torch.float32, device=dev)
        eng.forward(p, oid, probes[N], pos, I)
        I = torch.poisson(I * 1.05)
        templates.append(dict(p=p, prob=Problem.of(p), oid=oid, pos=pos, I=I, units=B * L))
    torch.cuda.synchronize()
    budget = args.serve_budget_gb << 30
    eng.serve_config(args.serve_slots, budget)
    n = args.serve_requests
    arrivals = np.cumsum(g.exponential(1.0 / args.serve_rate, n))
    which = g.integers(0, len(templates), n)
    # output buffers rotate over 2 x slots sets (results are not inspected here; the serving test
    # checks them)
    per_slot = [{L: (torch.zeros_like(vols[L][0]), torch.zeros_like(vols[L][1])) for L in Ls}
                for _ in range(2 * args.serve_slots)]
    gpos_buf = [torch.zeros((256, 2), dtype=torch.float32, device=dev) for _ in range(2 * args.serve_slots)]
    loss_buf = [torch.zeros((), dtype=torch.float64, device=dev) for _ in range(2 * args.serve_slots)]
    # warm the graphs of every template (twice per slot set: capture, then update), then time each
    # template alone on an idle device: its standalone service time, the denominator of the slowdown
    for rep in range(2):
        for t in templates:
            gd, gb = per_slot[0][t["p"]["L"]]
            tk = eng.submit(t["prob"], t["oid"], probes[t["p"]["N"]], t["pos"], t["I"], loss_buf[0], gd, gb, None,
                            gpos_buf[0][:t["p"]["B"]])
            eng.poll(tk, -1)
    alone_ms = []
    for t in templates:
        gd, gb = per_slot[0][t["p"]["L"]]
        tk = eng.submit(t["prob"], t["oid"], probes[t["p"]["N"]], t["pos"], t["I"], loss_buf[0], gd, gb, None,
                        gpos_buf[0][:t["p"]["B"]])
        t0a = time.perf_counter()
        eng.poll(tk, -1)
        alone_ms.append((time.perf_counter() - t0a) * 1e3)
    done_t = [0.0] * n
    parts = [(0.0, 0.0)] * n
    tickets = [None] * n
    t0 = time.perf_counter()

    def submitter():
        for i in range(n):
            now = time.perf_counter() - t0
            if arrivals[i] > now:
                time.sleep(arrivals[i] - now)
            t = templates[which[i]]
            slot = i % len(per_slot)
            gd, gb = per_slot[slot][t["p"]["L"]]
            tickets[i] = eng.submit(t["prob"], t["oid"], probes[t["p"]["N"]], t["pos"], t["I"], loss_buf[slot], gd,
                                    gb, None, gpos_buf[slot][:t["p"]["B"]])

    th = threading.Thread(target=submitter)
    th.start()
    for i in range(n):
        while tickets[i] is None:
            time.sleep(0.0001)
        rc, queued_us, run_us, _ = eng.poll_times(tickets[i], -1)
        assert rc == OK
        done_t[i] = time.perf_counter() - t0
        parts[i] = (queued_us / 1e3, run_us / 1e3)
    th.join()
    lat = np.array(done_t) - arrivals
    queued = np.array([q for q, _ in parts])
    run = np.array([r for _, r in parts])
    slowdown = lat * 1e3 / np.array([alone_ms[w] for w in which])
    units = np.array([templates[w]["units"] for w in which])
    span = done_t[-1] - arrivals[0]
    # plain path: per-template service time (sub-batches of <= 32 positions to bound autograd memory)
    svc = []
    for t in templates:
        td, tb, _ = vols[t["p"]["L"]]
        d = td.clone().requires_grad_()
        b = tb.clone().requires_grad_()
        pr = probes[t["p"]["N"]].clone().requires_grad_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for rep in range(2):
            s.record()
            B = t["p"]["B"]
            for c0 in range(0, B, 32):
                c1 = min(B, c0 + 32)
                pos = t["pos"][c0:c1].clone().requires_grad_()
                loss, _ = plain_loss(d, b, pr, pos, t["I"][c0:c1], dict(t["p"], B=c1 - c0))
                (loss * ((c1 - c0) / B)).backward()
            e.record()
            torch.cuda.synchronize()
        svc.append(s.elapsed_time(e) / 1e3)
        del d, b, pr
        torch.cuda.empty_cache()
    svc = np.array(svc)
    fin, plat = 0.0, []
    for i in range(n):
        fin = max(arrivals[i], fin) + svc[which[i]]
        plat.append(fin - arrivals[i])
    plat = np.array(plat)
    line = {"metric": "serving mix: loss+gradient requests, Poisson arrivals", "requests": n,
            "rate_per_s": args.serve_rate, "slots": args.serve_slots, "budget_gb": args.serve_budget_gb,
            "mix": "N in {64,128,256}, L in {1,8,32,64}, B in U{8..256}, Poisson loss, grads delta/beta/positions",
            "volumes": f"{side}x{side}x{{1,8,32,64}} resident", "templates": len(templates),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "throughput": float(units.sum() / span), "unit": UNIT,
            "admission_waits": eng.serve_stats()[1],
            "breakdown_ms": {"queued_p50": float(np.percentile(queued, 50)),
                             "queued_p99": float(np.percentile(queued, 99)),
                             "run_p50": float(np.percentile(run, 50)), "run_p99": float(np.percentile(run, 99)),
                             "how": "queued = submit to admission, run = admission to completion (poll_times)"},
            "alone_ms": {"p50": float(np.percentile([alone_ms[w] for w in which], 50)),
                         "p99": float(np.percentile([alone_ms[w] for w in which], 99)),
                         "max": float(max(alone_ms)),
                         "how": "each template submitted alone on an idle device, submit to poll return"},
            "slowdown": {"p50": float(np.percentile(slowdown, 50)), "p99": float(np.percentile(slowdown, 99)),
                         "how": "latency in the mix / the same request's latency alone"},
            "plain_one_at_a_time": {"p50_ms": float(np.percentile(plat, 50) * 1e3),
                                    "p99_ms": float(np.percentile(plat, 99) * 1e3),
                                    "throughput": float(units.sum() / (fin - arrivals[0])),
                                    "how": "measured service time per template, replayed on the same arrivals"}}
    print(json.dumps(line), flush=True)


def parity_bars(workload: str):
    """Relative-L2 bars against the FP64 oracle: 1e-4 for intensities and loss; for gradients
    1e-3, or at full size the FP32 floor stored in tests/golden/fp32_floor.json (the error of the
    same model evaluated with single-precision FFTs, written by tests/golden/make_fp32_floor.py
    from the oracle alone) where that floor is higher."""
    bars = {"I": 1e-4, "loss": 1e-4, "gd": 1e-3, "gb": 1e-3, "gp": 1e-3, "gpos": 1e-3}
    try:
        with open(os.path.join(ROOT, "tests", "golden", "fp32_floor.json")) as fh:
            fl = json.load(fh)["workloads"][workload]["fp32_fft"]
        for k in ("gd", "gb", "gp", "gpos"):
            bars[k] = max(bars[k], fl[k])
    except (OSError, KeyError, ValueError):
        pass
    return bars


KERNEL_SOURCES = ("k_path.cuh", "fft_block.cuh", "fft_block4.cuh", "numerics.cuh", "kernels.cuh")


def kernel_source_bytes() -> bytes:
    """Source of the fused shared-memory kernel (the files its code is compiled from)."""
    d = os.path.join(ROOT, "paper_2012_12686_gb300", "csrc")
    return b"".join(open(os.path.join(d, f), "rb").read() for f in KERNEL_SOURCES)


def profiled_traffic(src_hash: str):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary, if it was taken
    on the current kernel source (else null)."""
    path = os.path.join(ROOT, "profiles", "k_path_multislice_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        return rec["dram_bytes_per_launch"] if rec.get("source_sha256_16") == src_hash else None
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain torch GPU path")
    ap.add_argument("--workload", default=WORKLOAD, choices=["multislice", "ptycho2d", "tomo", "holo", "farfield256"],
                    help="workload of the timed steps (default: the metric's multislice configuration)")
    ap.add_argument("--batch", type=int, default=0,
                    help="override the workload's batch (positions / problems per call), e.g. a small case for "
                         "kernel captures; not a bench line of the metric")
    ap.add_argument("--serve", action="store_true", help="run the serving mix instead of the minibatch benchmark")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=int, default=24)
    ap.add_argument("--serve-templates", type=int, default=48)
    ap.add_argument("--serve-side", type=int, default=1024)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.serve:
        if rank == 0:
            run_serve(args)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
