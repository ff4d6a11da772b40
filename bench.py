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
        self.path = os.path.join(ROOT, "gpurun_out", f".clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={SMI_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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


def oracle_pool(workers: int):
    """Spawn pool of single-threaded oracle workers (one BLAS thread each)."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    return mp.get_context("spawn").Pool(workers)


def oracle_sample(w, I_meas_np, n_pos: int, workers: int, pool=None):
    """Time the FP64 oracle (as it stands) on n_pos positions of the minibatch, one position per
    task, over a spawn pool of `workers` single-threaded processes.  Returns (wall s, positions)."""
    import numpy as np
    N = w["problem"]["N"]
    p = dict(w["problem"], B=1, Ly=N, Lx=N)
    jobs = []
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
    own = pool is None
    if own:
        pool = oracle_pool(workers)
    try:
        pool.map(_oracle_one, jobs[:workers])          # warm: imports, DFT matrices
        t = time.perf_counter()
        pool.map(_oracle_one, jobs)
        wall = time.perf_counter() - t
    finally:
        if own:
            pool.close()
            pool.join()
    return wall, n_pos


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
    step_ms = [a.elapsed_time(bq) for a, bq in ev]
    t_ours = max_over_ranks(sum(step_ms) / 1e3, dev)
    value = units * args.steps * world / t_ours
    ms_sorted = sorted(step_ms)
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
    src = kernel_source_bytes()
    traffic = profiled_traffic(hashlib.sha256(src).hexdigest()[:16])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "global_batch": B * world, "slices": L, "tile": N,
                       "parallelism": f"replica{world}" if world > 1 else "single", "l2": "flushed between steps"},
            "latency_ms": {"p50": p50, "p99": p99},
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
    if args.workload != WORKLOAD:
        line["config"]["workload"] = args.workload
    if args.batch:
        line["config"]["workload"] = f"{args.workload} with batch {args.batch}"
    if not args.no_cpu_baseline and world == 1 and args.workload == WORKLOAD:
        cores = os.cpu_count() or 1
        n_pos = min(8 * cores, len(all_pos))
        Im_np = I_meas.reshape(-1, N, N)[:n_pos].cpu().numpy()
        ws = dict(w, pos=all_pos[:n_pos])
        wall_c, npos = oracle_sample(ws, Im_np, n_pos, cores)
        line["cpu_baseline"] = {"value": npos * L / wall_c, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{npos} positions x {L} slices of the epoch, one position per "
                                          f"single-threaded process ({wall_c:.1f} s wall)"}
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
    # warm the graphs of every template once
    for t in templates:
        gd, gb = per_slot[0][t["p"]["L"]]
        tk = eng.submit(t["prob"], t["oid"], probes[t["p"]["N"]], t["pos"], t["I"], loss_buf[0], gd, gb, None,
                        gpos_buf[0][:t["p"]["B"]])
        eng.poll(tk, -1)
    done_t = [0.0] * n
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
        assert eng.poll(tickets[i], -1) == OK
        done_t[i] = time.perf_counter() - t0
    th.join()
    lat = np.array(done_t) - arrivals
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
            "plain_one_at_a_time": {"p50_ms": float(np.percentile(plat, 50) * 1e3),
                                    "p99_ms": float(np.percentile(plat, 99) * 1e3),
                                    "throughput": float(units.sum() / (fin - arrivals[0])),
                                    "how": "measured service time per template, replayed on the same arrivals"}}
    print(json.dumps(line), flush=True)


KERNEL_SOURCES = ("k_path.cuh", "fft_block.cuh", "numerics.cuh", "kernels.cuh")


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
    ap.add_argument("--workload", default=WORKLOAD, choices=["multislice", "ptycho2d", "tomo", "holo"],
                    help="workload of the timed steps (default: the metric's multislice configuration)")
    ap.add_argument("--batch", type=int, default=0,
                    help="override the workload's batch (positions / problems per call), e.g. a small case for "
                         "kernel captures; not a bench line of the metric")
    ap.add_argument("--serve", action="store_true", help="run the serving mix instead of the minibatch benchmark")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-slots", type=int, default=4)
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
