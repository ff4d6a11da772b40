"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no step of the reconstruction method (no propagation, no
loss, no gradient): it only draws objects, probes, scan positions and noise
from ``numpy.random.default_rng(seed)``.  The CUDA path, its tests, the
benchmark and the FP64 oracle all take their inputs from here, so both sides
of every parity check see bit-identical arrays.

Workloads (sizes and magnitudes follow the paper's experiments):

* ``ptycho2d``  -- 2D far-field ptychography: object 64x64x1, delta and beta
  uniform in [0, 1e-3], 32x32 Gaussian probe (sigma 6 px) with uniform random
  phase, 7x7 raster at 4 px, LSQ loss (Sec. 3.2-style single-slice case).
* ``multislice`` -- 3D multislice far-field ptychography: object 512x512x32 of
  random ellipsoids (delta in [0, 5e-6], beta = delta/10), 10 nm voxels at
  0.248 nm, 128x128 focused probe with a random phase screen, 32x32 raster at
  12 px with +-0.5 px jitter, minibatch of 128, Poisson loss (the 128x128
  multislice experiment of Sec. 3.3 scaled to a synthetic object).
* ``tomo``      -- ptychographic tomography: 128^3 ellipsoid volume (delta in
  [0, 1e-5], beta = delta/20), 180 angles over [0, 180) deg, 8x8 positions at
  16 px centred on the volume, 64x64 probe, 128 slices, one angle per batch.
* ``farfield256`` -- one serving-mix request shape at the two-pass tile: 256x256 probe, 8
  slices, 64 positions on an 8x8 raster at 96 px over a 1024x1024x8 volume, Poisson loss.
* ``holo``      -- near-field multi-distance holography: 1024x1024 single
  slice, phase in [0, 2] rad, absorption at most 0.05, plane wave, Fresnel
  numbers 1e-3..8e-3, per-hologram shifts of +-5 px plus a sub-pixel part,
  8 problems per launch.
"""
from __future__ import annotations

import math

import numpy as np

# lambda = 0.248 nm (5 keV), voxel 10 nm, dz = one voxel
WAVELENGTH_NM = 0.248
VOXEL_NM = 10.0
KDZ_10NM = 2.0 * math.pi * VOXEL_NM / WAVELENGTH_NM          # k * dz
LAMBDA_DZ_OVER_PX2_10NM = WAVELENGTH_NM * VOXEL_NM / VOXEL_NM ** 2


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- objects
def uniform_object(shape, hi, seed):
    """delta, beta ~ U[0, hi] independently, float32 [Lz, Ly, Lx]."""
    g = rng(seed)
    d = g.uniform(0.0, hi, size=shape).astype(np.float32)
    b = g.uniform(0.0, hi, size=shape).astype(np.float32)
    return d, b


def ellipsoid_volume(shape, n, semi_lat, semi_ax, amp, vmax, seed):
    """Sum of ``n`` random axis-aligned ellipsoids, clipped to [0, vmax].

    shape = (Lz, Ly, Lx); lateral semi-axes ~ U[semi_lat], axial ~ U[semi_ax];
    each ellipsoid adds a constant drawn from U[amp].
    """
    Lz, Ly, Lx = shape
    g = rng(seed)
    vol = np.zeros(shape, np.float64)
    for _ in range(n):
        cz, cy, cx = g.uniform(0, Lz), g.uniform(0, Ly), g.uniform(0, Lx)
        ry, rx = g.uniform(*semi_lat), g.uniform(*semi_lat)
        rz = g.uniform(*semi_ax)
        a = g.uniform(*amp)
        z0, z1 = max(0, int(cz - rz)), min(Lz, int(cz + rz) + 1)
        y0, y1 = max(0, int(cy - ry)), min(Ly, int(cy + ry) + 1)
        x0, x1 = max(0, int(cx - rx)), min(Lx, int(cx + rx) + 1)
        if z0 >= z1 or y0 >= y1 or x0 >= x1:
            continue
        z = (np.arange(z0, z1) - cz)[:, None, None] / rz
        y = (np.arange(y0, y1) - cy)[None, :, None] / ry
        x = (np.arange(x0, x1) - cx)[None, None, :] / rx
        vol[z0:z1, y0:y1, x0:x1] += a * ((z * z + y * y + x * x) <= 1.0)
    return np.clip(vol, 0.0, vmax).astype(np.float32)


def smooth_field(shape, sigma, lo, hi, seed):
    """White noise low-passed by a periodic Gaussian filter, min-max scaled to [lo, hi]."""
    from scipy.ndimage import gaussian_filter
    g = rng(seed)
    f = gaussian_filter(g.standard_normal(shape), sigma, mode="wrap")
    f = (f - f.min()) / (f.max() - f.min())
    return (lo + (hi - lo) * f).astype(np.float32)


# ----------------------------------------------------------------- probes
def _gauss_amp(N, sigma):
    y = np.arange(N) - (N - 1) / 2.0
    return np.exp(-(y[:, None] ** 2 + y[None, :] ** 2) / (2.0 * sigma ** 2))


def _scale_photons(p, photons):
    return p * math.sqrt(photons / float(np.sum(np.abs(p) ** 2)))


def probe_random_phase(N, sigma, photons, seed, modes=1):
    """Gaussian amplitude times uniform random phase in [-pi, pi], |P|^2 summing to ``photons`` per mode."""
    g = rng(seed)
    out = np.empty((modes, N, N), np.complex64)
    for m in range(modes):
        ph = g.uniform(-math.pi, math.pi, size=(N, N))
        out[m] = _scale_photons(_gauss_amp(N, sigma) * np.exp(1j * ph), photons)
    return out


def probe_phase_screen(N, sigma, screen_sigma, screen_std, photons, seed, modes=1):
    """Gaussian focus times exp(i * screen); screen = Gaussian-filtered white noise of std ``screen_std`` rad."""
    from scipy.ndimage import gaussian_filter
    g = rng(seed)
    out = np.empty((modes, N, N), np.complex64)
    for m in range(modes):
        s = gaussian_filter(g.standard_normal((N, N)), screen_sigma, mode="wrap")
        s *= screen_std / s.std()
        out[m] = _scale_photons(_gauss_amp(N, sigma) * np.exp(1j * s), photons / (m + 1))
    return out


def plane_wave(N, modes=1):
    return np.ones((modes, N, N), np.complex64)


# --------------------------------------------------------------- positions
def raster(ny, nx, step, origin, jitter=0.0, seed=0):
    """[ny*nx, 2] (y, x) float32 raster; optional U[-jitter, jitter] per coordinate."""
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    pos = np.stack([origin + step * yy.ravel(), origin + step * xx.ravel()], 1).astype(np.float64)
    if jitter:
        pos += rng(seed).uniform(-jitter, jitter, size=pos.shape)
    return pos.astype(np.float32)


def hologram_shifts(n_problems, n_dist, max_int, seed):
    """Integer U{-max_int..max_int} plus U[-0.5, 0.5] per hologram and axis: [P, n_dist, 2]."""
    g = rng(seed)
    s = g.integers(-max_int, max_int + 1, size=(n_problems, n_dist, 2)).astype(np.float64)
    s += g.uniform(-0.5, 0.5, size=s.shape)
    return s.astype(np.float32)


def poisson(I, seed, scale=1.0):
    """Poisson counts of ``I * scale`` divided back by ``scale`` (float32)."""
    lam = np.maximum(np.asarray(I, np.float64) * scale, 0.0)
    return (rng(seed).poisson(lam) / scale).astype(np.float32)


# --------------------------------------------------------------- workloads
def workload(name: str, seed: int = 0, **over):
    """Inputs of one named workload, as a dict of numpy arrays and parameters.

    Keys: ``problem`` (dict of the physical/problem parameters), ``delta``,
    ``beta`` (float32 [Lz, Ly, Lx]), ``probe`` (complex64 [M, N, N]),
    ``pos`` (float32 [B, 2], or [B, n_dist, 2] hologram shifts for ``holo``),
    ``delta_meas``/``beta_meas`` (a second object from which measured data are
    simulated), ``photons`` (scale for the Poisson noise) and ``grads`` (the gradients the
    workload asks for, a subset of object / probe / positions; ``positions`` are the hologram
    shifts in the near field).  The measured
    intensities themselves are produced by the caller's forward model.
    """
    if name == "ptycho2d":
        p = dict(N=32, L=1, M=1, B=49, Lz=1, Ly=64, Lx=64, kdz=KDZ_10NM,
                 lambda_dz_over_px2=LAMBDA_DZ_OVER_PX2_10NM, farfield=1, nf=[],
                 loss="lsq", eps=1e-6, tomo=0, theta=0.0, checkpoint_every=0)
        p.update(over)
        shape = (p["Lz"], p["Ly"], p["Lx"])
        d, b = uniform_object(shape, 1e-3, seed)
        dm, bm = uniform_object(shape, 1e-3, seed + 1)
        probe = probe_random_phase(p["N"], 6.0, 1e4, seed + 2, p["M"])
        side = int(round(math.sqrt(p["B"])))
        pos = raster(side, side, 4, 4)
        return dict(problem=p, delta=d, beta=b, delta_meas=dm, beta_meas=bm,
                    probe=probe, pos=pos[: p["B"]], photons=1.0, grads=("object", "probe"))
    if name == "multislice":
        p = dict(N=128, L=32, M=1, B=128, Lz=32, Ly=512, Lx=512, kdz=KDZ_10NM,
                 lambda_dz_over_px2=LAMBDA_DZ_OVER_PX2_10NM, farfield=1, nf=[],
                 loss="poisson", eps=1e-6, tomo=0, theta=0.0, checkpoint_every=0)
        start = over.pop("batch_start", 0)
        p.update(over)
        shape = (p["Lz"], p["Ly"], p["Lx"])

        def obj(s):
            d = ellipsoid_volume(shape, 64, (8, 64), (2, 16), (1e-6, 3e-6), 5e-6, s)
            return d, (d / 10.0).astype(np.float32)
        d, b = obj(seed)
        dm, bm = obj(seed + 1)
        probe = probe_phase_screen(p["N"], 16.0, 4.0, 1.0, 1e6, seed + 2, p["M"])
        pos = raster(32, 32, 12, 6, jitter=0.5, seed=seed + 3)
        return dict(problem=p, delta=d, beta=b, delta_meas=dm, beta_meas=bm,
                    probe=probe, pos=pos[start:start + p["B"]], all_pos=pos, photons=1.0,
                    grads=("object", "probe", "positions"))
    if name == "tomo":
        p = dict(N=64, L=128, M=1, B=64, Lz=128, Ly=128, Lx=128, kdz=KDZ_10NM,
                 lambda_dz_over_px2=LAMBDA_DZ_OVER_PX2_10NM, farfield=1, nf=[],
                 loss="lsq", eps=1e-6, tomo=1, theta=0.0, checkpoint_every=0)
        angle_index = over.pop("angle_index", 30)
        p.update(over)
        p["theta"] = math.pi * angle_index / 180.0
        shape = (p["Lz"], p["Ly"], p["Lx"])

        def obj(s):
            d = ellipsoid_volume(shape, 48, (6, 32), (6, 32), (2e-6, 6e-6), 1e-5, s)
            return d, (d / 20.0).astype(np.float32)
        d, b = obj(seed)
        dm, bm = obj(seed + 1)
        probe = probe_phase_screen(p["N"], 10.0, 3.0, 1.0, 1e6, seed + 2, p["M"])
        side = int(round(math.sqrt(p["B"])))
        span = (side - 1) * 16 + p["N"]
        pos = raster(side, side, 16, (p["Ly"] - span) / 2.0)
        return dict(problem=p, delta=d, beta=b, delta_meas=dm, beta_meas=bm,
                    probe=probe, pos=pos, photons=1.0, grads=("object", "probe", "positions"))
    if name == "farfield256":
        # one request shape of the serving mix at the two-pass tile: 256 x 256 probe, 8 slices,
        # 64 positions over a resident 1024 x 1024 x 8 volume, Poisson loss
        p = dict(N=256, L=8, M=1, B=64, Lz=8, Ly=1024, Lx=1024, kdz=KDZ_10NM,
                 lambda_dz_over_px2=LAMBDA_DZ_OVER_PX2_10NM, farfield=1, nf=[],
                 loss="poisson", eps=1e-6, tomo=0, theta=0.0, checkpoint_every=0)
        p.update(over)
        shape = (p["Lz"], p["Ly"], p["Lx"])

        def obj(s):
            d = ellipsoid_volume(shape, 96, (16, 96), (1, 4), (1e-6, 3e-6), 5e-6, s)
            return d, (d / 10.0).astype(np.float32)
        d, b = obj(seed)
        dm, bm = obj(seed + 1)
        probe = probe_phase_screen(p["N"], 32.0, 8.0, 1.0, 1e6, seed + 2, p["M"])
        pos = raster(8, 8, 96, 8, jitter=0.5, seed=seed + 3)
        return dict(problem=p, delta=d, beta=b, delta_meas=dm, beta_meas=bm,
                    probe=probe, pos=pos[: p["B"]], photons=1.0, grads=("object", "probe", "positions"))
    if name == "holo":
        p = dict(N=1024, L=1, M=1, B=8, Lz=8, Ly=1024, Lx=1024, kdz=KDZ_10NM,
                 lambda_dz_over_px2=0.0, farfield=0, nf=[1e-3, 2e-3, 4e-3, 8e-3],
                 loss="lsq", eps=1e-6, tomo=0, theta=0.0, checkpoint_every=0)
        p.update(over)
        N, B = p["N"], p["B"]
        p["Ly"] = p["Lx"] = N
        p["Lz"] = B * p["L"]

        def obj(s):
            ph = np.stack([smooth_field((N, N), N / 64.0, 0.0, 2.0, s + 10 * i)
                           for i in range(p["Lz"])])
            ab = np.stack([smooth_field((N, N), N / 64.0, 0.0, 0.0513, s + 10 * i + 5)
                           for i in range(p["Lz"])])
            return (ph / p["kdz"]).astype(np.float32), (ab / p["kdz"]).astype(np.float32)
        d, b = obj(seed)
        dm, bm = obj(seed + 1)
        pos = hologram_shifts(B, len(p["nf"]), 5, seed + 3)
        return dict(problem=p, delta=d, beta=b, delta_meas=dm, beta_meas=bm,
                    probe=plane_wave(N, p["M"]), pos=pos, photons=1e4, grads=("object", "positions"))
    raise ValueError(f"unknown workload {name!r}")
