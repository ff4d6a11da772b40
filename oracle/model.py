"""FP64 oracle of the multislice ptychography loss and its gradient (test infrastructure only).

Plain, slow, per-position evaluation of the forward model of Algorithm 1
(far-field ptychography / ptychotomography predict function) and of the
near-field multi-distance variant, the LSQ / Poisson data-mismatch terms, and
a hand-derived adjoint written out step by step with the chain rule (the
paper leaves this step to automatic differentiation, Sec. 2.3.1 after
Eq. fourier_shift).  Every wavefield of the slice loop is kept (no
checkpointing): the oracle is the definition, not a fast program.

Conventions (each is a reading of the paper, stated where it is used):
* object volume [Lz, Ly, Lx] for delta and beta; probe [M, N, N] complex;
  positions [B, 2] as (y, x) in pixels.
* complex gradients are returned as dL/dRe + i dL/dIm.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .dft import dft_minus, dft_plus, freq, idft_minus


@dataclass
class Problem:
    N: int
    L: int
    M: int
    B: int
    Lz: int
    Ly: int
    Lx: int
    kdz: float                      # k * dz, k = 2 pi / lambda (Eq. ri_modulation)
    lambda_dz_over_px2: float       # lambda * dz / dx^2: slice-to-slice Fresnel step in pixel units
    farfield: int = 1
    nf: list = field(default_factory=list)   # near-field Fresnel numbers dx^2 / (lambda z)
    loss: str = "lsq"
    eps: float = 1e-6
    tomo: int = 0
    theta: float = 0.0
    checkpoint_every: int = 0
    gaps: list = None               # sparse / variable multislice: L-1 values lambda dz_j / dx^2 (None: uniform)

    def gap(self, j):
        """lambda dz_j / dx^2 of the Fresnel step from slice j to slice j + 1."""
        return self.lambda_dz_over_px2 if self.gaps is None else float(self.gaps[j])

    @staticmethod
    def of(d: dict) -> "Problem":
        keys = Problem.__dataclass_fields__.keys()
        return Problem(**{k: v for k, v in d.items() if k in keys})


# ------------------------------------------------------------------ S1
def split_positions(pos):
    """Integer patch corner p0 = floor(pos + 1/2) and residual dr = pos - p0 in [-1/2, 1/2).

    Sec. 2.3.1 (before Eq. fourier_shift): the integer part selects the
    object chunk, the floating-point residual is applied to the probe.
    """
    pos = np.asarray(pos, np.float64)
    p0 = np.floor(pos + 0.5)
    return p0.astype(np.int64), pos - p0


# ------------------------------------------------------------------ S2 (rotation)
def rotation_taps(Lz, Lx, theta):
    """Bilinear taps of Eq. rotation_transform in the x-z plane (rotation about y).

    Rotated-frame voxel (z_t, x_t) samples the unrotated volume at
      x0 = cos(t)(x_t - cx) - sin(t)(z_t - cz) + cx
      z0 = sin(t)(x_t - cx) + cos(t)(z_t - cz) + cz
    with (cz, cx) = ((Lz-1)/2, (Lx-1)/2); nodes outside the volume are dropped
    (zero fill).  Returns (dst, src, w): flat z*Lx + x indices and weights.
    """
    zt, xt = np.meshgrid(np.arange(Lz, dtype=np.float64), np.arange(Lx, dtype=np.float64), indexing="ij")
    cz, cx = (Lz - 1) / 2.0, (Lx - 1) / 2.0
    c, s = math.cos(theta), math.sin(theta)
    x0 = c * (xt - cx) - s * (zt - cz) + cx
    z0 = s * (xt - cx) + c * (zt - cz) + cz
    fx, fz = np.floor(x0), np.floor(z0)
    ax, az = x0 - fx, z0 - fz
    dst_all, src_all, w_all = [], [], []
    dst = (zt * Lx + xt).astype(np.int64).ravel()
    for dz_, wz in ((0, 1.0 - az), (1, az)):
        for dx_, wx in ((0, 1.0 - ax), (1, ax)):
            zi = (fz + dz_).astype(np.int64).ravel()
            xi = (fx + dx_).astype(np.int64).ravel()
            w = (wz * wx).ravel()
            ok = (zi >= 0) & (zi < Lz) & (xi >= 0) & (xi < Lx)
            dst_all.append(dst[ok]); src_all.append((zi * Lx + xi)[ok]); w_all.append(w[ok])
    return np.concatenate(dst_all), np.concatenate(src_all), np.concatenate(w_all)


def rotate(vol, theta):
    """Rotated volume O' = R_theta O (bilinear, Eq. rotation_transform), vol [Lz, Ly, Lx]."""
    Lz, Ly, Lx = vol.shape
    dst, src, w = rotation_taps(Lz, Lx, theta)
    v = np.transpose(np.asarray(vol, np.float64), (1, 0, 2)).reshape(Ly, Lz * Lx)
    out = np.zeros_like(v)
    np.add.at(out.T, dst, (w[:, None] * v[:, src].T))
    return np.transpose(out.reshape(Ly, Lz, Lx), (1, 0, 2))


def rotate_T(g, theta):
    """Exact transpose of ``rotate``: scatter-add with the same taps."""
    Lz, Ly, Lx = g.shape
    dst, src, w = rotation_taps(Lz, Lx, theta)
    v = np.transpose(np.asarray(g, np.float64), (1, 0, 2)).reshape(Ly, Lz * Lx)
    out = np.zeros_like(v)
    np.add.at(out.T, src, (w[:, None] * v[:, dst].T))
    return np.transpose(out.reshape(Ly, Lz, Lx), (1, 0, 2))


# ------------------------------------------------------------------ S2 (chunk)
def take_chunk(vol, p0, N):
    """TakeObjectChunk of Algorithm 1: vol[:, p0y:p0y+N, p0x:p0x+N], zero outside the volume."""
    Lz, Ly, Lx = vol.shape
    out = np.zeros((Lz, N, N), np.float64)
    y0, x0 = int(p0[0]), int(p0[1])
    ya, yb = max(y0, 0), min(y0 + N, Ly)
    xa, xb = max(x0, 0), min(x0 + N, Lx)
    if ya < yb and xa < xb:
        out[:, ya - y0:yb - y0, xa - x0:xb - x0] = vol[:, ya:yb, xa:xb]
    return out


def put_chunk_T(gvol, p0, chunk):
    """Transpose of ``take_chunk``: add the chunk into gvol; out-of-volume pixels are dropped."""
    Lz, Ly, Lx = gvol.shape
    N = chunk.shape[-1]
    y0, x0 = int(p0[0]), int(p0[1])
    ya, yb = max(y0, 0), min(y0 + N, Ly)
    xa, xb = max(x0, 0), min(x0 + N, Lx)
    if ya < yb and xa < xb:
        gvol[:, ya:yb, xa:xb] += chunk[:, ya - y0:yb - y0, xa - x0:xb - x0]


# ------------------------------------------------------------------ S3
def ramp(dr, N):
    """Fourier-shift phase ramp exp(-2 pi i dr . nu), nu in cycles/pixel (Eq. fourier_shift)."""
    f = freq(N)
    return np.exp(-2j * np.pi * (dr[0] * f[:, None] + dr[1] * f[None, :]))


def fourier_shift(P, dr):
    """psi_shifted(r) = P(r - dr): inverse DFT_- of DFT_-[P] times the ramp (Eq. fourier_shift)."""
    return idft_minus(dft_minus(P) * ramp(dr, P.shape[-1]))


# ------------------------------------------------------------------ S4, S5
def transmission(d, b, kdz):
    """exp(-k beta dz) exp(i k delta dz) (Eq. ri_modulation)."""
    return np.exp(-kdz * b) * np.exp(1j * kdz * d)


def fresnel_kernel(N, lambda_d_over_px2):
    """Paraxial kernel H1 = exp(i pi lambda d |nu|^2) with nu in cycles/pixel (Eq. paraxial_kernel)."""
    f = freq(N)
    return np.exp(1j * np.pi * lambda_d_over_px2 * (f[:, None] ** 2 + f[None, :] ** 2))


def near_field_kernel(N, nf):
    """H1 for the sample-detector distance z in pixel units: lambda z / dx^2 = 1 / N_F."""
    return fresnel_kernel(N, 1.0 / nf)


def propagate(phi, H):
    """Fresnel propagation F^-1{F[phi] H} (Eq. fresnel_prop); H is even in nu, so the DFT sign is immaterial."""
    return idft_minus(dft_minus(phi) * H)


def propagate_T(g, H):
    """Adjoint of ``propagate``: F^-1{F[g] conj(H)}."""
    return idft_minus(dft_minus(g) * np.conj(H))


# ------------------------------------------------------------------ S6
def farfield(phi):
    """Unitary Fraunhofer propagation with a positive exponent (Eq. fraunhofer), DC at [0, 0]."""
    return dft_plus(phi) / phi.shape[-1]


def farfield_T(g):
    """Adjoint of ``farfield``: DFT_- / N."""
    return dft_minus(g) / g.shape[-1]


# ------------------------------------------------------------------ S8, S10
def loss_terms(I, Im, kind, eps):
    """Per-pixel data mismatch: LSQ (Eq. lsq_loss, amplitudes with I + eps) or Poisson (Eq. poisson_loss)."""
    I = np.asarray(I, np.float64); Im = np.asarray(Im, np.float64)
    if kind == "lsq":
        return (np.sqrt(I + eps) - np.sqrt(Im + eps)) ** 2
    if kind == "poisson":
        return I - Im * np.log(I + eps)
    raise ValueError(kind)


def loss_dI(I, Im, kind, eps):
    """d(per-pixel term)/dI for ``loss_terms``."""
    I = np.asarray(I, np.float64); Im = np.asarray(Im, np.float64)
    if kind == "lsq":
        s = np.sqrt(I + eps)
        return (s - np.sqrt(Im + eps)) / s
    if kind == "poisson":
        return 1.0 - Im / (I + eps)
    raise ValueError(kind)


# ------------------------------------------------------------------ forward / adjoint
def _object_frames(pb: Problem, delta, beta):
    d = np.asarray(delta, np.float64); b = np.asarray(beta, np.float64)
    if pb.tomo:
        d, b = rotate(d, pb.theta), rotate(b, pb.theta)
    return d, b


def _slab(pb, vol, b):
    return vol[b * pb.L:(b + 1) * pb.L]


def _multislice(pb, T, psi0):
    """Algorithm 1 MultislicePropagate: modulate by T_j, then Fresnel-propagate (not after the last slice).

    Returns the exit wave phi_{L-1} and the list of pre-modulation fields psi_j.
    """
    psis, psi = [], psi0
    for j in range(pb.L):
        psis.append(psi)
        phi = T[j] * psi
        if j < pb.L - 1:
            psi = propagate(phi, fresnel_kernel(pb.N, pb.gap(j)))   # variable spacing: Sec. 2.2
    return phi, psis


def _multislice_T(pb, T, psis, phibar, kdz):
    """Reverse slice loop: returns psibar_0 and the per-slice (dL/ddelta, dL/dbeta) chunks.

    phi_j = T_j psi_j gives psibar_j = conj(T_j) phibar_j and, with
    dphi/ddelta = i kdz phi, dphi/dbeta = -kdz phi (Eq. ri_modulation):
      dL/ddelta_j = kdz Im(psibar_j conj(psi_j)),  dL/dbeta_j = -kdz Re(psibar_j conj(psi_j))
    summed over probe modes; phibar_{j-1} = P^H psibar_j.  Also returns dL/dc_j for the slice
    gaps c_j = lambda dz_j / dx^2 (slice-position refinement, Sec. 2.3.2): with
    psi_{j+1} = F^-1{F[phi_j] H_j}, dH_j/dc = i pi |f|^2 H_j and Parseval,
      dL/dc_j = Re[(1/N^2) sum_nu conj(F[psibar_{j+1}]) i pi |f|^2 F[psi_{j+1}]].
    """
    N = pb.N
    f = freq(N)
    f2 = f[:, None] ** 2 + f[None, :] ** 2
    gd = np.zeros((pb.L, N, N)); gb = np.zeros((pb.L, N, N))
    g_gap = np.zeros(max(pb.L - 1, 0))
    for j in range(pb.L - 1, -1, -1):
        if j < pb.L - 1:
            g_gap[j] = np.real(np.sum(np.conj(dft_minus(psibar)) * 1j * np.pi * f2 * dft_minus(psis[j + 1]))) / (N * N)
            phibar = propagate_T(psibar, fresnel_kernel(N, pb.gap(j)))
        psibar = np.conj(T[j]) * phibar
        z = psibar * np.conj(psis[j])
        gd[j] = kdz * np.sum(z.imag, axis=0)
        gb[j] = -kdz * np.sum(z.real, axis=0)
    return psibar, gd, gb, g_gap


def _farfield_position(pb, d, b, probe_hat, p0, dr):
    o_d = take_chunk(d, p0, pb.N); o_b = take_chunk(b, p0, pb.N)
    T = transmission(o_d, o_b, pb.kdz)[:, None]                 # [L, 1, N, N]
    rp = ramp(dr, pb.N)
    psi0 = idft_minus(probe_hat * rp)                            # [M, N, N]
    phi, psis = _multislice(pb, T, psi0)
    Psi = farfield(phi)
    return Psi, T, psis, rp


def _nearfield_problem(pb, d, b, probe, bi, shifts):
    T = transmission(_slab(pb, d, bi), _slab(pb, b, bi), pb.kdz)[:, None]
    phi, psis = _multislice(pb, T, np.asarray(probe, np.complex128))
    Phi = dft_minus(phi)                                         # shared by all distances
    G = [near_field_kernel(pb.N, nf) * ramp(shifts[di], pb.N) for di, nf in enumerate(pb.nf)]
    Psi = np.stack([idft_minus(Phi * g) for g in G])             # [n_dist, M, N, N]
    return Psi, Phi, G, T, psis


def forward(problem, delta, beta, probe, pos):
    """Predicted intensities: far field [B, N, N]; near field [B, n_dist, N, N] (Eq. multimode)."""
    pb = problem if isinstance(problem, Problem) else Problem.of(problem)
    d, b = _object_frames(pb, delta, beta)
    probe = np.asarray(probe, np.complex128)
    if pb.farfield:
        p0, dr = split_positions(pos)
        P_hat = dft_minus(probe)
        out = np.empty((pb.B, pb.N, pb.N))
        for i in range(pb.B):
            Psi = _farfield_position(pb, d, b, P_hat, p0[i], dr[i])[0]
            out[i] = np.sum(np.abs(Psi) ** 2, axis=0)
        return out
    shifts = np.asarray(pos, np.float64)
    out = np.empty((pb.B, len(pb.nf), pb.N, pb.N))
    for i in range(pb.B):
        Psi = _nearfield_problem(pb, d, b, probe, i, shifts[i])[0]
        out[i] = np.sum(np.abs(Psi) ** 2, axis=1)
    return out


def loss(problem, delta, beta, probe, pos, I_meas):
    """Mean data mismatch over every detector pixel of the batch (reading of 1/N_d in Eqs. lsq/poisson_loss)."""
    pb = problem if isinstance(problem, Problem) else Problem.of(problem)
    I = forward(pb, delta, beta, probe, pos)
    return float(np.mean(loss_terms(I, I_meas, pb.loss, pb.eps)))


def loss_grad(problem, delta, beta, probe, pos, I_meas, want_nf=False, want_gaps=False):
    """Loss and its gradients w.r.t. delta, beta (volume frame), probe and positions/shifts.

    Returns (loss, g_delta, g_beta, g_probe, g_pos) in FP64 / complex128; with want_nf (near
    field) also g_nf [B, n_dist], the gradient w.r.t. each problem's Fresnel numbers (the
    free-propagation distance refinement of Sec. 2.3.2: N_F = dx^2 / (lambda z)); with want_gaps
    also g_gaps [L-1], the gradient w.r.t. the slice gaps lambda dz_j / dx^2 (slice positions).
    """
    pb = problem if isinstance(problem, Problem) else Problem.of(problem)
    d, b = _object_frames(pb, delta, beta)
    probe = np.asarray(probe, np.complex128)
    I_meas = np.asarray(I_meas, np.float64)
    N = pb.N
    gvd = np.zeros(d.shape); gvb = np.zeros(b.shape)
    g_probe = np.zeros(probe.shape, np.complex128)
    g_gaps = np.zeros(max(pb.L - 1, 0))
    total = 0.0
    if pb.farfield:
        npix = pb.B * N * N
        p0, dr = split_positions(pos)
        P_hat = dft_minus(probe)
        f = freq(N)
        g_pos = np.zeros((pb.B, 2))
        for i in range(pb.B):
            Psi, T, psis, rp = _farfield_position(pb, d, b, P_hat, p0[i], dr[i])
            I = np.sum(np.abs(Psi) ** 2, axis=0)
            total += np.sum(loss_terms(I, I_meas[i], pb.loss, pb.eps))
            gI = loss_dI(I, I_meas[i], pb.loss, pb.eps) / npix
            Psibar = 2.0 * gI * Psi                              # dI = 2 Re(conj(Psi) dPsi)
            phibar = farfield_T(Psibar)
            psibar0, gd, gb, gg = _multislice_T(pb, T[:, :, :, :], psis, phibar, pb.kdz)
            g_gaps += gg
            put_chunk_T(gvd, p0[i], gd); put_chunk_T(gvb, p0[i], gb)
            Q = dft_minus(psibar0)                               # [M, N, N]
            g_probe += idft_minus(Q * np.conj(rp))
            # d psi0 / d dr_a = IDFT_-{P_hat ramp (-2 pi i nu_a)}; Parseval gives the 1/N^2 form
            base = np.conj(Q) * P_hat * rp
            g_pos[i, 0] = np.real(np.sum(base * (-2j * np.pi * f[:, None]))) / (N * N)
            g_pos[i, 1] = np.real(np.sum(base * (-2j * np.pi * f[None, :]))) / (N * N)
    else:
        nd = len(pb.nf)
        npix = pb.B * nd * N * N
        shifts = np.asarray(pos, np.float64)
        f = freq(N)
        g_pos = np.zeros((pb.B, nd, 2))
        g_nf = np.zeros((pb.B, nd))
        f2 = f[:, None] ** 2 + f[None, :] ** 2
        for i in range(pb.B):
            Psi, Phi, G, T, psis = _nearfield_problem(pb, d, b, probe, i, shifts[i])
            I = np.sum(np.abs(Psi) ** 2, axis=1)                 # [n_dist, N, N]
            total += np.sum(loss_terms(I, I_meas[i], pb.loss, pb.eps))
            gI = loss_dI(I, I_meas[i], pb.loss, pb.eps) / npix
            Phibar_sum = np.zeros_like(Phi)
            for di in range(nd):
                Q = dft_minus(2.0 * gI[di] * Psi[di])            # [M, N, N]
                Phibar_sum += np.conj(G[di]) * Q
                base = np.conj(Q) * Phi * G[di]
                g_pos[i, di, 0] = np.real(np.sum(base * (-2j * np.pi * f[:, None]))) / (N * N)
                g_pos[i, di, 1] = np.real(np.sum(base * (-2j * np.pi * f[None, :]))) / (N * N)
                # dH_d/dN_F = -i pi |f|^2 / N_F^2 H_d (Eq. paraxial_kernel with lambda z / dx^2 = 1 / N_F)
                g_nf[i, di] = np.real(np.sum(base * (-1j * np.pi * f2 / pb.nf[di] ** 2))) / (N * N)
            phibar = idft_minus(Phibar_sum)
            psibar0, gd, gb, gg = _multislice_T(pb, T, psis, phibar, pb.kdz)
            g_gaps += gg
            gvd[i * pb.L:(i + 1) * pb.L] += gd
            gvb[i * pb.L:(i + 1) * pb.L] += gb
            g_probe += psibar0
    if pb.tomo:
        gvd, gvb = rotate_T(gvd, pb.theta), rotate_T(gvb, pb.theta)
    out = (total / npix, gvd, gvb, g_probe, g_pos)
    if want_nf:
        if pb.farfield:
            raise ValueError("Fresnel-number gradients are defined for the near-field geometry")
        out = out + (g_nf,)
    if want_gaps:
        out = out + (g_gaps,)
    return out


# ------------------------------------------------------------------ per-angle position offset
def offset_loss_grad(problem, delta, beta, probe, pos, I_meas):
    """Loss and its gradient w.r.t. one position offset o shared by every position of the batch
    (the per-angle probe-position offset of ptychotomography, Sec. 2.3.2 "Probe position offset":
    one correction vector applies to all probe positions of an angle).  The model sees
    pos_b + o for every b, so by the chain rule dL/do = sum_b dL/dpos_b.  Returns (loss, [2]).
    """
    pb = problem if isinstance(problem, Problem) else Problem.of(problem)
    if not pb.farfield:
        raise ValueError("the position offset is defined for the far-field geometry")
    out = loss_grad(pb, delta, beta, probe, pos, I_meas)
    return out[0], np.sum(out[4], axis=0)

