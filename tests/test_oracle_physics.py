"""Pins of the oracle's forward model against physics and mathematics it does not itself encode.

* identity propagation at dz = 0, composition P(d1) P(d2) = P(d1 + d2);
* closed-form free-space propagation of a Gaussian beam;
* energy conservation (Parseval) through the whole multislice path for a
  pure-phase object;
* the thin-object limit: with no inter-slice propagation the multislice
  result equals the projection approximation (Eq. obj_ri_modulation), and
  the error shrinks as O(dz);
* Fourier shift: an integer shift is a circular roll, shifts compose;
* far field: a positive-exponent transform with DC at [0, 0] (Eq. fraunhofer
  and the sign-convention discussion after it);
* omitting the propagation after the last slice leaves far-field intensities
  unchanged;
* rotation: identity at 0, exact axis transposition at 90 degrees;
* loss terms on a hand-worked 2x2 example (tests/golden/loss_2x2.txt).
"""
import math
import os

import numpy as np
import pytest

from oracle import model
from oracle.dft import freq

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cplx(g, shape):
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def test_identity_propagation_at_zero_distance():
    g = np.random.default_rng(0)
    phi = _cplx(g, (3, 32, 32))
    out = model.propagate(phi, model.fresnel_kernel(32, 0.0))
    np.testing.assert_allclose(out, phi, atol=1e-12)


def test_propagation_composes():
    g = np.random.default_rng(1)
    phi = _cplx(g, (32, 32))
    a = model.propagate(model.propagate(phi, model.fresnel_kernel(32, 0.7)), model.fresnel_kernel(32, 1.9))
    b = model.propagate(phi, model.fresnel_kernel(32, 2.6))
    np.testing.assert_allclose(a, b, atol=1e-11)


def test_gaussian_beam_closed_form():
    """exp(-r^2/w0^2) propagated over lambda*d/dx^2 = c equals
    (pi w0^2/(pi w0^2 - i c)) exp(-pi r^2/(pi w0^2 - i c)) (paraxial solution)."""
    N, w0 = 128, 4.0
    c = 1.5 * math.pi * w0 ** 2                  # beam widens to ~1.8 w0, far from the window edge
    y = np.arange(N) - N / 2.0
    r2 = y[:, None] ** 2 + y[None, :] ** 2
    psi0 = np.exp(-r2 / w0 ** 2)
    q = math.pi * w0 ** 2 - 1j * c
    expect = (math.pi * w0 ** 2 / q) * np.exp(-math.pi * r2 / q)
    out = model.propagate(psi0, model.fresnel_kernel(N, c))
    assert np.max(np.abs(out - expect)) < 1e-10
    # and the opposite distance undoes it
    back = model.propagate(out, model.fresnel_kernel(N, -c))
    assert np.max(np.abs(back - psi0)) < 1e-10


def _small_problem(**kw):
    p = dict(N=16, L=4, M=2, B=3, Lz=4, Ly=24, Lx=24, kdz=253.354, lambda_dz_over_px2=0.3,
             farfield=1, nf=[], loss="lsq", eps=1e-6, tomo=0, theta=0.0)
    p.update(kw)
    return model.Problem.of(p)


def test_parseval_pure_phase_object():
    pb = _small_problem()
    g = np.random.default_rng(2)
    delta = g.uniform(0, 2e-3, (pb.Lz, pb.Ly, pb.Lx))
    beta = np.zeros_like(delta)
    probe = _cplx(g, (pb.M, pb.N, pb.N))
    pos = np.array([[3.2, 4.7], [-5.4, 2.1], [10.3, 12.6]])   # second patch leaves the volume
    I = model.forward(pb, delta, beta, probe, pos)
    e_in = np.sum(np.abs(probe) ** 2)
    for i in range(pb.B):
        assert abs(np.sum(I[i]) - e_in) / e_in < 1e-12
    # absorption removes energy
    I2 = model.forward(pb, delta, delta * 0.1, probe, pos)
    assert np.all(np.sum(I2, axis=(1, 2)) < e_in)


def _projection_reference(pb, delta, beta, probe, pos):
    """Eq. obj_ri_modulation + shifted probe + far field, via numpy's FFT library."""
    out = []
    N = pb.N
    f = np.fft.fftfreq(N)
    for p in pos:
        p0 = np.floor(p + 0.5); dr = p - p0
        y0, x0 = int(p0[0]), int(p0[1])
        sd = delta[:, y0:y0 + N, x0:x0 + N].sum(0); sb = beta[:, y0:y0 + N, x0:x0 + N].sum(0)
        rp = np.exp(-2j * np.pi * (dr[0] * f[:, None] + dr[1] * f[None, :]))
        psi0 = np.fft.ifft2(np.fft.fft2(probe) * rp)
        ex = psi0 * np.exp(-pb.kdz * sb) * np.exp(1j * pb.kdz * sd)
        Psi = np.fft.ifft2(ex) * N            # (1/N) * sum exp(+2 pi i ...)
        out.append(np.sum(np.abs(Psi) ** 2, axis=0))
    return np.array(out)


def test_thin_object_limit_equals_projection():
    pb = _small_problem(lambda_dz_over_px2=0.0)
    g = np.random.default_rng(3)
    delta = g.uniform(0, 1e-3, (pb.Lz, pb.Ly, pb.Lx)); beta = g.uniform(0, 1e-4, delta.shape)
    probe = _cplx(g, (pb.M, pb.N, pb.N))
    pos = np.array([[3.2, 4.7], [1.4, 2.1], [6.3, 7.6]])
    I = model.forward(pb, delta, beta, probe, pos)
    ref = _projection_reference(pb, delta, beta, probe, pos)
    assert np.linalg.norm(I - ref) / np.linalg.norm(ref) < 1e-12
    # first-order convergence in the slice spacing
    errs = []
    for c in (0.02, 0.01):
        Ic = model.forward(_small_problem(lambda_dz_over_px2=c), delta, beta, probe, pos)
        errs.append(np.linalg.norm(Ic - ref))
    assert 1.7 < errs[0] / errs[1] < 2.3


def test_integer_fourier_shift_is_roll():
    g = np.random.default_rng(4)
    P = _cplx(g, (2, 16, 16))
    np.testing.assert_allclose(model.fourier_shift(P, np.array([3.0, -2.0])),
                               np.roll(P, (3, -2), axis=(1, 2)), atol=1e-12)


def test_fourier_shifts_compose_and_invert():
    g = np.random.default_rng(5)
    P = _cplx(g, (16, 16))
    a, b = np.array([0.3, -0.45]), np.array([-0.2, 0.15])
    np.testing.assert_allclose(model.fourier_shift(model.fourier_shift(P, a), b),
                               model.fourier_shift(P, a + b), atol=1e-12)
    # adjoint of a shift is the opposite shift
    Q = _cplx(g, (16, 16))
    lhs = np.vdot(Q, model.fourier_shift(P, a))
    rhs = np.vdot(model.fourier_shift(Q, -a), P)
    assert abs(lhs - rhs) < 1e-10


def test_farfield_sign_and_dc_position():
    N = 16
    y, x = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    pw = np.exp(2j * np.pi * (2 * y + 5 * x) / N)
    Psi = model.farfield(pw)
    k = np.argmax(np.abs(Psi))
    assert np.unravel_index(k, Psi.shape) == ((-2) % N, (-5) % N)   # positive exponent
    assert abs(Psi[(-2) % N, (-5) % N] - N) < 1e-10                 # unitary scaling
    const = np.full((N, N), 2.0 + 0j)
    assert abs(model.farfield(const)[0, 0] - 2.0 * N) < 1e-10       # DC at [0, 0]


def test_last_slice_propagation_does_not_change_farfield_intensity():
    pb = _small_problem()
    g = np.random.default_rng(6)
    phi = _cplx(g, (16, 16))
    H = model.fresnel_kernel(16, pb.lambda_dz_over_px2)
    a = np.abs(model.farfield(phi)) ** 2
    b = np.abs(model.farfield(model.propagate(phi, H))) ** 2
    np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-11)


def test_rotation_identity_and_quarter_turn():
    g = np.random.default_rng(7)
    vol = g.standard_normal((9, 4, 9))
    np.testing.assert_allclose(model.rotate(vol, 0.0), vol, atol=1e-14)
    r = model.rotate(vol, math.pi / 2)
    # x0 = -(z_t - c) + c, z0 = (x_t - c) + c  ->  r[z_t, :, x_t] = vol[x_t, :, 8 - z_t]
    expect = np.transpose(vol, (2, 1, 0))[::-1, :, :]
    np.testing.assert_allclose(r, expect, atol=1e-12)


def test_loss_terms_hand_example():
    """Hand-worked values: see tests/golden/loss_2x2.txt."""
    rows = {}
    with open(os.path.join(GOLDEN, "loss_2x2.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                rows[k.strip()] = [float(t) for t in v.split()]
    I = np.array(rows["I"]).reshape(2, 2); Im = np.array(rows["I_meas"]).reshape(2, 2)
    np.testing.assert_allclose(np.mean(model.loss_terms(I, Im, "lsq", 0.0)), rows["lsq_mean"][0], rtol=1e-14)
    np.testing.assert_allclose(np.mean(model.loss_terms(I, Im, "poisson", 0.0)), rows["poisson_mean"][0], rtol=1e-14)
    np.testing.assert_allclose(model.loss_dI(I, Im, "lsq", 0.0).ravel(), rows["lsq_dI"], rtol=1e-14)
    np.testing.assert_allclose(model.loss_dI(I, Im, "poisson", 0.0).ravel(), rows["poisson_dI"], rtol=1e-14)


def test_poisson_stationary_point():
    I = np.array([0.5, 3.0, 40.0]); eps = 1e-3
    np.testing.assert_allclose(model.loss_dI(I, I + eps, "poisson", eps), 0.0, atol=1e-15)
    np.testing.assert_allclose(model.loss_dI(I, I, "lsq", eps), 0.0, atol=1e-15)


def test_split_positions_rounding():
    p0, dr = model.split_positions(np.array([[2.49, -0.5], [2.5, 3.0]]))
    np.testing.assert_array_equal(p0, [[2, 0], [3, 3]])
    np.testing.assert_allclose(dr, [[0.49, -0.5], [-0.5, 0.0]])


def test_nearfield_integer_shift_rolls_hologram():
    pb = model.Problem.of(dict(N=16, L=1, M=1, B=1, Lz=1, Ly=16, Lx=16, kdz=10.0,
                               lambda_dz_over_px2=0.0, farfield=0, nf=[0.05, 0.1]))
    g = np.random.default_rng(8)
    delta = g.uniform(0, 0.05, (1, 16, 16)); beta = g.uniform(0, 0.005, (1, 16, 16))
    probe = np.ones((1, 16, 16), complex)
    I0 = model.forward(pb, delta, beta, probe, np.zeros((1, 2, 2)))
    I1 = model.forward(pb, delta, beta, probe, np.array([[[2.0, -3.0], [0.0, 5.0]]]))
    np.testing.assert_allclose(I1[0, 0], np.roll(I0[0, 0], (2, -3), axis=(0, 1)), atol=1e-12)
    np.testing.assert_allclose(I1[0, 1], np.roll(I0[0, 1], (0, 5), axis=(0, 1)), atol=1e-12)
    # large Fresnel number (tiny distance): hologram -> contact image |T|^2
    pb2 = model.Problem.of(dict(pb.__dict__, nf=[1e9]))
    I2 = model.forward(pb2, delta, beta, probe, np.zeros((1, 1, 2)))
    np.testing.assert_allclose(I2[0, 0], np.exp(-2 * 10.0 * beta[0]), rtol=1e-8)


def _golden_kv(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if "=" in line:
                k, v = (t.strip() for t in line.split("=", 1))
                out[k] = v
    return out


def test_delta_phase_sign_by_far_field_peak():
    """A delta ramp with k dz delta = 2 pi a x / N deflects the whole beam into far-field bin
    (0, -a mod N) (tests/golden/phase_ramp_farfield.txt, worked by hand from Eq. ri_modulation and
    Eq. fraunhofer).  Exercises transmission() through the full forward model; flipping the sign of
    its delta phase moves the peak to (0, a)."""
    g = _golden_kv("phase_ramp_farfield.txt")
    N, a = int(g["N"]), int(g["a"])
    kdz = 253.354
    x = np.arange(N, dtype=np.float64)
    delta = np.broadcast_to(2 * math.pi * a * x / (N * kdz), (1, N, N)).copy()
    beta = np.zeros((1, N, N))
    p = dict(N=N, L=1, M=1, B=1, Lz=1, Ly=N, Lx=N, kdz=kdz, lambda_dz_over_px2=0.3, farfield=1, nf=[],
             loss="lsq", eps=1e-6)
    I = model.forward(p, delta, beta, np.ones((1, N, N), np.complex128), np.zeros((1, 2)))[0]
    ky, kx = np.unravel_index(np.argmax(I), I.shape)
    assert (ky, kx) == (int(g["peak_ky"]), int(g["peak_kx"]))
    assert abs(I[ky, kx] - float(g["peak_I"])) < 1e-9
    rest = I.copy()
    rest[ky, kx] = 0.0
    assert np.max(rest) < 1e-18
