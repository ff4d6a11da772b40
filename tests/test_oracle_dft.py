"""Pins of the oracle's naive DFT against definitions it does not itself use.

The oracle builds its transforms from explicit FP64 DFT matrices; here they
are checked against an O(N^4) direct double sum written with ``math``,
against numpy's FFT library (which the oracle never calls), and against the
closed-form transforms of a delta and of a plane wave.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import dft


def _direct(x, sign):
    Ny, Nx = x.shape
    out = np.zeros((Ny, Nx), np.complex128)
    for ky in range(Ny):
        for kx in range(Nx):
            acc = 0j
            for y in range(Ny):
                for xx in range(Nx):
                    acc += x[y, xx] * cmath.exp(sign * 2j * math.pi * (ky * y / Ny + kx * xx / Nx))
            out[ky, kx] = acc
    return out


@pytest.mark.parametrize("shape", [(8, 8), (6, 8), (5, 7)])
@pytest.mark.parametrize("sign", [-1, +1])
def test_dft_matches_direct_double_sum(shape, sign):
    g = np.random.default_rng(1)
    x = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    np.testing.assert_allclose(dft.dft2(x, sign), _direct(x, sign), rtol=0, atol=1e-11)


@pytest.mark.parametrize("N", [16, 64, 128])
def test_dft_matches_numpy_fft(N):
    g = np.random.default_rng(N)
    x = g.standard_normal((2, N, N)) + 1j * g.standard_normal((2, N, N))
    X = dft.dft_minus(x)
    ref = np.fft.fft2(x)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) < 1e-13
    Xp = dft.dft_plus(x)
    refp = np.fft.ifft2(x) * N * N
    assert np.linalg.norm(Xp - refp) / np.linalg.norm(refp) < 1e-13


def test_inverse_roundtrip():
    g = np.random.default_rng(3)
    x = g.standard_normal((32, 32)) + 1j * g.standard_normal((32, 32))
    np.testing.assert_allclose(dft.idft_minus(dft.dft_minus(x)), x, atol=1e-13)


def test_delta_and_plane_wave_closed_forms():
    N = 16
    d = np.zeros((N, N)); d[3, 5] = 1.0
    ky, kx = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    expect = np.exp(-2j * np.pi * (3 * ky + 5 * kx) / N)
    np.testing.assert_allclose(dft.dft_minus(d), expect, atol=1e-13)
    y, x = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    pw = np.exp(2j * np.pi * (2 * y + 7 * x) / N)
    X = dft.dft_minus(pw)
    ref = np.zeros((N, N), complex); ref[2, 7] = N * N
    np.testing.assert_allclose(X, ref, atol=1e-10)


@pytest.mark.parametrize("n", [1, 2, 7, 8, 128])
def test_freq_matches_numpy(n):
    np.testing.assert_array_equal(dft.freq(n), np.fft.fftfreq(n))
    if n % 2 == 0:
        assert dft.freq(n)[n // 2] == -0.5          # Nyquist reading
