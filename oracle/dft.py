"""Naive FP64 discrete Fourier transforms for the oracle (test infrastructure only).

No FFT library is used: each 1-D transform is the product with an explicit
DFT matrix whose twiddles are exp(sign * 2*pi*i * (j*k mod n) / n), built in
FP64 (reducing j*k modulo n first keeps the argument in [0, 2*pi)).  A 2-D
transform is the row transform followed by the column transform, i.e.
X = F_y @ x @ F_x^T.

Naming (numpy's sign for the forward transform is negative):
  dft_minus(x)   = sum_r x(r) exp(-2*pi*i r.nu)          (numpy fft2)
  dft_plus(x)    = sum_r x(r) exp(+2*pi*i r.nu)          (N^2 * numpy ifft2)
  idft_minus(X)  = dft_plus(X) / N^2                     (inverse of dft_minus)
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np


@lru_cache(maxsize=64)
def dft_matrix(n: int, sign: int) -> np.ndarray:
    j = np.arange(n, dtype=np.int64)
    jk = np.outer(j, j) % n
    return np.exp(sign * 2j * np.pi * jk.astype(np.float64) / n)


def dft2(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised 2-D DFT over the last two axes with exponent sign ``sign``."""
    x = np.asarray(x, np.complex128)
    Fy = dft_matrix(x.shape[-2], sign)
    Fx = dft_matrix(x.shape[-1], sign)
    return Fy @ x @ Fx.T


def dft_minus(x):
    return dft2(x, -1)


def dft_plus(x):
    return dft2(x, +1)


def idft_minus(X):
    X = np.asarray(X)
    return dft2(X, +1) / (X.shape[-2] * X.shape[-1])


def freq(n: int) -> np.ndarray:
    """Sample frequencies in cycles per pixel, DC first; for even n index n/2 maps to -1/2."""
    k = np.arange(n)
    return np.where(k <= (n - 1) // 2, k, k - n).astype(np.float64) / n
