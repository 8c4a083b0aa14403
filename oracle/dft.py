"""Naive discrete Fourier transforms for the oracle (test infrastructure only).

The oracle's spectral convention (Sec. 3.2: every operator is a Fourier
multiplier on the periodic grid) is the unnormalised forward sum

    F[m] = sum_j f[j] exp(-2 pi i m j / n),      f[j] = (1/n) sum_m F[m] exp(+2 pi i m j / n).

``dft`` evaluates that sum literally as a dense matrix product, O(n^2) per
line; the exponent is reduced modulo n in integers first so the matrix entries
are exact to one rounding. ``scipy.fft`` computes the same sums and serves as
the fast backend for large grids, with its lines spread over all host cores
(``workers``); tests check it against the defining sum, against ``numpy.fft``
and against closed forms (delta, single exponential, Parseval, shift theorem).
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft

WORKERS = os.cpu_count() or 1

_CACHE: dict = {}


def dft_matrix(n: int, inverse: bool = False) -> np.ndarray:
    """E[m, j] = exp(-+2 pi i (m j mod n) / n) (no 1/n factor)."""
    key = (n, inverse)
    E = _CACHE.get(key)
    if E is None:
        j = np.arange(n, dtype=np.int64)
        mj = np.outer(j, j) % n
        sgn = 1.0 if inverse else -1.0
        E = np.exp(sgn * 2j * np.pi * mj / n)
        if n * n <= 4_000_000:
            _CACHE[key] = E
    return E


def dft(x: np.ndarray, axis: int = -1, inverse: bool = False) -> np.ndarray:
    """Unnormalised DFT along one axis by the defining sum; inverse=True flips the sign only."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[axis]
    E = dft_matrix(n, inverse)
    xm = np.moveaxis(x, axis, -1)
    y = xm @ E.T
    return np.moveaxis(y, -1, axis)


def fwd2(f: np.ndarray, backend: str = "fft") -> np.ndarray:
    """2D unnormalised forward transform over the last two axes [nz][nx]."""
    if backend == "dft":
        return dft(dft(f, -1), -2)
    return sfft.fft2(f, workers=WORKERS)


def inv2(F: np.ndarray, backend: str = "fft") -> np.ndarray:
    """2D inverse transform including the 1/(nz nx) factor."""
    if backend == "dft":
        n = F.shape[-1] * F.shape[-2]
        return dft(dft(F, -1, inverse=True), -2, inverse=True) / n
    return sfft.ifft2(F, workers=WORKERS)
