"""Pins for the oracle's transforms: the naive DFT against closed forms and numpy.fft."""
import numpy as np
import pytest

from oracle.dft import dft, fwd2, inv2

SIZES = [1, 2, 3, 4, 6, 8, 12, 16, 24, 48, 64, 96, 128, 192, 384]


@pytest.mark.parametrize("n", SIZES)
def test_dft_matches_library_fft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    np.testing.assert_allclose(dft(x), np.fft.fft(x), rtol=0, atol=1e-12 * max(1, n))
    np.testing.assert_allclose(dft(x, inverse=True) / n, np.fft.ifft(x), rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [8, 96, 384])
def test_dft_closed_forms(n):
    # delta at j0 -> exp(-2 pi i m j0 / n); single exponential -> n at one bin
    j0, m0 = 3, 5
    d = np.zeros(n)
    d[j0] = 1.0
    m = np.arange(n)
    np.testing.assert_allclose(dft(d), np.exp(-2j * np.pi * m * j0 / n), atol=1e-13)
    e = np.exp(2j * np.pi * m0 * np.arange(n) / n)
    want = np.zeros(n, complex)
    want[m0] = n
    np.testing.assert_allclose(dft(e), want, atol=1e-11)


@pytest.mark.parametrize("n", [12, 96, 384])
def test_dft_parseval_shift_roundtrip(n):
    rng = np.random.default_rng(7 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = dft(x)
    assert abs(np.sum(abs(x) ** 2) - np.sum(abs(X) ** 2) / n) < 1e-12 * np.sum(abs(x) ** 2)
    s = 5
    Xs = dft(np.roll(x, s))
    np.testing.assert_allclose(Xs, X * np.exp(-2j * np.pi * np.arange(n) * s / n), atol=1e-11)
    np.testing.assert_allclose(dft(X, inverse=True) / n, x, atol=1e-13)


def test_2d_backends_agree():
    rng = np.random.default_rng(3)
    f = rng.standard_normal((24, 48))
    np.testing.assert_allclose(fwd2(f, "dft"), fwd2(f, "fft"), atol=1e-10)
    F = fwd2(f, "fft")
    np.testing.assert_allclose(inv2(F, "dft").real, f, atol=1e-13)


@pytest.mark.parametrize("shape", [(48, 96), (192, 128), (384, 384)])
def test_fast_backend_matches_defining_sum(shape):
    # the multi-threaded library backend against the literal sums, forward and inverse
    rng = np.random.default_rng(shape[0])
    f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    F = fwd2(f, "fft")
    np.testing.assert_allclose(F, fwd2(f, "dft"), rtol=0, atol=1e-11 * np.max(np.abs(F)))
    np.testing.assert_allclose(inv2(F, "fft"), inv2(F, "dft"), rtol=0, atol=1e-13 * np.max(np.abs(f)))
    np.testing.assert_allclose(inv2(F, "fft"), f, rtol=0, atol=1e-13 * np.max(np.abs(f)))
