"""The effective roundoff of the split-precision DFT-GEMM product, emulated on the CPU.

With unit roundoff u of the 16-bit format (2^-8 for BF16, 2^-11 for FP16), the rounding of the
low part and the dropped l l' term are each at most u^2 of the operands: 2^-16 (BF16) and
2^-22 (FP16) in the worst case, less on average since |v - h| averages about u/2. The GPU
tests of the split stages hold them to 128x (BF16 x3) and 8x (FP16 x3) the FP32 bar; this
measures the per-block error of the arithmetic itself, so that those factors sit above it
(measured: BF16 x3 rms 2^-18.6, max 2^-17.4, i.e. up to ~100x FP32's 2^-24; FP16 x3 rms
2^-24.4, max 2^-23, i.e. up to 2x). A length-8 DFT is applied to 8-point blocks as
the real product [[Fr, -Fi], [Fi, Fr]] [Re x; Im x]. Each operand v is split into h = rn(v)
and l = rn(v - h) in the 16-bit format, and the three products h h' + h l' + l h' are summed
exactly (FP64 here; FP32 accumulation on the GPU adds its own 2^-24). For FP16, each block is
first scaled by a power of two that puts its largest component in [2^13, 2^14). The result is
compared with the exact DFT-8 (numpy.fft), relative to each block's norm.
"""
import numpy as np


def rn_bf16(x):
    """Round FP32 values to BF16 (round to nearest, ties to even), returned as FP32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def rn_fp16(x):
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def split(v, rn):
    v = np.asarray(v, dtype=np.float32)
    h = rn(v)
    lo = rn((v - h).astype(np.float32))
    return h.astype(np.float64), lo.astype(np.float64)


def split_dft8(x, rn, scale):
    """x: complex [nblocks, 8] -> the split-product DFT-8 of each block."""
    xr, xi = x.real.astype(np.float32), x.imag.astype(np.float32)
    s = np.ones(x.shape[0], dtype=np.float32)
    if scale:
        m = np.maximum(np.abs(xr).max(axis=1), np.abs(xi).max(axis=1))
        e = np.floor(np.log2(np.where(m > 0, m, 1.0)))
        s = (2.0 ** (13 - e)).astype(np.float32)
        xr, xi = xr * s[:, None], xi * s[:, None]
    n = np.arange(8)
    F = np.exp(-2j * np.pi * np.outer(n, n) / 8)
    A = np.block([[F.real, -F.imag], [F.imag, F.real]]).astype(np.float32)
    X = np.concatenate([xr, xi], axis=1).T                 # [16, nblocks]
    Ah, Al = split(A, rn)
    Xh, Xl = split(X, rn)
    D = Al @ Xh + Ah @ Xl + Ah @ Xh                        # [16, nblocks]
    Y = (D[:8] + 1j * D[8:]).T / s[:, None]
    return Y


def rel_err(rn, scale, rng, blocks=4096):
    # blocks of mixed magnitude (the padded lines hold values over many decades)
    mag = 10.0 ** rng.uniform(-3, 3, size=(blocks, 1))
    x = (rng.standard_normal((blocks, 8)) + 1j * rng.standard_normal((blocks, 8))) * mag
    x = x.astype(np.complex64).astype(np.complex128)       # FP32 inputs
    exact = np.fft.fft(x, axis=1)
    got = split_dft8(x, rn, scale)
    return np.linalg.norm(got - exact, axis=1) / np.linalg.norm(exact, axis=1)


def test_bf16x3_roundoff():
    e = rel_err(rn_bf16, False, np.random.default_rng(1))
    rms = np.sqrt(np.mean(e ** 2))
    # below the worst case u^2 = 2^-16, and below the 128 x 2^-24 = 2^-17 the GPU bar assumes
    assert e.max() < 2.0 ** -17 and rms < 2.0 ** -18
    # at the BF16 level, not accidentally exact
    assert rms > 2.0 ** -20


def test_fp16x3_roundoff():
    e = rel_err(rn_fp16, True, np.random.default_rng(2))
    rms = np.sqrt(np.mean(e ** 2))
    # below the worst case u^2 = 2^-22 (and so below the 8 x 2^-24 = 2^-21 the GPU bar assumes)
    assert e.max() < 2.0 ** -22 and rms < 2.0 ** -23
    assert rms > 2.0 ** -26


def test_fp16_without_scaling_overflows():
    # the per-block scale is needed: raw magnitudes above 65504 are not representable
    rng = np.random.default_rng(3)
    x = (rng.standard_normal((16, 8)) * 1e6).astype(np.complex128)
    with np.errstate(over="ignore", invalid="ignore"):
        got = split_dft8(x, rn_fp16, False)
    assert not np.all(np.isfinite(got))
