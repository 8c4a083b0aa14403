"""Split-precision DFT-GEMM stages (the innermost radix-8 stage of every padded
transform on the tensor cores, BF16 x3 or FP16 x3) against the FP64 oracle.

Tolerances follow the FP32 bars of the parity tests, scaled by the per-product
error of the split arithmetic relative to FP32's 2^-24. test_split_roundoff.py
measures that error on a CPU emulation of the same split product (BF16 x3: at
most 2^-17.4, about 100x; FP16 x3: at most 2^-23, 2x); the factors used here,
128 and 8, sit above both. One right-hand side in FP32 is held to 2e-5, so the
split forms are held to 128 * 2e-5 and 8 * 2e-5. Each must also differ from the FP32 result (the
tensor-core stage really runs), and the FP16 form must be the more accurate.
"""
import numpy as np
import pytest

from oracle import Grid, Oracle
from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu

FP32_RHS_BAR = 2e-5
RATIO = {1: 128.0, 2: 8.0}     # mode -> split roundoff / FP32 roundoff


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def sea():
    # the sea workload's sea at 1024^2 (same grid spacing): padded lines of 1536
    n, L, h, M = 1024, 800.0, 50.0, 4
    e, p, _ = seas.jonswap_sea(n, n, L, L, h, 4.0, 12.0, 3)
    e32, p32 = e.astype(np.float32), p.astype(np.float32)
    o = Oracle(Grid(n, n, L, L, h), M, eps=0.5)
    eh, ph = o.spectrum(e32.astype(np.float64)), o.spectrum(p32.astype(np.float64))
    de, dp = o.rhs(eh, ph)
    return dict(n=n, L=L, h=h, M=M, e32=e32, p32=p32, G=o.physical(o.dno(eh, ph)),
                de=o.physical(de), dp=o.physical(dp))


def _ctx(zk, sea, mode):
    s = zk.Zakharov(sea["n"], sea["n"], sea["L"], sea["L"], sea["h"], M=sea["M"], eps=0.5)
    zk.zk_set_dft_precision(s.ctx, mode)
    s.set_state(sea["e32"], sea["p32"])
    return s


def test_split_rhs_and_dno_match_oracle(zk, sea):
    err = {}
    out = {}
    for mode in (zk.ZK_DFT_F32, zk.ZK_DFT_BF16X3, zk.ZK_DFT_FP16X3):
        s = _ctx(zk, sea, mode)
        G = s.dno()
        ge, gp = s.rhs()
        err[mode] = (rel(G, sea["G"]), rel(ge, sea["de"]), rel(gp, sea["dp"]))
        out[mode] = (ge, gp)
        s.close()
    assert max(err[zk.ZK_DFT_F32]) < FP32_RHS_BAR, err
    for mode in (zk.ZK_DFT_BF16X3, zk.ZK_DFT_FP16X3):
        assert max(err[mode]) < RATIO[mode] * FP32_RHS_BAR, (mode, err)
        # the tensor-core stage ran: the result is not the FP32 one
        assert rel(out[mode][0], out[zk.ZK_DFT_F32][0]) > 1e-7, (mode, err)
    assert max(err[zk.ZK_DFT_FP16X3]) < max(err[zk.ZK_DFT_BF16X3]), err


def test_split_steps_and_switch_back(zk, sea):
    """20 RK4 steps in each form stay within the stepped FP32 bar of the
    parity tests (4 * nsteps * u, linear accumulation of one rounding u per
    right-hand side) taken at the split roundoff, plus the FP32 run's own
    share; switching back to FP32 on the same context reproduces the FP32 run
    bitwise."""
    steps, dt = 20, 0.02
    ref = _ctx(zk, sea, zk.ZK_DFT_F32)
    ref.step(dt, steps)
    e_ref = ref.get_state(np.float32)[0]
    for mode in (zk.ZK_DFT_BF16X3, zk.ZK_DFT_FP16X3):
        s = _ctx(zk, sea, mode)
        s.step(dt, steps)
        e = s.get_state(np.float32)[0]
        assert rel(e, e_ref) < 4 * steps * (RATIO[mode] + 1) * 2.0 ** -24, mode
        zk.zk_set_dft_precision(s.ctx, zk.ZK_DFT_F32)
        s.set_state(sea["e32"], sea["p32"])
        s.step(dt, steps)
        assert np.array_equal(s.get_state(np.float32)[0], e_ref), mode
        s.close()
    ref.close()


def test_split_at_2048(zk):
    """Padded lines of 3072 (four warps per line): one right-hand side of the
    sea workload's sea within the same bars of the FP32 result."""
    n, L, h = 2048, 1600.0, 50.0
    e, p, _ = seas.jonswap_sea(n, n, L, L, h, 4.0, 12.0, 3)
    e32, p32 = e.astype(np.float32), p.astype(np.float32)
    res = {}
    for mode in (zk.ZK_DFT_F32, zk.ZK_DFT_BF16X3, zk.ZK_DFT_FP16X3):
        s = zk.Zakharov(n, n, L, L, h, M=5, eps=0.5)
        zk.zk_set_dft_precision(s.ctx, mode)
        s.set_state(e32, p32)
        res[mode] = s.rhs()
        s.close()
    f = res[zk.ZK_DFT_F32]
    for mode in (zk.ZK_DFT_BF16X3, zk.ZK_DFT_FP16X3):
        d = max(rel(res[mode][0], f[0]), rel(res[mode][1], f[1]))
        assert 1e-7 < d < RATIO[mode] * FP32_RHS_BAR, (mode, d)


def test_split_refusals(zk):
    small = zk.Zakharov(256, 256, 200.0, 200.0, 20.0, M=3)
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_set_dft_precision(small.ctx, zk.ZK_DFT_BF16X3)
    assert ei.value.status == zk.ZK_EUNSUPPORTED
    zk.zk_set_dft_precision(small.ctx, zk.ZK_DFT_F32)          # the FP32 form is always accepted
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_set_dft_precision(small.ctx, 3)
    assert ei.value.status == zk.ZK_EINVAL
    f64 = zk.Zakharov(1024, 1024, 800.0, 800.0, 50.0, M=3, precision=zk.ZK_F64)
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_set_dft_precision(f64.ctx, zk.ZK_DFT_FP16X3)
    assert ei.value.status == zk.ZK_EUNSUPPORTED
    s = zk.Zakharov(1024, 1024, 800.0, 800.0, 50.0, M=3)
    zk.zk_set_series_fp64(s.ctx, True)
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_set_dft_precision(s.ctx, zk.ZK_DFT_BF16X3)
    assert ei.value.status == zk.ZK_EUNSUPPORTED
    zk.zk_set_series_fp64(s.ctx, False)
    zk.zk_set_dft_precision(s.ctx, zk.ZK_DFT_BF16X3)
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_set_series_fp64(s.ctx, True)
    assert ei.value.status == zk.ZK_EUNSUPPORTED
    for c in (small, f64, s):
        c.close()
