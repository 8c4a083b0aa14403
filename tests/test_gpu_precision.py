"""Precision form: FP32 context with FP64 series sums (GPU) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import Grid, Oracle, run
from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,M", [(64, 3), (64, 5), (128, 6)])
def test_series64_rhs_matches_oracle(zk, n, M):
    L = n * 1.5
    e, p, _ = seas.jonswap_sea(n, n, L, L, 20.0, 1.5, 6.0, 17)
    e32, p32 = e.astype(np.float32), p.astype(np.float32)
    o = Oracle(Grid(n, n, L, L, 20.0), M, eps=0.7)
    de, dp = o.rhs(o.spectrum(e32.astype(np.float64)), o.spectrum(p32.astype(np.float64)))
    s = zk.Zakharov(n, n, L, L, 20.0, M=M, eps=0.7)
    zk.zk_set_series_fp64(s.ctx, True)
    s.set_state(e32, p32)
    ge, gp = s.rhs()
    assert rel(ge, o.physical(de)) < 2e-5 and rel(gp, o.physical(dp)) < 2e-5
    # switching back gives the plain FP32 result, bitwise
    zk.zk_set_series_fp64(s.ctx, False)
    a = s.rhs(np.float32)
    t = zk.Zakharov(n, n, L, L, 20.0, M=M, eps=0.7)
    t.set_state(e32, p32)
    b = t.rhs(np.float32)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_series64_steps_config1(zk):
    e, p, _ = seas.jonswap_sea(64, 64, 100.0, 100.0, 20.0, 1.0, 8.0, 1)
    e32, p32 = e.astype(np.float32), p.astype(np.float32)
    o = Oracle(Grid(64, 64, 100.0, 100.0, 20.0), 3)
    oe, op = run(o, e32.astype(np.float64), p32.astype(np.float64), 0.02, 200)
    s = zk.Zakharov(64, 64, 100.0, 100.0, 20.0, M=3)
    zk.zk_set_series_fp64(s.ctx, True)
    s.set_state(e32, p32)
    s.step(0.02, 200)
    ge, gp = s.get_state()
    tol = 4 * 200 * 2.0 ** -24
    assert rel(ge, oe) < tol and rel(gp, op) < tol


def test_series64_fp64_context_is_noop(zk):
    s = zk.Zakharov(64, 64, 100.0, 100.0, 20.0, M=3, precision=zk.ZK_F64)
    zk.zk_set_series_fp64(s.ctx, True)
    assert zk.load().zk_set_series_fp64(s.ctx, 2) == zk.ZK_EINVAL
