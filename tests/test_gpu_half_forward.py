"""The row rounds' half-length forward transform of the real Phi(r) against the oracle.

At 2048^2 the padded rows (3072 points) run the forward transform of each intermediate
round's Phi(r) as x[2n] + i x[2n+1] through the 1536-point plan, followed by the split into
the 3072-point spectrum. Rounds whose block width does not divide the plan's first-stage
stride (three line groups) keep the full-length transform, so orders 2, 3, 4 and 6 together
take both paths (order 6's fifth round has three lines). One right-hand side per order is
compared with the FP64 oracle on the same seeded sea: relative L2 below 2e-5 (the full-size
bar of test_gpu_fullsize.py) and relative max-norm below four times that.
"""
import numpy as np
import pytest

from oracle import Grid, Oracle
from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu

N, L, H, EPS = 2048, 1600.0, 50.0, 0.5


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


@pytest.fixture(scope="module")
def sea():
    eta, psi, _ = seas.jonswap_sea(N, N, L, L, H, 4.0, 12.0, 11)
    return eta.astype(np.float32), psi.astype(np.float32)


@pytest.mark.parametrize("M", [2, 3, 4, 6])
def test_rhs_every_order_at_3072_point_rows(zk, sea, M):
    eta, psi = sea
    o = Oracle(Grid(N, N, L, L, H), M, eps=EPS)
    de, dp = o.rhs(o.spectrum(eta.astype(np.float64)), o.spectrum(psi.astype(np.float64)))
    de, dp = o.physical(de), o.physical(dp)
    s = zk.Zakharov(N, N, L, L, H, M=M, eps=EPS)
    s.set_state(eta, psi)
    ge, gp = s.rhs()
    s.close()
    for g, r in ((ge, de), (gp, dp)):
        l2 = float(np.linalg.norm(g - r) / np.linalg.norm(r))
        mx = float(np.max(np.abs(g - r)) / np.max(np.abs(r)))
        print(f"M {M}: rel L2 {l2:.3e} rel max {mx:.3e}")
        assert l2 < 2e-5 and mx < 8e-5, (M, l2, mx)
