"""Exact de-aliasing (3N padding) on the GPU against the oracle (Grid pad=3),
and against an even larger oracle padding (4.5N) where the series is exact."""
import numpy as np
import pytest

from oracle import Grid, Oracle, run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _state(n, L, h):
    # every kept mode populated, so that aliasing is visible
    rng = np.random.default_rng(n + 7)
    o = Oracle(Grid(n, n, L, L, h), 1)
    eta = o.physical(o.spectrum(0.05 * rng.standard_normal((n, n))))
    psi = o.physical(o.spectrum(0.2 * rng.standard_normal((n, n))))
    return eta.astype(np.float32), psi.astype(np.float32)


@pytest.mark.parametrize("n,M", [(32, 3), (64, 4), (64, 5), (128, 5)])
def test_pad3_rhs_matches_oracle(zk, n, M):
    L, h = 40.0 * n / 32, 8.0
    e, p = _state(n, L, h)
    s = zk.Zakharov(n, n, L, L, h, M=M, eps=1.0, pad=zk.ZK_PAD_3)
    s.set_state(e, p)
    ge, gp = s.rhs()
    o = Oracle(Grid(n, n, L, L, h, pad=3.0), M, eps=1.0)
    de, dp = o.rhs(o.spectrum(e.astype(np.float64)), o.spectrum(p.astype(np.float64)))
    assert rel(ge, o.physical(de)) < 2e-5 and rel(gp, o.physical(dp)) < 2e-5
    # the DNO is exact: it equals the 4.5N-padded oracle within FP32 rounding,
    # while the 3/2 rule differs from it by its aliasing error
    o45 = Oracle(Grid(n, n, L, L, h, pad=4.5), M, eps=1.0)
    v45 = o45.physical(o45.dno(o45.spectrum(e.astype(np.float64)), o45.spectrum(p.astype(np.float64))))
    v = s.dno()
    assert rel(v, v45) < 2e-5
    t = zk.Zakharov(n, n, L, L, h, M=M, eps=1.0)
    t.set_state(e, p)
    assert rel(t.dno(), v45) > 1e-4


def test_pad3_steps_match_oracle(zk):
    n, L, h, M = 64, 80.0, 8.0, 4
    e, p = _state(n, L, h)
    s = zk.Zakharov(n, n, L, L, h, M=M, eps=0.5, pad=zk.ZK_PAD_3)
    s.set_state(e, p)
    s.step(0.01, 20)
    o = Oracle(Grid(n, n, L, L, h, pad=3.0), M, eps=0.5)
    oe, op = run(o, e.astype(np.float64), p.astype(np.float64), 0.01, 20)
    ge, gp = s.get_state()
    tol = 4 * 20 * 2.0 ** -24
    assert rel(ge, oe) < tol and rel(gp, op) < tol


def test_pad3_limits(zk):
    with pytest.raises(zk.ZkError) as e:
        zk.zk_create_ex(64, 64, 10.0, 10.0, 5.0, 9.81, 3, zk.ZK_F64, zk.ZK_PAD_3)
    assert e.value.status == zk.ZK_EUNSUPPORTED
    with pytest.raises(zk.ZkError) as e:
        zk.zk_create_ex(2048, 2048, 10.0, 10.0, 5.0, 9.81, 3, zk.ZK_F32, zk.ZK_PAD_3)
    assert e.value.status == zk.ZK_EUNSUPPORTED
    with pytest.raises(zk.ZkError) as e:
        zk.zk_create_ex(64, 64, 10.0, 10.0, 5.0, 9.81, 3, zk.ZK_F32, 2)
    assert e.value.status == zk.ZK_EINVAL
