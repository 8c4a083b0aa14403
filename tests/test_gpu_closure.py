"""The closure inside the Zakharov step (through the C ABI) against the oracle:
features, targets, the corrected right-hand side, RK4 steps, the fallback."""
import numpy as np
import pytest

from oracle import Grid, Oracle
from oracle import closure as cl
from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu

N, L, H, EPS = 64, 50.0, 15.0, 0.5


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def sea():
    e, p, _ = seas.jonswap_sea(N, N, L, L, H, 1.0, 5.0, 41)
    return e.astype(np.float32), p.astype(np.float32)


def _oracles():
    gr = Grid(N, N, L, L, H)
    return gr, Oracle(gr, 2, eps=EPS), Oracle(gr, 6, eps=EPS)


def _theta(seed, scale=0.02):
    rng = np.random.default_rng(seed)
    th = cl.init_params(seed) + scale * rng.standard_normal(cl.param_count())
    return th.astype(np.float32)


IN = np.array([0.3, 0.2, 0.2, 0.5, 0.05, 0.05], np.float32)
OUT = np.array([0.01, 0.02], np.float32)


def test_features_and_target(zk, sea):
    import torch
    gr, o2, o6 = _oracles()
    s = zk.Zakharov(N, N, L, L, H, M=6, eps=EPS)
    s.set_state(*sea)
    f = torch.empty((6, N, N), device="cuda")
    t = torch.empty((2, N, N), device="cuda")
    zk.zk_closure_features(s.ctx, 2, f, t, IN, OUT)
    eh, ph = o2.spectrum(sea[0].astype(np.float64)), o2.spectrum(sea[1].astype(np.float64))
    fo = cl.features(o2, eh, ph, IN)
    to = cl.target(o6, o2, eh, ph, OUT)
    fg = f.cpu().numpy()
    for c in range(6):
        assert rel(fg[c], fo[c]) < 2e-5, c       # one FP32 right-hand side, then a transform
    # the target is a difference of two FP32 right-hand sides: bar relative to f_6's size
    e6, p6 = o6.rhs(eh, ph)
    scale = np.array([np.linalg.norm(o2.physical(e6)) / OUT[0], np.linalg.norm(o2.physical(p6)) / OUT[1]])
    tg = t.cpu().numpy()
    for c in range(2):
        assert np.linalg.norm(tg[c] - to[c]) < 2e-5 * scale[c], c


def test_closure_rhs_and_steps(zk, sea):
    gr, o2, o6 = _oracles()
    theta = _theta(7)
    net = zk.Net(theta)
    s = zk.Zakharov(N, N, L, L, H, M=6, eps=EPS)
    s.set_state(*sea)
    zk.zk_closure_set(s.ctx, net.n, 2, IN, OUT, check_every=0)
    co = cl.ClosureOracle(gr, 2, theta.astype(np.float64), IN, OUT, eps=EPS)
    eh, ph = co.spectrum(sea[0].astype(np.float64)), co.spectrum(sea[1].astype(np.float64))
    de, dp = s.rhs()
    oe, op = co.rhs(eh, ph)
    # f_2 (2e-5) plus the network term (1e-4 of a residual-sized correction)
    assert rel(de, co.physical(oe)) < 3e-5 and rel(dp, co.physical(op)) < 3e-5
    n = 5
    s.step(0.02, n)
    for _ in range(n):
        eh, ph = co.step_rk4(eh, ph, 0.02)
    ge, gp = s.get_state()
    assert rel(ge, co.physical(eh)) < 4 * n * 2.0 ** -24 + 1e-6
    assert rel(gp, co.physical(ph)) < 4 * n * 2.0 ** -24 + 1e-6
    st = zk.zk_closure_status(s.ctx)
    assert st["active"] == 1 and st["checks"] == 0


def test_closure_once_per_step(zk, sea):
    # the network at the first RK stage only, its residual reused by stages 2-4: against the
    # oracle's RK4 with the residual frozen at each step's start state, same bar as above
    gr, o2, o6 = _oracles()
    theta = _theta(7)
    net = zk.Net(theta)
    s = zk.Zakharov(N, N, L, L, H, M=6, eps=EPS)
    s.set_state(*sea)
    zk.zk_closure_set(s.ctx, net.n, 2, IN, OUT, check_every=0)
    zk.zk_closure_set_once_per_step(s.ctx, 1)
    co = cl.ClosureOracle(gr, 2, theta.astype(np.float64), IN, OUT, eps=EPS)
    eh, ph = co.spectrum(sea[0].astype(np.float64)), co.spectrum(sea[1].astype(np.float64))
    n = 5
    s.step(0.02, n)
    for _ in range(n):
        eh, ph = co.step_rk4_frozen(eh, ph, 0.02)
    ge, gp = s.get_state()
    assert rel(ge, co.physical(eh)) < 4 * n * 2.0 ** -24 + 1e-6
    assert rel(gp, co.physical(ph)) < 4 * n * 2.0 ** -24 + 1e-6
    # and it is not the per-stage closure (the frozen residual changes the step)
    e2, p2 = co.spectrum(sea[0].astype(np.float64)), co.spectrum(sea[1].astype(np.float64))
    for _ in range(n):
        e2, p2 = co.step_rk4(e2, p2, 0.02)
    assert rel(co.physical(eh), co.physical(e2)) > 0
    with pytest.raises(zk.ZkError):
        zk.zk_closure_set_once_per_step(s.ctx, 2)


def test_zero_net_is_base_order(zk, sea):
    net = zk.Net(np.zeros(cl.param_count(), np.float32))
    s = zk.Zakharov(N, N, L, L, H, M=6, eps=EPS)
    s.set_state(*sea)
    zk.zk_closure_set(s.ctx, net.n, 2, IN, OUT, check_every=0)
    p = zk.Zakharov(N, N, L, L, H, M=2, eps=EPS)
    p.set_state(*sea)
    s.step(0.02, 5)
    p.step(0.02, 5)
    a, b = s.get_state(np.float32), p.get_state(np.float32)
    assert rel(a[0], b[0].astype(np.float64)) < 1e-6 and rel(a[1], b[1].astype(np.float64)) < 1e-6


def test_check_and_fallback(zk, sea):
    # a net far from the residual fails the first check: the context falls back
    # to order 6 before its first step and then matches a plain order-6 run bitwise
    net = zk.Net(_theta(11, scale=0.5))
    s = zk.Zakharov(N, N, L, L, H, M=6, eps=EPS)
    s.set_state(*sea)
    zk.zk_closure_set(s.ctx, net.n, 2, IN, OUT, check_every=3, check_tol=0.2)
    s.step(0.02, 6)
    st = zk.zk_closure_status(s.ctx)
    assert st["active"] == 0 and st["fallback_step"] == 0 and st["checks"] == 1 and st["last_err"] > 0.2
    p = zk.Zakharov(N, N, L, L, H, M=6, eps=EPS)
    p.set_state(*sea)
    p.step(0.02, 6)
    a, b = s.get_state(np.float32), p.get_state(np.float32)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # a check that passes keeps the closure on and counts every check_every steps
    net0 = zk.Net(np.zeros(cl.param_count(), np.float32))
    s2 = zk.Zakharov(N, N, L, L, H, M=6, eps=EPS)
    s2.set_state(*sea)
    zk.zk_closure_set(s2.ctx, net0.n, 2, IN, OUT, check_every=3, check_tol=1.5)
    s2.step(0.02, 7)
    st = zk.zk_closure_status(s2.ctx)
    assert st["active"] == 1 and st["checks"] == 3 and abs(st["last_err"] - 1.0) < 1e-6


def test_closure_argument_errors(zk, sea):
    net = zk.Net()
    s = zk.Zakharov(N, N, L, L, H, M=3, eps=EPS, precision=zk.ZK_F64)
    with pytest.raises(zk.ZkError) as e:
        zk.zk_closure_set(s.ctx, net.n, 2, IN, OUT)
    assert e.value.status == zk.ZK_EUNSUPPORTED
    s = zk.Zakharov(N, N, L, L, H, M=3, eps=EPS)
    with pytest.raises(zk.ZkError) as e:
        zk.zk_closure_set(s.ctx, net.n, 3, IN, OUT)
    assert e.value.status == zk.ZK_EINVAL
    with pytest.raises(zk.ZkError) as e:
        zk.zk_closure_set(s.ctx, net.n, 2, -IN, OUT)
    assert e.value.status == zk.ZK_EINVAL
