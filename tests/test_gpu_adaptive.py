"""Adaptive order on the GPU: the order chosen at each check, the measured
right-hand-side differences against the oracle's, and the stepping at the
chosen order (bitwise equal to a context created with that order)."""
import numpy as np
import pytest

from oracle import Grid, Oracle
from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu

N, L, H = 128, 100.0, 20.0


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


@pytest.fixture(scope="module")
def sea():
    e, p, _ = seas.jonswap_sea(N, N, L, L, H, 2.0, 6.0, 33)
    return e.astype(np.float32), p.astype(np.float32)


def test_measured_differences_match_oracle(zk, sea):
    s = zk.Zakharov(N, N, L, L, H, M=6, eps=1.0)
    s.set_state(*sea)
    zk.zk_set_adaptive_order(s.ctx, 2, 0.0, 10)      # tolerance 0: every order below 6 is measured
    s.step(0.02, 1)
    st = zk.zk_adaptive_status(s.ctx)
    assert st["order"] == 6 and st["checks"] == 1
    o6 = Oracle(Grid(N, N, L, L, H), 6, eps=1.0)
    eh, ph = o6.spectrum(sea[0].astype(np.float64)), o6.spectrum(sea[1].astype(np.float64))
    f6 = o6.rhs(eh, ph)
    n6 = np.sqrt(sum(np.linalg.norm(o6.physical(x)) ** 2 for x in f6))
    prev = np.inf
    for m in range(2, 6):
        fm = Oracle(Grid(N, N, L, L, H), m, eps=1.0).rhs(eh, ph)
        want = np.sqrt(sum(np.linalg.norm(o6.physical(a - b)) ** 2 for a, b in zip(fm, f6))) / n6
        got = st["err"][m - 1]
        # two FP32 right-hand sides, each within 2e-5 of |f|
        assert abs(got - want) <= 4e-5 + 1e-3 * want, (m, got, want)
        assert got < prev                               # the series converges in m
        prev = got
    assert st["err"][5] == 0.0 and st["err"][0] == -1.0


def test_chosen_order_steps_like_that_order(zk, sea):
    s = zk.Zakharov(N, N, L, L, H, M=6, eps=1.0)
    s.set_state(*sea)
    zk.zk_set_adaptive_order(s.ctx, 2, 1e30, 5)       # any order passes: the lowest is taken
    s.step(0.02, 7)
    st = zk.zk_adaptive_status(s.ctx)
    assert st["order"] == 2 and st["checks"] == 2
    p = zk.Zakharov(N, N, L, L, H, M=2, eps=1.0)
    p.set_state(*sea)
    p.step(0.02, 7)
    a, b = s.get_state(np.float32), p.get_state(np.float32)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # a tolerance between orders picks the first order that meets it
    t = zk.Zakharov(N, N, L, L, H, M=6, eps=1.0)
    t.set_state(*sea)
    zk.zk_set_adaptive_order(t.ctx, 2, 0.0, 10)
    t.step(0.02, 1)
    err = zk.zk_adaptive_status(t.ctx)["err"]
    tol = 0.5 * (err[2] + err[3])                      # between orders 3 and 4
    zk.zk_set_adaptive_order(t.ctx, 2, tol, 10)
    t.step(0.02, 1)
    assert zk.zk_adaptive_status(t.ctx)["order"] == 4
    zk.zk_set_adaptive_order(t.ctx, 2, 0.0, 0)         # off: back to order 6
    assert zk.zk_adaptive_status(t.ctx)["order"] == 6


def test_adaptive_arguments(zk, sea):
    s = zk.Zakharov(N, N, L, L, H, M=4, eps=1.0)
    with pytest.raises(zk.ZkError) as e:
        zk.zk_set_adaptive_order(s.ctx, 5, 1e-3, 10)
    assert e.value.status == zk.ZK_EINVAL
    with pytest.raises(zk.ZkError) as e:
        zk.zk_set_adaptive_order(s.ctx, 2, -1.0, 10)
    assert e.value.status == zk.ZK_EINVAL
    zk.zk_set_adaptive_order(s.ctx, 2, 1e-3, 10)
    net = zk.Net()
    with pytest.raises(zk.ZkError) as e:
        zk.zk_closure_set(s.ctx, net.n, 2, np.ones(6), np.ones(2))
    assert e.value.status == zk.ZK_EUNSUPPORTED


def test_ifab2_with_adaptive_order_matches_oracle(zk, sea):
    # a tolerance that every order meets: the first check switches 6 -> 2 before the
    # first step, so the run is the order-2 IF-AB2 run from its IF-Euler bootstrap
    s = zk.Zakharov(N, N, L, L, H, M=6, eps=1.0, precision=zk.ZK_F64)
    zk.zk_set_options(s.ctx, eps=1.0, integrator=zk.ZK_IFAB2)
    s.set_state(sea[0].astype(np.float64), sea[1].astype(np.float64))
    zk.zk_set_adaptive_order(s.ctx, 2, 1e30, 100)
    s.step(0.02, 10)
    o = Oracle(Grid(N, N, L, L, H), 2, eps=1.0)
    eh, ph = o.spectrum(sea[0].astype(np.float64)), o.spectrum(sea[1].astype(np.float64))
    hist = None
    for _ in range(10):
        eh, ph, hist = o.step_ifab2(eh, ph, 0.02, hist)
    ge, gp = s.get_state()
    assert np.linalg.norm(ge - o.physical(eh)) / np.linalg.norm(o.physical(eh)) < 1e-10


def test_ifrk4_with_adaptive_order_matches_oracle(zk, sea):
    # as for IF-AB2: every order meets the tolerance, so the first check switches 6 -> 2 and the
    # run is the order-2 IF-RK4 run of the oracle
    s = zk.Zakharov(N, N, L, L, H, M=6, eps=1.0, precision=zk.ZK_F64)
    zk.zk_set_options(s.ctx, eps=1.0, integrator=zk.ZK_IFRK4)
    s.set_state(sea[0].astype(np.float64), sea[1].astype(np.float64))
    zk.zk_set_adaptive_order(s.ctx, 2, 1e30, 100)
    s.step(0.02, 10)
    assert zk.zk_adaptive_status(s.ctx)["order"] == 2
    o = Oracle(Grid(N, N, L, L, H), 2, eps=1.0)
    eh, ph = o.spectrum(sea[0].astype(np.float64)), o.spectrum(sea[1].astype(np.float64))
    for _ in range(10):
        eh, ph = o.step_ifrk4(eh, ph, 0.02)
    ge, gp = s.get_state()
    assert np.linalg.norm(ge - o.physical(eh)) / np.linalg.norm(o.physical(eh)) < 1e-10
    assert np.linalg.norm(gp - o.physical(ph)) / np.linalg.norm(o.physical(ph)) < 1e-10
