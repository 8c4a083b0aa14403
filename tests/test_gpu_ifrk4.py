"""Integrating-factor RK4 on the GPU against the oracle's Lawson step."""
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


@pytest.mark.parametrize("prec", [1, 0])
def test_ifrk4_matches_oracle(zk, prec):
    n, L, h, M = 64, 100.0, 20.0, 4
    e, p, _ = seas.jonswap_sea(n, n, L, L, h, 1.5, 7.0, 12)
    e, p = e.astype(np.float32), p.astype(np.float32)
    o = Oracle(Grid(n, n, L, L, h), M, eps=0.8)
    oe, op = run(o, e.astype(np.float64), p.astype(np.float64), 0.05, 20, integrator="ifrk4")
    s = zk.Zakharov(n, n, L, L, h, M=M, eps=0.8, precision=prec)
    zk.zk_set_options(s.ctx, eps=0.8, integrator=zk.ZK_IFRK4)
    if prec == 1:
        s.set_state(e.astype(np.float64), p.astype(np.float64))
    else:
        s.set_state(e, p)
    s.step(0.05, 20)
    ge, gp = s.get_state()
    tol = 1e-10 if prec == 1 else 4 * 20 * 2.0 ** -24
    assert rel(ge, oe) < tol and rel(gp, op) < tol


def test_ifrk4_eps0_exact_linear_flow(zk):
    # eps = 0 and no filter: the step is the exact rotation for any dt (FP64)
    n, L, h = 64, 100.0, 20.0
    e, p, _ = seas.jonswap_sea(n, n, L, L, h, 1.0, 8.0, 5)
    s = zk.Zakharov(n, n, L, L, h, M=3, eps=0.0, precision=zk.ZK_F64, filter=False)
    zk.zk_set_options(s.ctx, eps=0.0, integrator=zk.ZK_IFRK4, filter=0)
    s.set_state(e, p)
    s.step(0.5, 6)
    o = Oracle(Grid(n, n, L, L, h), 3, eps=0.0, filt=False)
    we, wp = o.linear_propagate(o.spectrum(e), o.spectrum(p), 3.0)
    ge, gp = s.get_state()
    assert rel(ge, o.physical(we)) < 1e-12 and rel(gp, o.physical(wp)) < 1e-12


def test_ifrk4_config1_fp64_200_steps(zk):
    """Config 1 (64^2, L = 100 m, h = 20 m, M = 3, seed 1, eps = 1, dt = 0.02 s, filter on):
    200 IF-RK4 steps in FP64 against the oracle, the bar of the RK4 config-1 run (1e-10), and
    the Hamiltonian at the end to 1e-12."""
    e, p, _ = seas.jonswap_sea(64, 64, 100.0, 100.0, 20.0, 1.0, 8.0, 1)
    o = Oracle(Grid(64, 64, 100.0, 100.0, 20.0), 3)
    oe, op = run(o, e, p, 0.02, 200, integrator="ifrk4")
    s = zk.Zakharov(64, 64, 100.0, 100.0, 20.0, M=3, precision=zk.ZK_F64)
    zk.zk_set_options(s.ctx, eps=1.0, integrator=zk.ZK_IFRK4)
    s.set_state(e, p)
    s.step(0.02, 200)
    ge, gp = s.get_state()
    assert rel(ge, oe) < 1e-10 and rel(gp, op) < 1e-10
    H = o.energy(o.spectrum(oe), o.spectrum(op))[0]
    assert abs(s.energy()[0] - H) / H < 1e-12
