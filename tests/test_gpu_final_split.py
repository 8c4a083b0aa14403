"""The final column pass with its update as a separate launch (lines of 1536 points and more)
against the FP64 oracle, in every update mode, and the paper's IF-AB2 at the sea workload's size.

At 1024^2 (1536-point padded columns) the final column kernel stores the transformed nonlinear
parts and fin_epilogue_kernel applies the update over the compact spectra. In an FP64 context
each mode is compared with the oracle: one right-hand side, one RK4 step, two IF-AB2 steps (the
IF-Euler bootstrap, then AB2), one IF-RK4 step and the inverse DNO map (8 fixed-point
iterations). Bar: 1e-11 relative L2 (the FP64 parity bar of the small-grid tests), and the
energy (the fused final pass, FP64 sums) to 1e-12.
"""
import numpy as np
import pytest

from oracle import Grid, Oracle
from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu

N, L, H, M, EPS, DT = 1024, 800.0, 50.0, 4, 0.5, 0.02


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


@pytest.fixture(scope="module")
def case():
    e, p, _ = seas.jonswap_sea(N, N, L, L, H, 4.0, 12.0, 21)
    o = Oracle(Grid(N, N, L, L, H), M, eps=EPS)
    return e, p, o, o.spectrum(e), o.spectrum(p)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _sim(zk, e, p, integrator):
    s = zk.Zakharov(N, N, L, L, H, M=M, eps=EPS, precision=zk.ZK_F64)
    zk.zk_set_options(s.ctx, eps=EPS, integrator=integrator)
    s.set_state(e, p)
    return s


def test_rhs_and_energy(zk, case):
    e, p, o, eh, ph = case
    de, dp = o.rhs(eh, ph)
    s = _sim(zk, e, p, zk.ZK_RK4)
    ge, gp = s.rhs()
    H0 = s.energy()[0]
    s.close()
    assert rel(ge, o.physical(de)) < 1e-11 and rel(gp, o.physical(dp)) < 1e-11
    assert abs(H0 - o.energy(eh, ph)[0]) < 1e-12 * abs(o.energy(eh, ph)[0])


def test_rk4_step(zk, case):
    e, p, o, eh, ph = case
    we, wp = o.step_rk4(eh, ph, DT)
    s = _sim(zk, e, p, zk.ZK_RK4)
    s.step(DT, 1)
    ge, gp = s.get_state()
    s.close()
    assert rel(ge, o.physical(we)) < 1e-11 and rel(gp, o.physical(wp)) < 1e-11


def test_ifab2_two_steps(zk, case):
    e, p, o, eh, ph = case
    we, wp, hist = o.step_ifab2(eh, ph, DT)
    we, wp, hist = o.step_ifab2(we, wp, DT, hist)
    s = _sim(zk, e, p, zk.ZK_IFAB2)
    s.step(DT, 2)
    ge, gp = s.get_state()
    s.close()
    assert rel(ge, o.physical(we)) < 1e-11 and rel(gp, o.physical(wp)) < 1e-11


def test_ifrk4_step(zk, case):
    e, p, o, eh, ph = case
    we, wp = o.step_ifrk4(eh, ph, DT)
    s = _sim(zk, e, p, zk.ZK_IFRK4)
    s.step(DT, 1)
    ge, gp = s.get_state()
    s.close()
    assert rel(ge, o.physical(we)) < 1e-11 and rel(gp, o.physical(wp)) < 1e-11


def test_dno_inverse(zk, case):
    e, p, o, eh, ph = case
    vh = o.dno(eh, ph)
    want = o.physical(o.dno_inverse(eh, vh, iters=8, ph0=ph))
    s = _sim(zk, e, p, zk.ZK_RK4)
    s.dno_inverse(o.physical(vh), iters=8)
    _, gp = s.get_state()
    s.close()
    assert rel(gp, want) < 1e-11


def test_ifab2_fp32_at_2048(zk):
    # the sea workload's grid (3072-point rows and columns: surface planes, half-length forward
    # transform, split final pass) in FP32, two IF-AB2 steps against the oracle from the same
    # FP32-rounded state. Bar: 4 n 2^-24 for the n steps (the stepped FP32 bar of the parity
    # tests) plus the state conversions on the unpadded grid, a forward transform at set_state
    # and an inverse one at get_state, each O(log2(nx nz)) roundings: (4 n + 2 log2(nx nz)) 2^-24
    n, L, h = 2048, 1600.0, 50.0
    e, p, _ = seas.jonswap_sea(n, n, L, L, h, 4.0, 12.0, 3)
    e, p = e.astype(np.float32), p.astype(np.float32)
    o = Oracle(Grid(n, n, L, L, h), 5, eps=0.5)
    eh, ph = o.spectrum(e.astype(np.float64)), o.spectrum(p.astype(np.float64))
    we, wp, hist = o.step_ifab2(eh, ph, DT)
    we, wp, _ = o.step_ifab2(we, wp, DT, hist)
    s = zk.Zakharov(n, n, L, L, h, M=5, eps=0.5)
    zk.zk_set_options(s.ctx, eps=0.5, integrator=zk.ZK_IFAB2)
    s.set_state(e, p)
    s.step(DT, 2)
    ge, gp = s.get_state()
    s.close()
    bar = (4 * 2 + 2 * np.log2(n * n)) * 2.0 ** -24
    assert rel(ge, o.physical(we)) < bar and rel(gp, o.physical(wp)) < bar, (rel(ge, o.physical(we)), rel(gp, o.physical(wp)))
