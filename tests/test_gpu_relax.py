"""Forcing strip on the GPU vs the oracle: inverse DNO (Eq. 19), relaxation and psi resync (Eqs. 33-35)."""
import numpy as np
import pytest

from oracle import Grid, Oracle, sigma_box
from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu

CASE = (64, 64, 100.0, 100.0, 20.0, 4)


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _inputs():
    nx, nz, Lx, Lz, h, M = CASE
    eta, psi, _ = seas.jonswap_sea(nx, nz, Lx, Lz, h, Hs=1.5, Tp=7.0, seed=41)
    gr = Grid(nx, nz, Lx, Lz, h)
    o = Oracle(gr, M)
    sigma = sigma_box(gr, 0.0, 30.0, 0.0, 100.0, wb=10.0, sigma_max=4.0)
    target = 0.25 * np.cos(2 * np.pi * 2 * np.arange(nx) * gr.dx / Lx)[None, :] * np.ones((nz, 1))
    return gr, o, eta, psi, sigma, target


@pytest.mark.parametrize("prec,tol", [(1, 1e-11), (0, 3e-5)])
def test_dno_inverse_matches_oracle(zk, prec, tol):
    gr, o, eta, psi, _, _ = _inputs()
    eh, ph = o.spectrum(eta), o.spectrum(psi)
    vh = o.dno(eh, ph)
    want = o.physical(o.dno_inverse(eh, vh, iters=8, ph0=ph))
    s = zk.Zakharov(*CASE[:5], M=CASE[5], precision=prec)
    dt = np.float64 if prec == 1 else np.float32
    s.set_state(eta.astype(dt), psi.astype(dt))
    s.dno_inverse(o.physical(vh).astype(dt), iters=8)
    _, gp = s.get_state()
    assert rel_l2(gp, want) < tol
    assert rel_l2(gp, o.physical(ph)) < max(tol, 1e-8)


@pytest.mark.parametrize("prec,tol", [(1, 1e-11), (0, 5e-5)])
def test_step_then_relax_matches_oracle(zk, prec, tol):
    gr, o, eta, psi, sigma, target = _inputs()
    dt, nsub = 0.05, 3
    eh, ph = o.spectrum(eta), o.spectrum(psi)
    hist = None
    for _ in range(nsub):
        eh, ph, hist = o.step_ifab2(eh, ph, dt, hist)
        eh, ph = o.relax(eh, ph, dt, sigma, target, iters=8)
    s = zk.Zakharov(*CASE[:5], M=CASE[5], precision=prec)
    zk.zk_set_options(s.ctx, integrator=zk.ZK_IFAB2)
    d = np.float64 if prec == 1 else np.float32
    s.set_state(eta.astype(d), psi.astype(d))
    for _ in range(nsub):
        s.step(dt, 1)
        s.relax(sigma.astype(d), target.astype(d), dt, iters=8)
    ge, gp = s.get_state()
    assert rel_l2(ge, o.physical(eh)) < tol and rel_l2(gp, o.physical(ph)) < tol


def test_relax_pins_eta_inside_the_box(zk):
    gr, o, eta, psi, sigma, target = _inputs()
    s = zk.Zakharov(*CASE[:5], M=CASE[5], precision=1)
    s.set_state(eta, psi)
    big = np.where(sigma > 0, 1e4, 0.0)
    s.relax(big, target, 1.0, iters=8)
    ge, _ = s.get_state()
    inside = sigma > 3.9
    # band-limiting of the relaxed field smooths the box edge; deep inside it is the target
    core = inside & (np.arange(gr.nx)[None, :] * gr.dx > 8) & (np.arange(gr.nx)[None, :] * gr.dx < 22)
    assert np.max(np.abs(ge[core] - target[core])) < 0.05
