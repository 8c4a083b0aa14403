"""The paper's integrating-factor AB2 integrator (Sec. 3.4, Eqs. 13-16) on the GPU vs the oracle."""
import numpy as np
import pytest

from oracle import Grid, Oracle
from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _oracle_run(o, eta, psi, plan):
    """plan: list of (dt, nsteps); history follows the paper's bootstrap rule."""
    eh, ph = o.spectrum(eta), o.spectrum(psi)
    hist = None
    for dt, n in plan:
        for _ in range(n):
            eh, ph, hist = o.step_ifab2(eh, ph, dt, hist)
    return o.physical(eh), o.physical(ph)


def _gpu(zk, case, prec, **kw):
    nx, nz, Lx, Lz, h, M = case
    s = zk.Zakharov(nx, nz, Lx, Lz, h, M=M, precision=prec, **kw)
    zk.zk_set_options(s.ctx, eps=kw.get("eps", 1.0), integrator=zk.ZK_IFAB2,
                      taper=int(kw.get("taper", True)), filter=int(kw.get("filter", True)))
    return s


CASE = (64, 32, 100.0, 50.0, 20.0, 4)


def test_ifab2_fp64_matches_oracle(zk):
    nx, nz, Lx, Lz, h, M = CASE
    eta, psi, _ = seas.jonswap_sea(nx, nz, Lx, Lz, h, Hs=1.5, Tp=7.0, seed=21)
    o = Oracle(Grid(nx, nz, Lx, Lz, h), M)
    e, p = _oracle_run(o, eta, psi, [(0.05, 20)])
    s = _gpu(zk, CASE, 1)
    s.set_state(eta, psi)
    s.step(0.05, 20)
    ge, gp = s.get_state()
    assert rel_l2(ge, e) < 1e-11 and rel_l2(gp, p) < 1e-11
    assert zk.zk_launches_per_step(s.ctx) == 2 * M + 1


def test_ifab2_fp32_matches_oracle(zk):
    case = (256, 256, 400.0, 400.0, 30.0, 5)
    nx, nz, Lx, Lz, h, M = case
    eta, psi, _ = seas.jonswap_sea(nx, nz, Lx, Lz, h, Hs=3.0, Tp=10.0, seed=2)
    o = Oracle(Grid(nx, nz, Lx, Lz, h), M)
    n = 50
    e, p = _oracle_run(o, eta, psi, [(0.02, n)])
    s = _gpu(zk, case, 0)
    s.set_state(eta.astype(np.float32), psi.astype(np.float32))
    s.step(0.02, n)
    ge, gp = s.get_state()
    tol = 4 * n * 2.0 ** -24
    assert rel_l2(ge, e) < tol and rel_l2(gp, p) < tol


def test_ifab2_linear_is_exact_rotation(zk):
    nx, nz, Lx, Lz, h, M = CASE
    eta, psi, _ = seas.jonswap_sea(nx, nz, Lx, Lz, h, Hs=1.0, Tp=8.0, seed=22)
    gr = Grid(nx, nz, Lx, Lz, h)
    dt, n = 0.3, 25
    s = _gpu(zk, CASE, 1, eps=0.0)
    s.set_state(eta, psi)
    s.step(dt, n)
    ge, gp = s.get_state()
    o = Oracle(gr, M)
    eh, ph = o.spectrum(eta), o.spectrum(psi)
    w = np.sqrt(gr.g * gr.G0)
    T = n * dt
    A = gr.filt ** n
    with np.errstate(invalid="ignore", divide="ignore"):
        we = np.cos(w * T) * eh + np.where(w > 0, gr.G0 / w * np.sin(w * T), 0) * ph
        wp = -np.where(w > 0, gr.g / w * np.sin(w * T), gr.g * T) * eh + np.cos(w * T) * ph
    assert rel_l2(ge, o.physical(A * we)) < 1e-12 and rel_l2(gp, o.physical(A * wp)) < 1e-12


def test_ifab2_dt_change_and_reset_bootstrap(zk):
    nx, nz, Lx, Lz, h, M = CASE
    eta, psi, _ = seas.jonswap_sea(nx, nz, Lx, Lz, h, Hs=1.5, Tp=7.0, seed=23)
    o = Oracle(Grid(nx, nz, Lx, Lz, h), M)
    e, p = _oracle_run(o, eta, psi, [(0.05, 6), (0.03, 7)])
    s = _gpu(zk, CASE, 1)
    s.set_state(eta, psi)
    s.step(0.05, 6)
    s.step(0.03, 7)
    ge, gp = s.get_state()
    assert rel_l2(ge, e) < 1e-11 and rel_l2(gp, p) < 1e-11
    # set_state drops the history: the next step is IF-Euler again
    s.step(0.05, 3)
    s.set_state(eta, psi)
    s.step(0.05, 4)
    e2, p2 = _oracle_run(o, eta, psi, [(0.05, 4)])
    ge2, gp2 = s.get_state()
    assert rel_l2(ge2, e2) < 1e-11 and rel_l2(gp2, p2) < 1e-11
