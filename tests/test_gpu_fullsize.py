"""Parity at the benchmark's full size (2048 x 2048, M = 5, FP32) in its launch configuration.

* one right-hand side and one RK4 step (the captured step graph zk_step
  replays) against the FP64 oracle on the same seeded sea (the oracle takes
  ~15 s per right-hand side here);
* properties that hold at any size: with eps = 0 the step is linear and each
  mode must follow the closed form (A(k) P(dt L))^n of RK4 with the filter
  (computed per mode in numpy, no oracle); the mean of eta is conserved
  exactly; repeated runs are bitwise identical.
"""
import numpy as np
import pytest

from oracle import Grid, Oracle
from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu

W = dict(nx=2048, nz=2048, Lx=1600.0, Lz=1600.0, h=50.0, M=5, eps=0.5, dt=0.02, Hs=4.0, Tp=12.0, seed=3)


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


@pytest.fixture(scope="module")
def sea():
    eta, psi, _ = seas.jonswap_sea(W["nx"], W["nz"], W["Lx"], W["Lz"], W["h"], W["Hs"], W["Tp"], W["seed"])
    return eta, psi


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _sim(zk, **kw):
    kw.setdefault("eps", W["eps"])
    return zk.Zakharov(W["nx"], W["nz"], W["Lx"], W["Lz"], W["h"], M=W["M"], **kw)


def test_fullsize_rhs_and_step_match_oracle(zk, sea):
    eta, psi = sea
    o = Oracle(Grid(W["nx"], W["nz"], W["Lx"], W["Lz"], W["h"]), W["M"], eps=W["eps"])
    eh, ph = o.spectrum(eta), o.spectrum(psi)
    de, dp = o.rhs(eh, ph)
    s = _sim(zk)
    s.set_state(eta.astype(np.float32), psi.astype(np.float32))
    ge, gp = s.rhs()
    assert rel_l2(ge, o.physical(de)) < 2e-5
    assert rel_l2(gp, o.physical(dp)) < 2e-5
    e1, p1 = o.step_rk4(eh, ph, W["dt"])
    s.step(W["dt"], 1)
    se, sp = s.get_state()
    assert rel_l2(se, o.physical(e1)) < 4 * 2.0 ** -24 * 10
    assert rel_l2(sp, o.physical(p1)) < 4 * 2.0 ** -24 * 10


def test_fullsize_linear_closed_form(zk, sea):
    eta, psi = sea
    gr = Grid(W["nx"], W["nz"], W["Lx"], W["Lz"], W["h"])
    n, dt = 20, W["dt"]
    s = _sim(zk, eps=0.0)
    s.set_state(eta.astype(np.float32), psi.astype(np.float32))
    s.step(dt, n)
    ge, gp = s.get_state()
    eh = np.fft.fft2(eta.astype(np.float32).astype(np.float64))
    ph = np.fft.fft2(psi.astype(np.float32).astype(np.float64))
    eh[~gr.keep] = 0
    ph[~gr.keep] = 0
    # per-mode RK4 polynomial of dt L, L = [[0, G0], [-g, 0]]
    a, b = dt * gr.G0, -dt * gr.g          # Z = [[0, a], [b, 0]], Z^2 = ab I
    ab = a * b
    p_even = 1 + ab / 2 + ab * ab / 24     # coefficient of I
    p_odd = 1 + ab / 6                      # coefficient of Z
    P11, P12, P21 = p_even, p_odd * a, p_odd * b
    e, p = eh.copy(), ph.copy()
    for _ in range(n):
        e, p = gr.filt * (P11 * e + P12 * p), gr.filt * (P21 * e + P11 * p)
    we, wp = np.fft.ifft2(e).real, np.fft.ifft2(p).real
    tol = 4 * n * 2.0 ** -24
    assert rel_l2(ge, we) < tol and rel_l2(gp, wp) < tol


def test_fullsize_mean_conserved_and_deterministic(zk, sea):
    eta, psi = sea
    outs = []
    for _ in range(2):
        s = _sim(zk)
        s.set_state(eta.astype(np.float32), psi.astype(np.float32))
        m0 = s.energy()[3]
        s.step(W["dt"], 10)
        m1 = s.energy()[3]
        assert abs(m1 - m0) < 1e-9
        outs.append(s.get_state(np.float32))
        s.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
