"""The paper's Stokes-wave accuracy study (Sec. 8) as a pin on the oracle.

Setup as the paper states it: periodic 1D domain of length 2 pi (here nz = 1),
one wavelength, the analytic second-order Stokes profile with the third-order
frequency correction as reference, error |eta - eta_St| / a averaged over space
and time, ten linear periods, HOS truncation orders 2 and 3 (M = 2, 3). The
claims checked: the error falls monotonically as eps goes 0 -> 0.5 -> 1; at
(ka, kh) = (0.08, 1.0) orders 2 and 3 are nearly indistinguishable; at
(0.20, 2.0) order 3 is clearly better. The initial psi is the textbook
second-order Stokes potential on the surface, whose coefficients are first
checked here against the exact free-surface conditions (residual O(a^3)).
"""
import math

import numpy as np
import pytest

from oracle import Grid, Oracle, run
from paper_2608_25203_b300 import seas

G = 9.81


def _residuals(ka, h=1.0, k=1.0):
    """Max residuals of the exact kinematic and dynamic surface conditions for (eta_St, phi_St)."""
    a = ka / k
    x = np.linspace(0, 2 * math.pi, 64, endpoint=False)
    t, dx, dt, dy = 0.3, 1e-5, 1e-5, 1e-5
    eta = lambda xx, tt: seas.stokes_eta(xx, tt, k, a, h)  # noqa: E731
    phi = lambda xx, yy, tt: seas.stokes_potential(xx, yy, tt, k, a, h)  # noqa: E731
    e = eta(x, t)
    e_t = (eta(x, t + dt) - eta(x, t - dt)) / (2 * dt)
    e_x = (eta(x + dx, t) - eta(x - dx, t)) / (2 * dx)
    p_x = (phi(x + dx, e, t) - phi(x - dx, e, t)) / (2 * dx)
    p_y = (phi(x, e + dy, t) - phi(x, e - dy, t)) / (2 * dy)
    p_t = (phi(x, e, t + dt) - phi(x, e, t - dt)) / (2 * dt)
    kin = e_t + p_x * e_x - p_y
    dyn = p_t + 0.5 * (p_x ** 2 + p_y ** 2) + G * e
    dyn = dyn - dyn.mean()  # Bernoulli constant
    return np.max(np.abs(kin)), np.max(np.abs(dyn))


def test_stokes_potential_is_second_order_accurate():
    k1, d1 = _residuals(0.04)
    k2, d2 = _residuals(0.02)
    # third-order residuals: halving the amplitude divides them by ~8 (a wrong
    # second-order coefficient would leave an O(a^2) residual, ratio ~4)
    assert 6.5 < k1 / k2 < 9.5, (k1, k2)
    assert 6.5 < d1 / d2 < 9.5, (d1, d2)


def _stokes_error(ka, kh, eps, M, nx=32, ppp=100, periods=10):
    L, h = 2 * math.pi, kh
    gr = Grid(nx, 1, L, 1.0, h)
    eta, psi, (k, a, _) = seas.stokes2(nx, 1, L, 1.0, h, ka)
    T = 2 * math.pi / math.sqrt(G * k * math.tanh(k * h))
    dt = T / ppp
    o = Oracle(gr, M, eps=eps)
    x = np.arange(nx) * L / nx
    errs = []

    def cb(n, eh, ph):
        e = o.physical(eh)[0]
        errs.append(np.mean(np.abs(e - seas.stokes_eta(x, n * dt, k, a, h))) / a)

    run(o, eta, psi, dt, ppp * periods, integrator="ifab2", callback=cb)
    return float(np.mean(errs))


def test_stokes_error_sweep_matches_paper_claims():
    err = {}
    for (ka, kh) in ((0.08, 1.0), (0.20, 2.0)):
        for M in (2, 3):
            for eps in (0.0, 0.5, 1.0):
                err[(ka, M, eps)] = _stokes_error(ka, kh, eps, M)
    for ka in (0.08, 0.20):
        for M in (2, 3):
            e0, e5, e1 = err[(ka, M, 0.0)], err[(ka, M, 0.5)], err[(ka, M, 1.0)]
            assert e0 > e5 > e1, (ka, M, e0, e5, e1)
            # eps = 0.5 lies between the two, closer to the linear result (Sec. 8)
            assert abs(e5 - e0) < abs(e5 - e1)
    # mild case: orders 2 and 3 nearly indistinguishable
    assert abs(err[(0.08, 2, 1.0)] - err[(0.08, 3, 1.0)]) < 0.1 * err[(0.08, 2, 1.0)]
    # steep case: order 3 noticeably better than order 2
    assert err[(0.20, 3, 1.0)] < 0.6 * err[(0.20, 2, 1.0)]
    # eps = 0 (linear) is independent of the order
    assert err[(0.20, 2, 0.0)] == pytest.approx(err[(0.20, 3, 0.0)], rel=1e-12)


def test_stokes_phase_fidelity_hos3():
    # one of the long-time regimes (ka, kh) = (0.13, 2.0), 10 periods: HOS-3 stays phase-locked
    lin = _stokes_error(0.13, 2.0, 0.0, 3)
    nl = _stokes_error(0.13, 2.0, 1.0, 3)
    assert nl < 0.25 * lin, (nl, lin)
