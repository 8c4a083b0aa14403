"""Pins for the oracle's time integration and invariants (Sec. 3.4, Eqs. 13-17; Eq. 1).

  * eps = 0 reduces the system to the linear operator L of Eq. 13; classical
    RK4 must then equal the per-mode matrix polynomial P(dt L)^n exactly, and
    the IF step must equal the rotation of Eq. 14 (closed forms, any size);
  * the eigenfrequency of L is the dispersion relation omega^2 = g |k| tanh(|k| h);
  * the filter of Eq. 17 is 1 at k = 0 and 0 at the Nyquist mode;
  * the mean of eta is conserved exactly; the Hamiltonian drifts only by the
    filter's dissipation and the integrator's error;
  * RK4 is fourth order on the nonlinear system.
"""
import math

import numpy as np
import pytest

from oracle import Grid, Oracle, run
from paper_2608_25203_b300 import seas


def _lin_matrix_power(gr, dt, n, poly):
    G0, g = gr.G0, gr.g
    Z = np.zeros(G0.shape + (2, 2))
    Z[..., 0, 1] = dt * G0
    Z[..., 1, 0] = -dt * g
    I = np.broadcast_to(np.eye(2), Z.shape)
    P = np.zeros_like(Z)
    term = I.copy()
    for j, c in enumerate(poly):
        if j > 0:
            term = term @ Z
        P = P + c * term
    return np.linalg.matrix_power(P, n)


def test_rk4_linear_closed_form():
    gr = Grid(32, 16, 100.0, 60.0, 20.0)
    o = Oracle(gr, 3, eps=0.0, filt=False)
    eta, psi, _ = seas.jonswap_sea(32, 16, 100.0, 60.0, 20.0, Hs=1.0, Tp=8.0, seed=1)
    eh, ph = o.spectrum(eta), o.spectrum(psi)
    dt, n = 0.05, 40
    e, p = eh.copy(), ph.copy()
    for _ in range(n):
        e, p = o.step_rk4(e, p, dt)
    P = _lin_matrix_power(gr, dt, n, [1, 1, 1 / 2, 1 / 6, 1 / 24])
    we = P[..., 0, 0] * eh + P[..., 0, 1] * ph
    wp = P[..., 1, 0] * eh + P[..., 1, 1] * ph
    assert np.max(np.abs(e - we)) <= 1e-11 * np.max(np.abs(eh))
    assert np.max(np.abs(p - wp)) <= 1e-11 * np.max(np.abs(ph))


def test_ifab2_linear_is_exact_rotation_with_filter():
    gr = Grid(32, 16, 100.0, 60.0, 20.0)
    o = Oracle(gr, 3, eps=0.0, filt=True)
    eta, psi, _ = seas.jonswap_sea(32, 16, 100.0, 60.0, 20.0, Hs=1.0, Tp=8.0, seed=2)
    eh, ph = o.spectrum(eta), o.spectrum(psi)
    dt, n = 0.3, 25
    e, p, hist = eh.copy(), ph.copy(), None
    for _ in range(n):
        e, p, hist = o.step_ifab2(e, p, dt, hist)
    w = np.sqrt(gr.g * gr.G0)
    T = n * dt
    A = gr.filt ** n
    with np.errstate(invalid="ignore", divide="ignore"):
        we = np.cos(w * T) * eh + np.where(w > 0, gr.G0 / w * np.sin(w * T), 0) * ph
        wp = -np.where(w > 0, gr.g / w * np.sin(w * T), gr.g * T) * eh + np.cos(w * T) * ph
    assert np.max(np.abs(e - A * we)) <= 1e-11 * np.max(np.abs(eh))
    assert np.max(np.abs(p - A * wp)) <= 1e-11 * np.max(np.abs(ph))


def test_dispersion_relation_single_mode():
    # one mode on a 64 x 64, L = 400 m, h = 30 m grid; eps = 0 and IF-AB2: phase exact
    gr = Grid(64, 64, 400.0, 400.0, 30.0)
    eta, psi, w = seas.single_mode(64, 64, 400.0, 400.0, 30.0, a=1e-3, mx=3, mz=2)
    k = math.hypot(2 * math.pi * 3 / 400, 2 * math.pi * 2 / 400)
    assert abs(w * w - 9.81 * k * math.tanh(k * 30.0)) < 1e-15
    o = Oracle(gr, 3, eps=0.0, filt=False)
    dt, n = 0.1, 200
    e, p = run(o, eta, psi, dt, n, integrator="ifab2")
    x = np.arange(64) * 400 / 64
    Z, X = np.meshgrid(x, x, indexing="ij")
    want = 1e-3 * np.cos(2 * math.pi * 3 / 400 * X + 2 * math.pi * 2 / 400 * Z - w * n * dt)
    assert np.max(np.abs(e - want)) < 1e-14
    # RK4: phase error of order (w dt)^4 w T
    e4, _ = run(o, eta, psi, dt, n, integrator="rk4")
    err = np.max(np.abs(e4 - want)) / 1e-3
    assert err < 0.05 * (w * dt) ** 4 * w * n * dt + 1e-12


def test_filter_values():
    gr = Grid(16, 8, 10.0, 5.0, 3.0)
    assert gr.filt[0, 0] == 1.0
    # Nyquist index (m = -n/2) on either axis: factor 0
    assert abs(gr.filt[0, 8]) < 1e-15 and abs(gr.filt[4, 0]) < 1e-15
    r = 0.5
    want = (5 + 4 * math.cos(math.pi * r) - math.cos(2 * math.pi * r)) / 8
    assert abs(gr.filt[0, 4] - want) < 1e-15


def _config1(M=3, eps=1.0):
    gr = Grid(64, 64, 100.0, 100.0, 20.0)
    eta, psi, info = seas.jonswap_sea(64, 64, 100.0, 100.0, 20.0, Hs=1.0, Tp=8.0, seed=1)
    return gr, Oracle(gr, M, eps=eps), eta, psi, info


def test_mean_and_energy_conservation_config1():
    gr, o, eta, psi, info = _config1()
    assert info["steepness"] <= 0.1
    eh0, ph0 = o.spectrum(eta), o.spectrum(psi)
    drift = {}
    for filt in (False, True):
        for eps in (0.0, 1.0):
            o = Oracle(gr, 3, eps=eps, filt=filt)
            eh, ph = eh0.copy(), ph0.copy()
            H0, _, _, m0 = o.energy(eh, ph)
            for _ in range(100):
                eh, ph = o.step_rk4(eh, ph, 0.02)
            H1, _, _, m1 = o.energy(eh, ph)
            assert abs(m1 - m0) <= 1e-15 * (1 + abs(m0)) + 1e-16
            # degree >= 3 products are only partly de-aliased on the 3/2 grid, so the
            # discrete mean of d eta/dt is small but not zero before it is set to zero
            assert o.last_mean_residual < 1e-5 * np.max(np.abs(eh))
            drift[(filt, eps)] = (H1 - H0) / H0
    # no filter: the Hamiltonian is conserved up to RK4 and truncation error
    assert abs(drift[(False, 0.0)]) < 1e-9
    assert abs(drift[(False, 1.0)]) < 2e-5
    # with the Eq. 17 filter every step, the loss is the filter's (same with and without nonlinearity)
    assert drift[(True, 0.0)] < 0 and drift[(True, 1.0)] < 0
    assert abs(drift[(True, 1.0)] - drift[(True, 0.0)]) < 0.01 * abs(drift[(True, 0.0)])


def test_rk4_fourth_order_nonlinear():
    gr = Grid(32, 32, 100.0, 100.0, 20.0)
    eta, psi, _ = seas.jonswap_sea(32, 32, 100.0, 100.0, 20.0, Hs=3.0, Tp=8.0, seed=4)
    o = Oracle(gr, 3, filt=False)
    T = 2.0
    ref, _ = run(o, eta, psi, T / 64, 64)
    e1, _ = run(o, eta, psi, T / 8, 8)
    e2, _ = run(o, eta, psi, T / 16, 16)
    r = np.max(np.abs(e1 - ref)) / np.max(np.abs(e2 - ref))
    assert 12.0 < r < 20.0, r
