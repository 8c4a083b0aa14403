"""Pins for the oracle's state recovery (Sec. 3.5, Eq. 19) and relaxation source (Sec. 5, Eqs. 33-35).

  * the inverse DNO map inverts the forward map: G^{-1}(G psi) = psi (mean
    kept) to the fixed point's accuracy, and the error contracts
    geometrically with the iteration count (the iteration is a contraction
    when the nonlinear part is subdominant, as Sec. 3.5 states);
  * at eta = 0 the map is exactly G0^{-1} (one step);
  * Eq. 34 is the closed-form solution of d eta/dt = -sigma (eta - eta_t):
    sigma = 0 leaves eta unchanged, large sigma dt pins eta to the target,
    and the decay matches exp(-sigma dt) pointwise;
  * Eq. 33: sigma is zero outside the box, sigma_max in the interior beyond
    the band, monotone across the band;
  * after relaxation the pair stays consistent: G(eta_relaxed) psi_relaxed = v.
"""
import math

import numpy as np
import pytest

from oracle import Grid, Oracle, sigma_box
from paper_2608_25203_b300 import seas


def _setup(M=4, Hs=1.5):
    gr = Grid(64, 64, 100.0, 100.0, 20.0)
    eta, psi, _ = seas.jonswap_sea(64, 64, 100.0, 100.0, 20.0, Hs=Hs, Tp=8.0, seed=31)
    o = Oracle(gr, M)
    return gr, o, o.spectrum(eta), o.spectrum(psi)


def test_inverse_dno_roundtrip_and_contraction():
    gr, o, eh, ph = _setup()
    vh = o.dno(eh, ph)
    errs = []
    for it in (0, 1, 2, 4, 8):
        p2 = o.dno_inverse(eh, vh, iters=it, ph0=ph)
        errs.append(np.linalg.norm(p2 - ph) / np.linalg.norm(ph))
    assert errs[-1] < 1e-9, errs
    for a, b in zip(errs[:-1], errs[1:]):
        assert b < a, errs


def test_inverse_dno_flat_surface_is_G0_inverse():
    gr, o, eh, ph = _setup()
    vh = gr.G0 * ph
    p2 = o.dno_inverse(np.zeros_like(eh), vh, iters=3, ph0=ph)
    assert np.max(np.abs(p2 - ph)) <= 1e-12 * np.max(np.abs(ph))


def test_relaxation_closed_form_and_limits():
    gr, o, eh, ph = _setup()
    rng = np.random.default_rng(3)
    target = 0.3 * rng.standard_normal((gr.nz, gr.nx))
    target = o.physical(o.spectrum(target))
    sigma = sigma_box(gr, 20.0, 70.0, 30.0, 80.0, wb=10.0, sigma_max=5.0)
    eta = o.physical(eh)
    # sigma = 0: eta unchanged; psi recovered from v at the same eta
    e0, p0 = o.relax(eh, ph, 0.1, np.zeros_like(sigma), target)
    assert np.max(np.abs(o.physical(e0) - eta)) < 1e-12
    assert np.linalg.norm(p0 - ph) / np.linalg.norm(ph) < 1e-9
    # decay factor exp(-sigma dt) pointwise (target band-limited, so no spectral loss)
    dt = 0.1
    e1, _ = o.relax(eh, ph, dt, sigma, target)
    want = target + (eta - target) * np.exp(-sigma * dt)
    want = o.physical(o.spectrum(want))
    assert np.max(np.abs(o.physical(e1) - want)) < 1e-12


def test_relaxation_pair_consistency():
    gr, o, eh, ph = _setup()
    sigma = sigma_box(gr, 20.0, 70.0, 30.0, 80.0, wb=10.0, sigma_max=2.0)
    target = np.zeros((gr.nz, gr.nx))
    vh = o.dno(eh, ph)
    e1, p1 = o.relax(eh, ph, 0.05, sigma, target, iters=30)
    v1 = o.dno(e1, p1)
    assert np.linalg.norm(v1 - vh) / np.linalg.norm(vh) < 1e-8


def test_sigma_box_shape():
    gr = Grid(64, 64, 100.0, 100.0, 20.0)
    s = sigma_box(gr, 20.0, 70.0, 30.0, 80.0, wb=10.0, sigma_max=5.0)
    x = np.arange(64) * gr.dx
    assert s[0, 0] == 0.0 and np.all(s[:, x < 20.0] == 0.0)
    iz, ix = int(55 / gr.dz), int(45 / gr.dx)
    assert s[iz, ix] == 5.0
    row = s[iz, (x >= 20.0) & (x <= 40.0)]
    assert np.all(np.diff(row) >= 0)
