"""Pins for the oracle's absolute scales: the taper of Sec. 6.1, the Hamiltonian of Eq. 1
and the state filter of Eq. 17.

Each value is measured through the oracle's own pipeline (a forward transform of a
nonlinear product, an energy evaluation, a time step) on a single Fourier mode, and
compared with a number worked out by hand from the paper's definitions:

* taper exp[-(|k|/kc)^8], kc = 2/3 kNyq (Sec. 6.1, reading kNyq = pi / max(dx, dz)):
  at |k| = kc the factor is e^-1, at kc/2 it is exp(-2^-8), at 15/16 kc it is
  exp(-(15/16)^8). An exponent of 4, a cut-off factor other than 2/3, or kNyq from
  the finer axis each move one of these values by far more than the tolerance.
* Hamiltonian: a linear standing mode eta = a cos(k.x), psi = (g a / w) sin(k.x)
  with w^2 = g |k| tanh(|k| h) has, by Eq. 1 with G = G0 (Eq. 6), kinetic and
  potential energy g a^2 Lx Lz / 4 each, so H = g a^2 Lx Lz / 2 exactly. A missing
  1/2, or a wrong Parseval weight dx dz / (nx nz), fails it.
* filter (Eq. 17): per axis (5 + 4 cos(pi r) - cos(2 pi r)) / 8 with
  r = |k_a| / kNyq_a; by hand that is 15/16 at r = 1/3, 3/4 at r = 1/2, 7/16 at
  r = 2/3, and the 2D factor is the product over the axes (9/16 at r = (1/2, 1/2)).
  Measured as the ratio of one RK4 step with and without the filter.
"""
import math

import numpy as np
import pytest

from oracle import Grid, Oracle


def _taper_factor(gr, o, mx, mz):
    """Taper applied by the oracle's nonlinear forward transform to the mode (mx, mz)."""
    xp = np.arange(gr.npx) * gr.Lx / gr.npx
    zp = np.arange(gr.npz) * gr.Lz / gr.npz
    Z, X = np.meshgrid(zp, xp, indexing="ij")
    p = np.cos(2 * math.pi * mx / gr.Lx * X + 2 * math.pi * mz / gr.Lz * Z)
    F = o.nl_transform(p)
    # cos -> half the grid size at the mode after truncation to the (nz, nx) grid
    return F[mz % gr.nz, mx % gr.nx].real / (gr.nx * gr.nz / 2)


def test_taper_square_grid_closed_values():
    # dx = dz = 1: kNyq = pi, kc = 2 pi / 3, so mode number m has |k| / kc = m / 16
    gr = Grid(48, 48, 48.0, 48.0, 10.0)
    o = Oracle(gr, 3, taper=True)
    assert abs(_taper_factor(gr, o, 16, 0) - math.exp(-1.0)) < 1e-13
    assert abs(_taper_factor(gr, o, 0, 16) - math.exp(-1.0)) < 1e-13
    assert abs(_taper_factor(gr, o, 8, 0) - math.exp(-2.0 ** -8)) < 1e-13
    # oblique mode (9, 12): |m| = 15
    assert abs(_taper_factor(gr, o, 9, 12) - math.exp(-(15.0 / 16.0) ** 8)) < 1e-13
    assert abs(_taper_factor(gr, o, -12, 9) - math.exp(-(15.0 / 16.0) ** 8)) < 1e-13
    # the taper never touches the mean
    assert abs(_taper_factor(gr, o, 0, 0) * 0.5 - 1.0) < 1e-13
    # with the taper off the transform is exact
    o2 = Oracle(gr, 3, taper=False)
    assert abs(_taper_factor(gr, o2, 16, 0) - 1.0) < 1e-13


def test_taper_non_square_grid_uses_coarser_spacing():
    # dx = 1, dz = 2: kNyq = pi / 2 (the coarser axis), kc = pi / 3.
    # |k| = kc at mx = 8 (Lx = 48) and at mz = 16 (Lz = 96).
    gr = Grid(48, 48, 48.0, 96.0, 10.0)
    o = Oracle(gr, 2, taper=True)
    assert abs(gr.knyq - math.pi / 2) < 1e-15
    assert abs(_taper_factor(gr, o, 8, 0) - math.exp(-1.0)) < 1e-13
    assert abs(_taper_factor(gr, o, 0, 16) - math.exp(-1.0)) < 1e-13
    assert abs(_taper_factor(gr, o, 4, 0) - math.exp(-2.0 ** -8)) < 1e-13


@pytest.mark.parametrize("nx,nz,Lx,Lz,mx,mz", [(32, 32, 100.0, 100.0, 3, 0), (32, 16, 120.0, 50.0, 2, 3),
                                              (24, 40, 30.0, 90.0, -5, 7)])
def test_hamiltonian_linear_mode_closed_form(nx, nz, Lx, Lz, mx, mz):
    h, g, a = 8.0, 9.81, 0.05
    gr = Grid(nx, nz, Lx, Lz, h, g)
    kx, kz = 2 * math.pi * mx / Lx, 2 * math.pi * mz / Lz
    k = math.hypot(kx, kz)
    w = math.sqrt(g * k * math.tanh(k * h))
    x = np.arange(nx) * Lx / nx
    z = np.arange(nz) * Lz / nz
    Z, X = np.meshgrid(z, x, indexing="ij")
    th = kx * X + kz * Z
    eta = a * np.cos(th)
    psi = (g * a / w) * np.sin(th)
    want = g * a * a * Lx * Lz / 2
    for M, eps in ((1, 1.0), (4, 0.0)):
        o = Oracle(gr, M, eps=eps)
        H, kin, pot, mean = o.energy(o.spectrum(eta), o.spectrum(psi))
        assert abs(H - want) <= 1e-12 * want, (H, want)
        assert abs(kin - want / 2) <= 1e-12 * want
        assert abs(pot - want / 2) <= 1e-12 * want
        assert abs(mean) < 1e-15


def test_hamiltonian_constant_elevation_potential():
    # eta = c, psi = 0: H = 1/2 g c^2 Lx Lz (Eq. 1, no kinetic energy)
    gr = Grid(16, 8, 30.0, 12.0, 5.0)
    o = Oracle(gr, 3)
    c = 0.2
    eta = np.full((8, 16), c)
    H, kin, pot, mean = o.energy(o.spectrum(eta), o.spectrum(np.zeros_like(eta)))
    assert abs(H - 0.5 * 9.81 * c * c * 30.0 * 12.0) < 1e-12 * H
    assert kin == 0.0
    assert abs(mean - c) < 1e-15


@pytest.mark.parametrize("mx,mz,want", [(0, 0, 1.0), (8, 0, 15 / 16), (12, 0, 3 / 4), (16, 0, 7 / 16),
                                        (0, 8, 15 / 16), (12, 8, 3 / 4 * 15 / 16), (12, -12, 9 / 16)])
def test_filter_through_a_step(mx, mz, want):
    # non-square spacing: Eq. 17 scales each axis by its own Nyquist wavenumber
    gr = Grid(48, 48, 60.0, 30.0, 10.0)
    x = np.arange(48) * 60.0 / 48
    z = np.arange(48) * 30.0 / 48
    Z, X = np.meshgrid(z, x, indexing="ij")
    eta = 1e-3 * np.cos(2 * math.pi * mx / 60.0 * X + 2 * math.pi * mz / 30.0 * Z)
    psi = np.zeros_like(eta)
    on, off = Oracle(gr, 1, eps=0.0, filt=True), Oracle(gr, 1, eps=0.0, filt=False)
    eh, ph = on.spectrum(eta), on.spectrum(psi)
    e1, p1 = on.step_rk4(eh, ph, 0.05)
    e0, p0 = off.step_rk4(eh, ph, 0.05)
    i = (mz % 48, mx % 48)
    assert abs(e1[i] / e0[i] - want) < 1e-14
    if mx or mz:
        assert abs(p1[i] / p0[i] - want) < 1e-14
