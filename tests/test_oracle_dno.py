"""Pins for the oracle's Dirichlet-Neumann series (Sec. 3.2, Eqs. 6-9 and the HOS recursion).

Each test checks the oracle against something other than itself:
  * flat surface: G(0) psi = |k| tanh(|k| h) psi exactly (Eq. 6);
  * constant elevation c: a flat surface at height c, so the exact operator is
    |k| tanh(|k| (h + c)); the order-M series must equal its Taylor polynomial
    in c of degree M-1 (coefficients from sympy), and converge to it;
  * a manufactured exact solution: Phi = cos(k.x) cosh(|k|(y+h))/cosh(|k|h) is
    harmonic with a no-flux bed, so for any surface eta, psi = Phi(x, eta) and
    G(eta) psi = Phi_y - grad eta . grad_x Phi at y = eta (Eq. 3); the series
    error must fall geometrically with M;
  * Eqs. 7 and 8 written out term by term agree with the general recursion;
  * G(eta) is symmetric and non-negative (it is the Hessian of the kinetic
    energy of Eq. 1).
"""
import math

import numpy as np
import pytest
import sympy as sp

from oracle import Grid, Oracle


def _rand_band(gr, rng, kmax_frac=0.4, amp=1.0):
    """Random real field with modes |m| <= kmax_frac * n/2 (smooth), as a spectrum."""
    F = (rng.standard_normal(gr.K.shape) + 1j * rng.standard_normal(gr.K.shape))
    F *= (np.abs(gr.MX) <= kmax_frac * gr.nx / 2) & (np.abs(gr.MZ) <= kmax_frac * gr.nz / 2)
    f = np.fft.ifft2(F).real
    f *= amp / np.max(np.abs(f))
    return f


@pytest.mark.parametrize("M", [1, 2, 3, 5, 6])
def test_flat_surface_is_G0(M):
    gr = Grid(32, 24, 50.0, 40.0, 7.0)
    o = Oracle(gr, M)
    rng = np.random.default_rng(M)
    psi = _rand_band(gr, rng)
    ph = o.spectrum(psi)
    Gh = o.dno(np.zeros_like(ph), ph)
    want = np.abs(gr.K) * np.tanh(np.abs(gr.K) * 7.0) * ph
    want[0, 0] = 0
    assert np.max(np.abs(Gh - want)) <= 1e-14 * np.max(np.abs(want))


def _taylor_tanh_coeffs(k, h, order):
    """Coefficients of k tanh(k (h + c)) in powers of c, up to c^order, from sympy."""
    c = sp.symbols("c")
    ser = sp.series(sp.Integer(1) * k * sp.tanh(k * (h + c)), c, 0, order + 1).removeO()
    poly = sp.Poly(ser, c)
    return [float(poly.coeff_monomial(c ** j)) for j in range(order + 1)]


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5, 6, 8])
def test_constant_elevation_taylor_polynomial(M):
    # Lx = Lz = 2 pi so |k| is the mode number; h = 1.3; c = 0.03.
    gr = Grid(16, 16, 2 * math.pi, 2 * math.pi, 1.3)
    o = Oracle(gr, M, taper=False)
    c = 0.03
    modes = [(1, 0), (2, 1), (0, 3), (3, 2)]
    rng = np.random.default_rng(11)
    ph = np.zeros(gr.K.shape, complex)
    for (mx, mz) in modes:
        v = rng.standard_normal() + 1j * rng.standard_normal()
        ph[mz % 16, mx % 16] += v
        ph[-mz % 16, -mx % 16] += np.conj(v)
    eh = np.zeros_like(ph)
    eh[0, 0] = c * gr.nx * gr.nz
    Gh = o.dno(eh, ph)
    for (mx, mz) in modes:
        k = math.hypot(mx, mz)
        coef = _taylor_tanh_coeffs(sp.sqrt(mx * mx + mz * mz), sp.Rational(13, 10), M - 1)
        poly = sum(coef[j] * c ** j for j in range(M))
        got = Gh[mz % 16, mx % 16] / ph[mz % 16, mx % 16]
        assert abs(got - poly) <= 1e-12 * abs(poly), (M, mx, mz, got, poly)
        exact = k * math.tanh(k * (1.3 + c))
        # truncation error of the Taylor polynomial ~ (k c)^M, shrinking with M
        assert abs(got - exact) <= 5 * (k * c) ** M * k + 1e-12


def _manufactured(gr, eta_fn, kvec):
    """psi = Phi(x, eta) and exact G psi for the flat-strip harmonic Phi = cos(k.x) C(y)."""
    x = np.arange(gr.nx) * gr.dx
    z = np.arange(gr.nz) * gr.dz
    Z, X = np.meshgrid(z, x, indexing="ij")
    eta, etax, etaz = eta_fn(X, Z)
    kx, kz = kvec
    k = math.hypot(kx, kz)
    h = gr.h
    ch = math.cosh(k * h)
    Cy = np.cosh(k * (eta + h)) / ch
    Sy = k * np.sinh(k * (eta + h)) / ch
    ph = kx * X + kz * Z
    psi = np.cos(ph) * Cy
    Phix = -kx * np.sin(ph) * Cy
    Phiz = -kz * np.sin(ph) * Cy
    Phiy = np.cos(ph) * Sy
    G = Phiy - (etax * Phix + etaz * Phiz)
    return eta, psi, G


def _eta_fn(X, Z, A=0.06):
    e = A * np.cos(X) + 0.5 * A * np.sin(Z) + 0.4 * A * np.cos(X + Z)
    ex = -A * np.sin(X) - 0.4 * A * np.sin(X + Z)
    ez = 0.5 * A * np.cos(Z) - 0.4 * A * np.sin(X + Z)
    return e, ex, ez


def test_manufactured_exact_harmonic_converges_in_M():
    gr = Grid(48, 48, 2 * math.pi, 2 * math.pi, 0.9)
    eta, psi, G = _manufactured(gr, _eta_fn, (2.0, 1.0))
    errs = []
    for M in range(1, 8):
        o = Oracle(gr, M, taper=False)
        Gh = o.dno(o.spectrum(eta), o.spectrum(psi))
        errs.append(np.max(np.abs(o.physical(Gh) - G)) / np.max(np.abs(G)))
    # geometric decrease in M (series convergence), down to the grid's truncation level
    for a, b in zip(errs[:5], errs[1:6]):
        assert b < 0.35 * a, errs
    assert errs[6] < 1e-7, errs


def test_manufactured_taper_is_harmless_for_smooth_fields():
    gr = Grid(48, 48, 2 * math.pi, 2 * math.pi, 0.9)
    eta, psi, G = _manufactured(gr, _eta_fn, (2.0, 1.0))
    o = Oracle(gr, 6, taper=True)
    Gh = o.dno(o.spectrum(eta), o.spectrum(psi))
    assert np.max(np.abs(o.physical(Gh) - G)) / np.max(np.abs(G)) < 1e-5


def test_recursion_G1_equals_eq7():
    gr = Grid(24, 32, 30.0, 40.0, 4.0)
    rng = np.random.default_rng(5)
    eta = _rand_band(gr, rng, amp=0.3)
    psi = _rand_band(gr, rng, amp=2.0)
    o = Oracle(gr, 2, taper=False)
    eh, ph = o.spectrum(eta), o.spectrum(psi)
    G1 = o.dno_terms(eh, ph)["G"][1]
    lit = o.g1_literal(eh, ph)
    # the divergence form and the product-rule form agree once truncated (3/2 rule is exact for quadratics)
    a, b = o.from_padded(G1), o.from_padded(lit)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


@pytest.mark.parametrize("taper", [False, True])
def test_recursion_G2_equals_eq8(taper):
    gr = Grid(24, 32, 30.0, 40.0, 4.0)
    rng = np.random.default_rng(6)
    eta = _rand_band(gr, rng, amp=0.3)
    psi = _rand_band(gr, rng, amp=2.0)
    o = Oracle(gr, 3, taper=taper)
    eh, ph = o.spectrum(eta), o.spectrum(psi)
    G2 = o.dno_terms(eh, ph)["G"][2]
    lit = o.g2_literal(eh, ph)
    assert np.max(np.abs(G2 - lit)) <= 1e-12 * np.max(np.abs(lit))


def test_planted_sign_error_is_caught():
    """A plausible slip (sign of the grad-eta.grad-psi term in G1) must break the Eq. 7 pin."""
    gr = Grid(24, 32, 30.0, 40.0, 4.0)
    rng = np.random.default_rng(5)
    eta = _rand_band(gr, rng, amp=0.3)
    psi = _rand_band(gr, rng, amp=2.0)
    o = Oracle(gr, 2, taper=False)
    eh, ph = o.spectrum(eta), o.spectrum(psi)
    t = o.dno_terms(eh, ph)
    wrong = t["W"][1] + t["d"]
    b = o.from_padded(o.g1_literal(eh, ph))
    assert np.max(np.abs(o.from_padded(wrong) - b)) > 1e-3 * np.max(np.abs(b))


def test_symmetric_and_nonnegative():
    gr = Grid(32, 32, 2 * math.pi, 2 * math.pi, 1.0)
    rng = np.random.default_rng(9)
    eta = _rand_band(gr, rng, kmax_frac=0.2, amp=0.05)
    phi = _rand_band(gr, rng, kmax_frac=0.3)
    psi = _rand_band(gr, rng, kmax_frac=0.3)
    o = Oracle(gr, 4, taper=False)
    eh = o.spectrum(eta)
    Gpsi = o.physical(o.dno(eh, o.spectrum(psi)))
    Gphi = o.physical(o.dno(eh, o.spectrum(phi)))
    a, b = np.sum(phi * Gpsi), np.sum(psi * Gphi)
    assert abs(a - b) <= 1e-12 * np.sqrt(np.sum(phi * Gphi) * np.sum(psi * Gpsi))
    assert np.sum(psi * Gpsi) > 0 and np.sum(phi * Gphi) > 0
