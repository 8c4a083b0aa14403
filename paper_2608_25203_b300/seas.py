"""Seeded synthetic sea states: the inputs both the CUDA path and the oracle consume.

This module only *generates* initial conditions (surface elevation eta and
surface potential psi as physical arrays, row-major [nz][nx], x fastest). It
holds none of the wave step's arithmetic: no Dirichlet-Neumann series, no
de-aliasing, no time stepping. Every array it returns is handed to both sides
as data.

Generators
----------
* ``jonswap_sea``  - random-phase JONSWAP sea with cos^2 directional spreading
  (the paper initialises from an ocean spectrum, Sec. 6 "Implementation
  Details"; the spectrum family here is JONSWAP, gamma = 3.3).
* ``single_mode``  - one linear Airy mode, eta = a cos(k.x), psi from linear
  theory (the dispersion check of Sec. 3.2, Eq. 6: omega^2 = g G0).
* ``stokes2``      - the second-order Stokes wave with the third-order
  frequency correction used as the analytic reference of Sec. 8 ("Stokes Wave
  Accuracy under Varying Nonlinearity"); psi is the textbook second-order
  Stokes potential evaluated on the surface.
* ``gaussian_bump`` - the tank's initial bump of Sec. 8 ("Wave Propagation").
* ``batch_tiles``  - the per-tile parameters (grid, depth, order, Hs, Tp, seed)
  of the mixed batch of independent sea tiles.

Random phases come from splitmix64 (S. Vigna's published 64-bit mixer) keyed
by (seed, linear mode index), so a mode's phase does not depend on the grid
traversal order or on numpy's RNG version.
"""
from __future__ import annotations

import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied elementwise to uint64 keys (wrapping arithmetic)."""
    z = np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, idx: np.ndarray) -> np.ndarray:
    """Uniform [0,1) doubles from splitmix64(splitmix64(seed) xor idx), top 53 bits."""
    with np.errstate(over="ignore"):
        s = splitmix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        z = splitmix64(np.asarray(idx, dtype=np.uint64) ^ s)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _mode_index(n: int) -> np.ndarray:
    """Signed integer mode numbers in FFT order: 0..n/2-1, -n/2..-1 (n=1 -> [0])."""
    j = np.arange(n)
    return np.where(j < (n + 1) // 2, j, j - n)


def _omega(k: np.ndarray, h: float, g: float) -> np.ndarray:
    """Linear finite-depth frequency sqrt(g k tanh(k h)) (input generation only)."""
    return np.sqrt(g * k * np.tanh(k * h))


def peak_wavenumber(Tp: float, h: float, g: float = 9.81) -> float:
    """Solve omega_p^2 = g k tanh(k h) for k by Newton from the deep-water guess."""
    wp = 2.0 * math.pi / Tp
    k = wp * wp / g
    for _ in range(100):
        f = g * k * math.tanh(k * h) - wp * wp
        df = g * math.tanh(k * h) + g * k * h / math.cosh(k * h) ** 2
        dk = f / df
        k -= dk
        if abs(dk) < 1e-15 * k:
            break
    return k


def jonswap_sea(nx: int, nz: int, Lx: float, Lz: float, h: float, Hs: float, Tp: float,
                seed: int, g: float = 9.81, gamma: float = 3.3):
    """Random-phase JONSWAP sea, cos^2 spreading about +x, psi from linear theory.

    Recipe (all deterministic given ``seed``):
      S(w)  = w^-5 exp(-5/4 (wp/w)^4) gamma^exp(-(w-wp)^2 / (2 s^2 wp^2)), s = 0.07 (w<=wp) / 0.09
      S(k)  = S(w(k)) dw/dk with the finite-depth dispersion relation,
      F(kx,kz) = S(k) D(theta) / k,  D = (2/pi) cos^2(theta) for |theta| < pi/2,
      amplitude a = sqrt(2 F dkx dkz), phase 2 pi u(seed, mode), modes with
      |k| <= min(10 kp, kNyq/2), kNyq = pi / max(dx, dz),
      psi_k = -i (g / w) eta_k on kx > 0 (linear theory), Hermitian mirror,
      then both fields scaled so that 4 * std(eta) = Hs on the grid.
    Returns (eta, psi, info) with float64 arrays [nz][nx].
    """
    dx, dz = Lx / nx, Lz / nz
    dkx, dkz = 2 * math.pi / Lx, 2 * math.pi / Lz
    kp = peak_wavenumber(Tp, h, g)
    wp = 2 * math.pi / Tp
    spac = [d for d, n in ((dx, nx), (dz, nz)) if n > 1]
    knyq = math.pi / max(spac)
    kcut = min(10.0 * kp, 0.5 * knyq)

    mx = _mode_index(nx)
    mz = _mode_index(nz)
    MZ, MX = np.meshgrid(mz, mx, indexing="ij")
    KX, KZ = MX * dkx, MZ * dkz
    K = np.hypot(KX, KZ)
    sel = (MX > 0) & (K <= kcut) & (K > 0)
    k = K[sel]
    w = _omega(k, h, g)
    sig = np.where(w <= wp, 0.07, 0.09)
    Sw = w ** -5 * np.exp(-1.25 * (wp / w) ** 4) * gamma ** np.exp(-((w - wp) ** 2) / (2 * sig ** 2 * wp ** 2))
    cg = 0.5 * g / w * (np.tanh(k * h) + k * h / np.cosh(k * h) ** 2)
    theta = np.arctan2(KZ[sel], KX[sel])
    D = np.where(np.abs(theta) < 0.5 * math.pi, (2.0 / math.pi) * np.cos(theta) ** 2, 0.0)
    F = Sw * cg * D / k
    amp = np.sqrt(2.0 * F * dkx * dkz)
    lin = (MZ[sel] % nz).astype(np.uint64) * np.uint64(nx) + (MX[sel] % nx).astype(np.uint64)
    phase = 2.0 * math.pi * uniform01(seed, lin)

    eh = np.zeros((nz, nx), dtype=np.complex128)
    ph = np.zeros((nz, nx), dtype=np.complex128)
    iz, ix = np.nonzero(sel)
    c = 0.5 * nx * nz * amp * np.exp(1j * phase)
    eh[iz, ix] = c
    ph[iz, ix] = -1j * (g / w) * c
    # Hermitian mirror (kx > 0 modes never coincide with their mirrors)
    eh[(-iz) % nz, (-ix) % nx] = np.conj(c)
    ph[(-iz) % nz, (-ix) % nx] = np.conj(-1j * (g / w) * c)
    eta = np.ascontiguousarray(np.fft.ifft2(eh).real)
    psi = np.ascontiguousarray(np.fft.ifft2(ph).real)
    std = float(np.sqrt(np.mean(eta ** 2)))
    scale = Hs / (4.0 * std) if std > 0 else 0.0
    eta *= scale
    psi *= scale
    info = dict(kp=kp, lambda_p=2 * math.pi / kp, steepness=kp * Hs / 2, kcut=kcut,
                nmodes=int(sel.sum()))
    return eta, psi, info


def single_mode(nx: int, nz: int, Lx: float, Lz: float, h: float, a: float, mx: int, mz: int = 0,
                g: float = 9.81):
    """eta = a cos(k.x), psi = (g a / w) sin(k.x): one linear mode travelling along +k."""
    x = np.arange(nx) * (Lx / nx)
    z = np.arange(nz) * (Lz / nz)
    Z, X = np.meshgrid(z, x, indexing="ij")
    kx, kz = 2 * math.pi * mx / Lx, 2 * math.pi * mz / Lz
    k = math.hypot(kx, kz)
    w = math.sqrt(g * k * math.tanh(k * h))
    ph = kx * X + kz * Z
    return a * np.cos(ph), (g * a / w) * np.sin(ph), w


def stokes_params(k: float, a: float, h: float, g: float = 9.81):
    """Second-order amplitude ratio and third-order-corrected frequency (Sec. 8, Stokes check).

    Returns (c2, omega, omega0) with eta_St = a cos(th) + c2 cos(2 th),
    c2 = k a^2 (3 - T^2) / (4 T^3), omega^2 = g k T (1 + delta),
    delta = (k a)^2 (9 - 10 T^2 + 9 T^4) / (8 T^4), T = tanh(k h).
    """
    T = math.tanh(k * h)
    c2 = k * a * a * (3.0 - T * T) / (4.0 * T ** 3)
    delta = (k * a) ** 2 * (9.0 - 10.0 * T * T + 9.0 * T ** 4) / (8.0 * T ** 4)
    omega = math.sqrt(g * k * T * (1.0 + delta))
    omega0 = math.sqrt(g * k * T)
    return c2, omega, omega0


def stokes_eta(x: np.ndarray, t: float, k: float, a: float, h: float, g: float = 9.81):
    """Analytic second-order Stokes elevation at time t, phase th = k x - omega t."""
    c2, omega, _ = stokes_params(k, a, h, g)
    th = k * x - omega * t
    return a * np.cos(th) + c2 * np.cos(2 * th)


def stokes_potential(x: np.ndarray, y: np.ndarray, t: float, k: float, a: float, h: float,
                     g: float = 9.81):
    """Textbook second-order Stokes velocity potential (y up, still level y=0, bed y=-h).

    phi = (a w0 / k) cosh(k(h+y)) / sinh(kh) sin(th)
        + (3/8) a^2 w0 cosh(2k(h+y)) / sinh(kh)^4 sin(2 th),   th = k x - w t,
    with w0 the linear frequency in the amplitudes (second-order theory) and the
    corrected frequency w in the phase.
    """
    _, omega, w0 = stokes_params(k, a, h, g)
    th = k * x - omega * t
    s = math.sinh(k * h)
    return (a * w0 / k) * np.cosh(k * (h + y)) / s * np.sin(th) + \
        0.375 * a * a * w0 * np.cosh(2 * k * (h + y)) / s ** 4 * np.sin(2 * th)


def stokes2(nx: int, nz: int, Lx: float, Lz: float, h: float, ka: float, nwaves: int = 1,
            g: float = 9.81):
    """Stokes wave along x with nwaves wavelengths in Lx: (eta, psi, (k, a, omega)).

    psi is the second-order potential evaluated on the second-order surface.
    The field is constant along z.
    """
    k = 2 * math.pi * nwaves / Lx
    a = ka / k
    x = np.arange(nx) * (Lx / nx)
    eta1 = stokes_eta(x, 0.0, k, a, h, g)
    psi1 = stokes_potential(x, eta1, 0.0, k, a, h, g)
    _, omega, _ = stokes_params(k, a, h, g)
    return np.tile(eta1, (nz, 1)), np.tile(psi1, (nz, 1)), (k, a, omega)


def gaussian_bump(nx: int, nz: int, Lx: float, Lz: float, A: float, sigma: float = 1.0,
                  R: float = 6.0):
    """eta0 = A exp(-r^2 / (2 sigma^2)) for r < R about the domain centre, psi = 0."""
    x = (np.arange(nx) + 0.5) * (Lx / nx)
    z = (np.arange(nz) + 0.5) * (Lz / nz)
    Z, X = np.meshgrid(z, x, indexing="ij")
    r = np.hypot(X - Lx / 2, Z - Lz / 2)
    eta = np.where(r < R, A * np.exp(-r * r / (2 * sigma * sigma)), 0.0)
    return eta, np.zeros_like(eta)


def batch_tiles(counts=((128, 40), (256, 32), (512, 16), (1024, 8)), dx: float = 0.78125,
                orders=(3, 4, 5, 6), seed0: int = 1000, g: float = 9.81, max_steepness: float = 0.1):
    """Tile list of the mixed batch: tile t draws Hs ~ U[0.5, 4], h ~ U[10, 100],
    Tp ~ U[6, 12] from the counter-based generator with seed seed0 + t; orders
    cycle through `orders` within each size. Hs is clipped so that
    k_ref Hs / 2 <= max_steepness, with k_ref = max(k_p, 2 pi / L): on tiles
    shorter than the peak wavelength only the spectral tail is resolved and the
    grid normalisation puts all of Hs there. Returns dicts with nx, nz, Lx, Lz,
    h, M, Hs, Tp, seed."""
    tiles = []
    t = 0
    for n, cnt in counts:
        L = n * dx
        for j in range(cnt):
            seed = seed0 + t
            u = uniform01(seed, np.arange(3, dtype=np.uint64))
            Hs = 0.5 + 3.5 * float(u[0])
            h = 10.0 + 90.0 * float(u[1])
            Tp = 6.0 + 6.0 * float(u[2])
            kref = max(peak_wavenumber(Tp, h, g), 2 * math.pi / L)
            Hs = min(Hs, 2 * max_steepness / kref)
            tiles.append(dict(nx=n, nz=n, Lx=L, Lz=L, h=h, M=orders[j % len(orders)], Hs=Hs, Tp=Tp, seed=seed))
            t += 1
    return tiles
