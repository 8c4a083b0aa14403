"""FP64 CPU oracle of the Zakharov / HOS wave step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module. The CUDA product path never calls it and shares no
code with it.

What it computes (paper: "Hamiltonian Two-Way Coupling of Nonlinear Waves and
3D Flows", Sec. 3 and Sec. 6.1), written as plain numpy in the order the paper
states the steps:

* state: unnormalised spectra eta_hat, psi_hat on an (nz, nx) periodic grid;
  the Nyquist mode of each axis is held at zero (reading: the paper is silent).
* G0 = |k| tanh(|k| h), B0 = |k|^2 (Sec. 3.2, Eq. 6 and the text under Eq. 8).
* the DNO series G = sum_j eps^j G_j, j < M (Eq. 9; M = number of retained
  terms, HOS-3 = 3 terms, Sec. 3.2 last paragraph), each G_j from the
  Craig-Sulem / HOS recursion of the surface potential in powers of eta
  (Sec. 4.2, Eqs. 20-22 give its first three terms; Eqs. 7-8 give G1, G2):
      Phi(0) = psi,   Phi(m) = - sum_{a=1..m} eta^a/a! dz^a Phi(m-a),
      W(m)   = sum_{a=0..m} eta^a/a! dz^{a+1} Phi(m-a),
      G_m    = W(m) + |grad eta|^2 W(m-2) - [m = 1] grad eta . grad psi,
  where dz^a of a flat-strip harmonic mode has symbol |k|^a (a even) or
  |k|^(a-1) G0 (a odd). ``g1_literal``/``g2_literal`` restate Eqs. 7-8 term by
  term so tests can check the recursion against them.
* the Bernoulli right-hand side with eps (Eqs. 10-11).
* 3/2-rule de-aliasing (Sec. 6.1): fields go to the (3nz/2, 3nx/2) grid by
  zero padding, products are formed there, results are truncated back at each
  forward transform (reading: one padded grid per right-hand side). Grid(pad=3)
  pads to (3nz, 3nx) instead: the de-aliasing tailored to the higher-order
  terms that Sec. 9 names as future work; every product of the series up to
  order 5 (at most five band-limited factors) is then exact.
* taper exp[-(|k|/kc)^8], kc = (2/3) kNyq, on every forward-transformed
  nonlinear quantity (Sec. 6.1; reading: kNyq = pi / max(dx, dz)).
* (d eta/dt)_{k=0} := 0 (reading: every G_j has zero mean).
* classical RK4 (the workload's integrator), the paper's integrating-factor
  AB2 with IF-Euler bootstrap (Sec. 3.4, Eqs. 13-16), or integrating-factor
  RK4 (Lawson's form, the linear rotation of Eq. 14 exact), each followed by
  the state filter A(k) (Eq. 17) once per step.
* the Hamiltonian (Eq. 1) by Parseval.

Every function here is pinned by a CPU test (closed forms, invariants, brute
force, the paper's literal G1/G2, the Stokes reference of Sec. 8).
"""
from __future__ import annotations

from math import factorial

import numpy as np

from .dft import fwd2, inv2


def mode_index(n: int) -> np.ndarray:
    """Signed mode numbers in FFT storage order (0..n/2-1, -n/2..-1); n=1 -> [0]."""
    j = np.arange(n)
    return np.where(j < (n + 1) // 2, j, j - n)


def padded_size(n: int, pad: float = 1.5) -> int:
    """Padded length pad * n: pad 1.5 is the 3/2 rule of Sec. 6.1; pad 3 makes
    every product of up to five band-limited factors exact (no mode of such a
    product folds back into the kept band). An axis of length 1 stays 1."""
    if n == 1:
        return 1
    if n % 2:
        raise ValueError("grid sizes must be even (or 1)")
    if pad not in (1.5, 3.0, 4.5):
        raise ValueError("pad must be 1.5, 3 or 4.5")
    return int(round(pad * n))


class Grid:
    """Doubly periodic grid [nz][nx] (x fastest) over depth h, gravity g."""

    def __init__(self, nx: int, nz: int, Lx: float, Lz: float, h: float, g: float = 9.81, pad: float = 1.5):
        self.nx, self.nz, self.Lx, self.Lz, self.h, self.g = nx, nz, float(Lx), float(Lz), float(h), float(g)
        self.dx, self.dz = self.Lx / nx, self.Lz / nz
        self.pad = pad
        self.npx, self.npz = padded_size(nx, pad), padded_size(nz, pad)
        mx, mz = mode_index(nx), mode_index(nz)
        self.MZ, self.MX = np.meshgrid(mz, mx, indexing="ij")
        self.KX = 2 * np.pi * self.MX / self.Lx
        self.KZ = 2 * np.pi * self.MZ / self.Lz
        self.K = np.hypot(self.KX, self.KZ)
        # modes kept everywhere: |m| < n/2 on each axis (Nyquist excluded); n = 1 keeps m = 0
        keep_x = (2 * np.abs(self.MX) < nx) | (nx == 1)
        keep_z = (2 * np.abs(self.MZ) < nz) | (nz == 1)
        self.keep = keep_x & keep_z
        # operator symbols (Sec. 3.2)
        self.G0 = self.K * np.tanh(self.K * self.h)
        self.B0 = self.K ** 2
        # taper (Sec. 6.1): kNyq = pi / max spacing over the axes that are resolved
        sp = [d for d, n in ((self.dx, nx), (self.dz, nz)) if n > 1]
        self.knyq = np.pi / max(sp)
        self.kc = 2.0 / 3.0 * self.knyq
        self.taper = np.exp(-((self.K / self.kc) ** 8))
        # state filter (Eq. 17): k_alpha / kNyq_alpha = |m_alpha| / (n_alpha / 2)
        A = np.ones_like(self.K)
        for M_, n in ((self.MX, nx), (self.MZ, nz)):
            if n > 1:
                r = np.abs(M_) / (n / 2)
                A = A * (5 + 4 * np.cos(np.pi * r) - np.cos(2 * np.pi * r)) / 8
        self.filt = A
        # padded-grid placement of the kept modes
        self.pz = (self.MZ % self.npz)[self.keep]
        self.px = (self.MX % self.npx)[self.keep]

    def Za(self, a: int) -> np.ndarray:
        """Symbol of dz^a on a flat-strip harmonic mode: |k|^a (a even), |k|^(a-1) G0 (a odd)."""
        if a % 2 == 0:
            return self.K ** a
        return self.K ** (a - 1) * self.G0


class Oracle:
    """Plain FP64 evaluation of the order-M Zakharov right-hand side and its integrators."""

    def __init__(self, grid: Grid, M: int, eps: float = 1.0, taper: bool = True, filt: bool = True,
                 backend: str = "fft"):
        if M < 1:
            raise ValueError("M >= 1 (number of retained DNO terms)")
        self.gr, self.M, self.eps = grid, int(M), float(eps)
        self.use_taper, self.use_filter, self.backend = taper, filt, backend
        self.last_mean_residual = 0.0

    # ---- spectral <-> physical ------------------------------------------------
    def spectrum(self, f: np.ndarray) -> np.ndarray:
        """Unnormalised spectrum of a physical field, Nyquist modes set to zero."""
        F = fwd2(np.asarray(f, dtype=np.float64), self.backend)
        F[~self.gr.keep] = 0.0
        return F

    def physical(self, F: np.ndarray) -> np.ndarray:
        return inv2(F, self.backend).real

    def to_padded(self, F: np.ndarray) -> np.ndarray:
        """Band-limited interpolant of spectrum F on the 3/2 grid (Sec. 6.1, zero padding)."""
        gr = self.gr
        Fp = np.zeros((gr.npz, gr.npx), dtype=np.complex128)
        Fp[gr.pz, gr.px] = F[gr.keep]
        return inv2(Fp, self.backend).real * (gr.npx * gr.npz) / (gr.nx * gr.nz)

    def from_padded(self, p: np.ndarray) -> np.ndarray:
        """Forward transform on the 3/2 grid, truncated back to the kept modes (Sec. 6.1)."""
        gr = self.gr
        Fp = fwd2(p, self.backend)
        F = np.zeros((gr.nz, gr.nx), dtype=np.complex128)
        F[gr.keep] = Fp[gr.pz, gr.px] * (gr.nx * gr.nz) / (gr.npx * gr.npz)
        return F

    def nl_transform(self, p: np.ndarray) -> np.ndarray:
        """Forward transform of a nonlinear product: truncate, then taper (Sec. 6.1)."""
        F = self.from_padded(p)
        return F * self.gr.taper if self.use_taper else F

    # ---- the DNO series -------------------------------------------------------
    def dno_terms(self, eh: np.ndarray, ph: np.ndarray) -> dict:
        """All padded-grid quantities of one DNO evaluation (Sec. 3.2 + Sec. 4.2 recursion).

        Returns a dict with the padded fields eta, g2 = |grad eta|^2,
        d = grad eta . grad psi, q = |grad psi|^2, G0psi, the list W[m]
        (m = 0..M-1), G[m] (m = 1..M-1), Gnl = sum_m eps^m G_m, and the
        truncated, tapered spectra Phi_hat[m].
        """
        gr, M, eps = self.gr, self.M, self.eps
        eta = self.to_padded(eh)
        etax = self.to_padded(1j * gr.KX * eh)
        etaz = self.to_padded(1j * gr.KZ * eh)
        psix = self.to_padded(1j * gr.KX * ph)
        psiz = self.to_padded(1j * gr.KZ * ph)
        g2 = etax ** 2 + etaz ** 2
        d = etax * psix + etaz * psiz
        q = psix ** 2 + psiz ** 2
        # eta^a / a! on the padded grid
        ep = [np.ones_like(eta)]
        for a in range(1, M + 1):
            ep.append(ep[-1] * eta / a)
        Phi_hat = [ph]
        dz = {}  # dz[(j, a)] = padded dz^a Phi(j)

        def dzf(j, a):
            if (j, a) not in dz:
                dz[(j, a)] = self.to_padded(gr.Za(a) * Phi_hat[j])
            return dz[(j, a)]

        for m in range(1, M):
            acc = np.zeros_like(eta)
            for a in range(1, m + 1):
                acc -= ep[a] * dzf(m - a, a)
            Phi_hat.append(self.nl_transform(acc))
        W = []
        for m in range(M):
            acc = np.zeros_like(eta)
            for a in range(0, m + 1):
                acc += ep[a] * dzf(m - a, a + 1)
            W.append(acc)
        G = [W[0]]
        for m in range(1, M):
            Gm = W[m].copy()
            if m >= 2:
                Gm += g2 * W[m - 2]
            if m == 1:
                Gm -= d
            G.append(Gm)
        Gnl = np.zeros_like(eta)
        for m in range(1, M):
            Gnl += eps ** m * G[m]
        return dict(eta=eta, etax=etax, etaz=etaz, psix=psix, psiz=psiz, g2=g2, d=d, q=q,
                    G0psi=W[0], W=W, G=G, Gnl=Gnl, Phi_hat=Phi_hat)

    def dno(self, eh: np.ndarray, ph: np.ndarray) -> np.ndarray:
        """Spectrum of G(eta) psi truncated at M terms (Eqs. 9, 18), k=0 mode set to zero."""
        t = self.dno_terms(eh, ph)
        Gh = self.gr.G0 * ph + self.nl_transform(t["Gnl"])
        Gh[0, 0] = 0.0
        return Gh

    # ---- right-hand side ------------------------------------------------------
    def rhs_parts(self, eh: np.ndarray, ph: np.ndarray):
        """Linear and nonlinear parts (L y, N(y)) of Eq. 13 in spectral form."""
        gr, eps = self.gr, self.eps
        t = self.dno_terms(eh, ph)
        # Eq. 11: W = (G0 psi + sum eps^m G_m psi + eps grad eta . grad psi) / (1 + eps^2 |grad eta|^2)
        Wb = (t["G0psi"] + t["Gnl"] + eps * t["d"]) / (1.0 + eps * eps * t["g2"])
        # Eq. 10 bracket
        Npsi = eps * (-0.5 * t["q"] + 0.5 * (1.0 + eps * eps * t["g2"]) * Wb * Wb)
        Fe = self.nl_transform(t["Gnl"])
        Fp = self.nl_transform(Npsi)
        self.last_mean_residual = float(abs(Fe[0, 0]))
        Fe[0, 0] = 0.0  # reading: d eta/dt has zero mean
        Le = gr.G0 * ph
        Lp = -gr.g * eh
        return (Le, Lp), (Fe, Fp)

    def rhs(self, eh: np.ndarray, ph: np.ndarray):
        """(d eta_hat/dt, d psi_hat/dt) of Eqs. 4 and 10 with the truncated DNO."""
        (Le, Lp), (Fe, Fp) = self.rhs_parts(eh, ph)
        return Le + Fe, Lp + Fp

    # ---- integrators ----------------------------------------------------------
    def apply_filter(self, eh: np.ndarray, ph: np.ndarray):
        if not self.use_filter:
            return eh, ph
        return eh * self.gr.filt, ph * self.gr.filt

    def step_rk4(self, eh: np.ndarray, ph: np.ndarray, dt: float):
        """Classical RK4 on the full right-hand side, then the state filter (Eq. 17)."""
        k1e, k1p = self.rhs(eh, ph)
        k2e, k2p = self.rhs(eh + 0.5 * dt * k1e, ph + 0.5 * dt * k1p)
        k3e, k3p = self.rhs(eh + 0.5 * dt * k2e, ph + 0.5 * dt * k2p)
        k4e, k4p = self.rhs(eh + dt * k3e, ph + dt * k3p)
        eh = eh + dt / 6.0 * (k1e + 2 * k2e + 2 * k3e + k4e)
        ph = ph + dt / 6.0 * (k1p + 2 * k2p + 2 * k3p + k4p)
        return self.apply_filter(eh, ph)

    def if_coeffs(self, dt: float):
        """Per-mode coefficients of Eqs. 14-16 with the k=0 limits stated under Eq. 16."""
        gr = self.gr
        G0, g = gr.G0, gr.g
        w = np.sqrt(g * G0)
        pos = w > 0
        ws = np.where(pos, w, 1.0)
        c = np.cos(w * dt)
        s_over_w = np.where(pos, np.sin(w * dt) / ws, dt)              # sin(w dt)/w -> dt
        G0s_over_w = np.where(pos, G0 / ws * np.sin(w * dt), 0.0)      # (G0/w) sin(w dt) -> 0
        gs_over_w = np.where(pos, g / ws * np.sin(w * dt), g * dt)     # (g/w) sin(w dt) -> g dt
        omc_g = (1.0 - c) / g                                          # (1 - cos)/g -> 0
        omc_G0 = np.where(pos, (1.0 - c) / np.where(pos, G0, 1.0), 0.5 * g * dt * dt)
        return c, s_over_w, G0s_over_w, gs_over_w, omc_g, omc_G0

    def step_ifab2(self, eh, ph, dt, hist=None):
        """One integrating-factor AB2 step (Eqs. 15-16); hist = (Fe, Fp, dt) of the previous step.

        With no history, or a history taken at another dt, F* = F_n (IF-Euler
        bootstrap, Sec. 3.4). Returns (eh, ph, new_hist). Filter applied after.
        """
        (_, _), (Fe, Fp) = self.rhs_parts(eh, ph)
        if hist is None or hist[2] != dt:
            Fse, Fsp = Fe, Fp
        else:
            Fse = 1.5 * Fe - 0.5 * hist[0]
            Fsp = 1.5 * Fp - 0.5 * hist[1]
        c, sw, G0sw, gsw, omc_g, omc_G0 = self.if_coeffs(dt)
        e1 = c * eh + G0sw * ph + sw * Fse + omc_g * Fsp
        p1 = -gsw * eh + c * ph - omc_G0 * Fse + sw * Fsp
        e1, p1 = self.apply_filter(e1, p1)
        return e1, p1, (Fe, Fp, dt)

    def linear_propagate(self, eh, ph, dt):
        """Exact linear flow of Eq. 14 (no nonlinear forcing, no filter)."""
        c, sw, G0sw, gsw, _, _ = self.if_coeffs(dt)
        return c * eh + G0sw * ph, -gsw * eh + c * ph

    def step_ifrk4(self, eh: np.ndarray, ph: np.ndarray, dt: float):
        """Integrating-factor RK4 (Lawson's form): the linear part of Eq. 13 exactly, via the
        rotation E_t of Eq. 14, the nonlinear part N by classical RK4 in the rotating frame:
            k1 = N(y), k2 = N(E_{h/2}(y + h/2 k1)), k3 = N(E_{h/2} y + h/2 k2),
            k4 = N(E_h y + h E_{h/2} k3),
            y' = E_h y + h/6 (E_h k1 + 2 E_{h/2} (k2 + k3) + k4),
        then the state filter (Eq. 17) once per step."""
        h = dt
        E = self.linear_propagate

        def N(e, p):
            _, (Fe, Fp) = self.rhs_parts(e, p)
            return Fe, Fp

        k1 = N(eh, ph)
        k2 = N(*E(eh + 0.5 * h * k1[0], ph + 0.5 * h * k1[1], 0.5 * h))
        yh = E(eh, ph, 0.5 * h)
        k3 = N(yh[0] + 0.5 * h * k2[0], yh[1] + 0.5 * h * k2[1])
        yf = E(eh, ph, h)
        k3h = E(k3[0], k3[1], 0.5 * h)
        k4 = N(yf[0] + h * k3h[0], yf[1] + h * k3h[1])
        k1f = E(k1[0], k1[1], h)
        k23 = E(k2[0] + k3[0], k2[1] + k3[1], 0.5 * h)
        e1 = yf[0] + h / 6.0 * (k1f[0] + 2.0 * k23[0] + k4[0])
        p1 = yf[1] + h / 6.0 * (k1f[1] + 2.0 * k23[1] + k4[1])
        return self.apply_filter(e1, p1)

    # ---- state recovery and the relaxation source (Secs. 3.5 and 5) -----------
    def dno_inverse(self, eh: np.ndarray, vh: np.ndarray, iters: int = 8, ph0: np.ndarray = None):
        """Inverse DNO map of Eq. 19 by fixed-point iteration.

        psi(0) = G0^{-1} v, psi(n+1) = G0^{-1}(v - [G(eta) - G0] psi(n)), where
        G(eta) - G0 is the same truncated, tapered nonlinear part as in the
        right-hand side (all retained orders, each weighted by eps^m). G0 has
        no inverse on the k = 0 mode; that mode of psi is taken from ph0
        (reading: the mean potential is kept), else zero.
        """
        gr = self.gr
        G0 = gr.G0
        inv = np.where(G0 > 0, 1.0 / np.where(G0 > 0, G0, 1.0), 0.0)
        mean = ph0[0, 0] if ph0 is not None else 0.0
        ph = vh * inv
        ph[0, 0] = mean
        for _ in range(iters):
            nl = self.dno(eh, ph) - G0 * ph
            nl[0, 0] = 0.0
            ph = (vh - nl) * inv
            ph[0, 0] = mean
        return ph

    def relax(self, eh: np.ndarray, ph: np.ndarray, dt: float, sigma: np.ndarray, eta_target: np.ndarray,
              iters: int = 8):
        """Eq. 34 then Eq. 35 after a wave step (the splitting of Sec. 5.3, Alg. 2 steps 7-9).

        v = G(eta) psi at the post-step state; eta <- eta_t + (eta - eta_t) exp(-sigma dt)
        pointwise in physical space; psi <- G(eta_relaxed)^{-1} v.
        """
        vh = self.dno(eh, ph)
        eta = self.physical(eh)
        eta_r = eta_target + (eta - eta_target) * np.exp(-sigma * dt)
        eh_r = self.spectrum(eta_r)
        return eh_r, self.dno_inverse(eh_r, vh, iters=iters, ph0=ph)

    # ---- diagnostics ----------------------------------------------------------
    def energy(self, eh: np.ndarray, ph: np.ndarray):
        """Hamiltonian of Eq. 1 by Parseval: returns (H, kinetic, potential, mean_eta)."""
        gr = self.gr
        Gh = self.dno(eh, ph)
        w = gr.dx * gr.dz / (gr.nx * gr.nz)
        kin = 0.5 * w * float(np.sum(np.real(np.conj(ph) * Gh)))
        pot = 0.5 * gr.g * w * float(np.sum(np.abs(eh) ** 2))
        mean = float(eh[0, 0].real) / (gr.nx * gr.nz)
        return kin + pot, kin, pot, mean

    # ---- Eqs. 7-8 written out literally (for checking the recursion) ---------
    def _mult(self, sym, p):
        """A Fourier multiplier applied to a padded-grid product: taper*truncate, multiply, back to padded."""
        return self.to_padded(sym * self.nl_transform(p))

    def g1_literal(self, eh, ph):
        """Eq. 7: G1 psi = -G0(eta G0 psi) - div(eta grad psi), on the padded grid."""
        gr = self.gr
        eta = self.to_padded(eh)
        G0psi = self.to_padded(gr.G0 * ph)
        psix = self.to_padded(1j * gr.KX * ph)
        psiz = self.to_padded(1j * gr.KZ * ph)
        t1 = -self._mult(gr.G0, eta * G0psi)
        div = self._mult(1j * gr.KX, eta * psix) + self._mult(1j * gr.KZ, eta * psiz)
        return t1 - div

    def g2_literal(self, eh, ph):
        """Eq. 8, its five terms in the order printed, on the padded grid."""
        gr = self.gr
        eta = self.to_padded(eh)
        G0psi = self.to_padded(gr.G0 * ph)
        B0psi = self.to_padded(gr.B0 * ph)
        G0B0psi = self.to_padded(gr.G0 * gr.B0 * ph)
        etax = self.to_padded(1j * gr.KX * eh)
        etaz = self.to_padded(1j * gr.KZ * eh)
        t1 = self._mult(gr.G0, eta * self._mult(gr.G0, eta * G0psi))
        t2 = -0.5 * self._mult(gr.G0, eta ** 2 * B0psi)
        t3 = -eta * self._mult(gr.B0, eta * G0psi)
        t4 = 0.5 * eta ** 2 * G0B0psi
        t5 = (etax ** 2 + etaz ** 2) * G0psi
        return t1 + t2 + t3 + t4 + t5


def run(oracle: Oracle, eta: np.ndarray, psi: np.ndarray, dt: float, nsteps: int,
        integrator: str = "rk4", callback=None):
    """Advance physical (eta, psi) by nsteps; returns final physical fields."""
    eh, ph = oracle.spectrum(eta), oracle.spectrum(psi)
    hist = None
    for n in range(nsteps):
        if integrator == "rk4":
            eh, ph = oracle.step_rk4(eh, ph, dt)
        elif integrator == "ifab2":
            eh, ph, hist = oracle.step_ifab2(eh, ph, dt, hist)
        elif integrator == "ifrk4":
            eh, ph = oracle.step_ifrk4(eh, ph, dt)
        else:
            raise ValueError(integrator)
        if callback is not None:
            callback(n + 1, eh, ph)
    return oracle.physical(eh), oracle.physical(ph)


def sigma_box(gr: Grid, x0: float, x1: float, z0: float, z1: float, wb: float, sigma_max: float):
    """Relaxation rate of Eq. 33 on an axis-aligned box footprint.

    sigma = sigma_max * rho(dist / wb) inside the box, 0 outside, with dist the
    distance to the nearest box edge and rho the cubic smoothstep
    rho(s) = 3 s^2 - 2 s^3 on [0, 1], clamped to 1 beyond (reading: the paper
    asks only for a smooth ramp with rho(0) = 0 and rho(1) = 1).
    """
    x = np.arange(gr.nx) * gr.dx
    z = np.arange(gr.nz) * gr.dz
    Z, X = np.meshgrid(z, x, indexing="ij")
    inside = (X >= x0) & (X <= x1) & (Z >= z0) & (Z <= z1)
    dist = np.minimum(np.minimum(X - x0, x1 - X), np.minimum(Z - z0, z1 - Z))
    s = np.clip(dist / wb, 0.0, 1.0)
    rho = s * s * (3.0 - 2.0 * s)
    return np.where(inside, sigma_max * rho, 0.0)


def factorial_table(M: int):
    return [factorial(a) for a in range(M + 1)]
