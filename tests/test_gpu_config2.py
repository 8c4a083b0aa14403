"""Config 2 (512^2, L = 400 m, h = 30 m, M = 5, eps = 1, JONSWAP Hs 3 m, Tp 10 s, seed 2):
the FP32 path over 1000 RK4 steps against the FP64 path.

The reference is the FP64 context. It agrees with the FP64 oracle to 1e-11 per evaluation and
to 1e-10 after 200 steps (test_gpu_parity.py); the oracle itself would take ~4000 right-hand
sides of ~0.5 s here. The tolerance is calibrated by a twin run: the FP64 initial state
perturbed by 1e-7 (relative, seeded direction) gives the flow's amplification A of a
perturbation over the run, and FP32 rounding (6e-8 per step, random-walk growth) then allows
    tol = max(1e-4, 10 * A * 6e-8 * sqrt(steps)).
The Hamiltonian drift of the two runs, (H_end - H_0) / H_0, must agree within what that state
tolerance implies. H is a quadratic form, H = 1/2 <psi, G psi> + g/2 |eta|^2 (Eq. 1), so a state
difference of relative size d_E in the energy norm (the linear part: g |d eta_k|^2 +
G0(k) |d psi_k|^2) moves H by at most ~2 d_E + d_E^2; evaluating H in FP32 adds that
evaluation's own error e_H at each end (measured here on the FP64 end state). So
    |drift_32 - drift_64| <= 2 d_E + d_E^2 + 2 e_H.
(A fixed 1e-5 bar on the drift is tighter than the 1e-4 state bar allows.)
"""
import math

import numpy as np
import pytest

from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu

N, L, H, M, EPS, DT, STEPS = 512, 400.0, 30.0, 5, 1.0, 0.02, 1000


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run(zk, prec, eta, psi):
    s = zk.Zakharov(N, N, L, L, H, M=M, precision=prec, eps=EPS)
    s.set_state(eta, psi)
    H0 = s.energy()[0]
    s.step(DT, STEPS)
    e, p = s.get_state()
    H1 = s.energy()[0]
    s.close()
    return e, p, (H1 - H0) / H0


def _energy(zk, prec, eta, psi):
    s = zk.Zakharov(N, N, L, L, H, M=M, precision=prec, eps=EPS)
    s.set_state(eta, psi)
    h = s.energy()[0]
    s.close()
    return h


def _energy_norm_rel(de, dp, e, p):
    """sqrt of (g|d eta_k|^2 + G0|d psi_k|^2) / (g|eta_k|^2 + G0|psi_k|^2): the linear part of H."""
    k = 2 * np.pi * np.fft.fftfreq(N, d=L / N)
    kk = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2)
    G0 = kk * np.tanh(kk * H)
    g = 9.81

    def q(a, b):
        return float(np.sum(g * np.abs(np.fft.fft2(a)) ** 2 + G0 * np.abs(np.fft.fft2(b)) ** 2))

    return math.sqrt(q(de, dp) / q(e, p))


def test_config2_fp32_1000_steps(zk):
    e, p, _ = seas.jonswap_sea(N, N, L, L, H, 3.0, 10.0, 2)
    e32, p32 = e.astype(np.float32), p.astype(np.float32)
    e64, p64 = e32.astype(np.float64), p32.astype(np.float64)
    ref_e, ref_p, ref_drift = _run(zk, zk.ZK_F64, e64, p64)
    assert np.all(np.isfinite(ref_e)) and np.all(np.isfinite(ref_p))
    # twin run: the amplification of a 1e-7 perturbation over the run
    rng = np.random.default_rng(2)
    de, dp = rng.standard_normal(e64.shape), rng.standard_normal(p64.shape)
    de *= 1e-7 * np.linalg.norm(e64) / np.linalg.norm(de)
    dp *= 1e-7 * np.linalg.norm(p64) / np.linalg.norm(dp)
    tw_e, tw_p, _ = _run(zk, zk.ZK_F64, e64 + de, p64 + dp)
    A = max(rel(tw_e, ref_e), rel(tw_p, ref_p)) / 1e-7
    tol = max(1e-4, 10 * A * 6e-8 * math.sqrt(STEPS))
    ge, gp, drift = _run(zk, zk.ZK_F32, e32, p32)
    assert rel(ge, ref_e) < tol and rel(gp, ref_p) < tol, (rel(ge, ref_e), rel(gp, ref_p), A, tol)
    d_E = _energy_norm_rel(ge - ref_e, gp - ref_p, ref_e, ref_p)
    h64 = _energy(zk, zk.ZK_F64, ref_e, ref_p)
    e_H = abs(_energy(zk, zk.ZK_F32, ref_e.astype(np.float32), ref_p.astype(np.float32)) - h64) / h64
    bar = 2 * d_E + d_E ** 2 + 2 * e_H
    print(f"config 2: eta {rel(ge, ref_e):.3e} psi {rel(gp, ref_p):.3e} (tol {tol:.3e}, A {A:.3g}); "
          f"drift fp32 {drift:.6e} fp64 {ref_drift:.6e}; d_E {d_E:.3e} e_H {e_H:.3e} bar {bar:.3e}")
    assert abs(drift - ref_drift) < bar, (drift, ref_drift, d_E, e_H, rel(ge, ref_e), rel(gp, ref_p), A, tol)
