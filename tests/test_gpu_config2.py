"""Config 2 (512^2, L = 400 m, h = 30 m, M = 5, eps = 1, JONSWAP Hs 3 m, Tp 10 s, seed 2):
the FP32 and FP64 GPU paths over 1000 RK4 steps against the FP64 oracle.

The expected end state comes from the oracle's own run of the same case (FP64 numpy, 1000 RK4
steps from the FP32-rounded initial state), written by tests/golden/make_oracle_runs.py, which
imports only the oracle and the sea generator. The same script ran the oracle twin: the initial
state perturbed by 1e-7 (relative, seeded direction); the end-state difference gives the flow's
amplification A of a perturbation over the run. FP32 rounding (6e-8 per step, random-walk
growth) then allows
    tol = max(1e-4, 10 * A * 6e-8 * sqrt(steps))          (relative L2 of eta and psi).
A relative max-norm bar sits beside it: for a sea whose values and errors are both roughly
Gaussian, max|e| / max|f| tracks |e| / |f|, and 4 * tol leaves room for heavier tails.
The Hamiltonian drift (H_end - H_0) / H_0 must agree with the oracle's within what the state
error implies: H is a quadratic form (Eq. 1), so a state difference of relative size d_E in the
energy norm (g |d eta_k|^2 + G0(k) |d psi_k|^2) moves H by at most ~2 d_E + d_E^2, plus the FP32
evaluation error e_H of H at each end.
The FP64 GPU path follows the oracle to 1e-9 over the whole run (the flow contracts, A < 1, so
rounding-order differences do not grow).
"""
import math
import os

import numpy as np
import pytest

from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu

N, L, H, M, EPS, DT, STEPS = 512, 400.0, 30.0, 5, 1.0, 0.02, 1000
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config2_rk4_1000.npz")


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


@pytest.fixture(scope="module")
def golden():
    d = np.load(GOLDEN)
    assert int(d["steps"]) == STEPS
    return {k: d[k] for k in d.files}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


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


def _initial():
    e, p, _ = seas.jonswap_sea(N, N, L, L, H, 3.0, 10.0, 2)
    return e.astype(np.float32), p.astype(np.float32)


def test_config2_fp32_1000_steps_against_oracle(zk, golden):
    e32, p32 = _initial()
    oe, op = golden["eta"], golden["psi"]
    A = float(golden["A"])
    tol = max(1e-4, 10 * A * 6e-8 * math.sqrt(STEPS))
    ge, gp, drift = _run(zk, zk.ZK_F32, e32, p32)
    errs = (rel(ge, oe), rel(gp, op), rel_max(ge, oe), rel_max(gp, op))
    odrift = (float(golden["H1"]) - float(golden["H0"])) / float(golden["H0"])
    d_E = _energy_norm_rel(ge - oe, gp - op, oe, op)
    h64 = _energy(zk, zk.ZK_F64, oe, op)
    e_H = abs(_energy(zk, zk.ZK_F32, oe.astype(np.float32), op.astype(np.float32)) - h64) / h64
    bar = 2 * d_E + d_E ** 2 + 2 * e_H
    print(f"config 2 FP32 vs oracle: eta {errs[0]:.3e} psi {errs[1]:.3e} max-norm {errs[2]:.3e} {errs[3]:.3e} "
          f"(tol {tol:.3e}, A {A:.3g}); drift {drift:.6e} oracle {odrift:.6e}; d_E {d_E:.3e} e_H {e_H:.3e}")
    assert errs[0] < tol and errs[1] < tol, (errs, tol)
    assert errs[2] < 4 * tol and errs[3] < 4 * tol, (errs, tol)
    assert abs(drift - odrift) < bar, (drift, odrift, d_E, e_H)


def test_config2_fp64_1000_steps_against_oracle(zk, golden):
    e32, p32 = _initial()
    ge, gp, drift = _run(zk, zk.ZK_F64, e32.astype(np.float64), p32.astype(np.float64))
    oe, op = golden["eta"], golden["psi"]
    odrift = (float(golden["H1"]) - float(golden["H0"])) / float(golden["H0"])
    errs = (rel(ge, oe), rel(gp, op), rel_max(ge, oe), rel_max(gp, op))
    print(f"config 2 FP64 vs oracle: {errs}; drift {drift:.9e} oracle {odrift:.9e}")
    assert max(errs) < 1e-9, errs
    assert abs(drift - odrift) < 1e-10
