"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
  * FP64 contexts compute the same discrete algorithm as the oracle in the
    same precision; only the FFT factorisation and summation order differ,
    so results agree to ~1e-13 relative per evaluation (bar: 1e-11), and to
    1e-10 after 200 RK4 steps.
  * FP32 contexts: one transform has relative error ~ log2(N) * 6e-8; a
    right-hand side chains 2M+1 of them plus products, so a single evaluation
    is bounded by 2e-5 relative (L2). Stepped runs: a twin oracle run shows
    the flow does not amplify perturbations (the state filter contracts
    them: 6e-8 in -> 1e-8 after 200 steps of config 1), so the error is the
    FP32 rounding each step adds; bar = worst-case linear accumulation,
    4 * nsteps * 2^-24.
"""
import math

import numpy as np
import pytest

from oracle import Grid, Oracle, run
from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401  (initialises the CUDA context the library shares)
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _sea(nx, nz, Lx, Lz, h, Hs, Tp, seed):
    eta, psi, _ = seas.jonswap_sea(nx, nz, Lx, Lz, h, Hs=Hs, Tp=Tp, seed=seed)
    return eta, psi


CASES = [
    # nx, nz, Lx, Lz, h, M, Hs, Tp
    (64, 64, 100.0, 100.0, 20.0, 3, 1.0, 8.0),    # config 1 grid
    (16, 16, 40.0, 40.0, 10.0, 2, 0.5, 6.0),      # smallest grid
    (128, 32, 200.0, 50.0, 15.0, 5, 1.0, 7.0),    # non-square
    (32, 256, 60.0, 480.0, 25.0, 4, 1.5, 8.0),    # non-square, other way
    (256, 256, 400.0, 400.0, 30.0, 6, 3.0, 10.0),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", CASES[:4])
def test_state_roundtrip(zk, case, prec):
    nx, nz, Lx, Lz, h, M, Hs, Tp = case
    rng = np.random.default_rng(nx + nz)
    eta = rng.standard_normal((nz, nx))
    psi = rng.standard_normal((nz, nx))
    o = Oracle(Grid(nx, nz, Lx, Lz, h), M)
    want_e = o.physical(o.spectrum(eta))  # Nyquist modes removed
    want_p = o.physical(o.spectrum(psi))
    s = zk.Zakharov(nx, nz, Lx, Lz, h, M=M, precision=prec)
    s.set_state(eta, psi)
    e, p = s.get_state()
    tol = 1e-13 if prec == 1 else 3e-7
    assert rel_l2(e, want_e) < tol and rel_l2(p, want_p) < tol


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("case", CASES)
def test_dno_and_rhs_match_oracle(zk, case, prec):
    nx, nz, Lx, Lz, h, M, Hs, Tp = case
    eta, psi = _sea(nx, nz, Lx, Lz, h, Hs, Tp, seed=nx * 7 + nz)
    o = Oracle(Grid(nx, nz, Lx, Lz, h), M)
    eh, ph = o.spectrum(eta), o.spectrum(psi)
    Gw = o.physical(o.dno(eh, ph))
    de, dp = o.rhs(eh, ph)
    de, dp = o.physical(de), o.physical(dp)
    s = zk.Zakharov(nx, nz, Lx, Lz, h, M=M, precision=prec)
    s.set_state(eta, psi)
    G = s.dno()
    ge, gp = s.rhs()
    tol = 1e-11 if prec == 1 else 2e-5
    assert rel_l2(G, Gw) < tol
    assert rel_l2(ge, de) < tol
    assert rel_l2(gp, dp) < tol
    # the nonlinear part alone (RHS minus its linear part) also matches
    lin = o.physical(-o.gr.g * eh)
    assert rel_l2(gp - lin, dp - lin) < (1e-10 if prec == 1 else 1e-3)


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5, 6, 7, 8])
def test_every_order_fp64(zk, M):
    nx, nz, Lx, Lz, h = 32, 32, 80.0, 80.0, 12.0
    eta, psi = _sea(nx, nz, Lx, Lz, h, 1.2, 6.0, seed=M)
    o = Oracle(Grid(nx, nz, Lx, Lz, h), M, eps=0.7)
    de, dp = o.rhs(o.spectrum(eta), o.spectrum(psi))
    s = zk.Zakharov(nx, nz, Lx, Lz, h, M=M, precision=1, eps=0.7)
    s.set_state(eta, psi)
    ge, gp = s.rhs()
    assert rel_l2(ge, o.physical(de)) < 1e-11
    assert rel_l2(gp, o.physical(dp)) < 1e-11


@pytest.mark.parametrize("taper,filt,eps", [(0, 1, 1.0), (1, 0, 1.0), (1, 1, 0.0), (0, 0, 0.35)])
def test_options_fp64(zk, taper, filt, eps):
    nx, nz, Lx, Lz, h, M = 64, 32, 100.0, 50.0, 20.0, 4
    eta, psi = _sea(nx, nz, Lx, Lz, h, 1.0, 8.0, seed=5)
    o = Oracle(Grid(nx, nz, Lx, Lz, h), M, eps=eps, taper=bool(taper), filt=bool(filt))
    e, p = run(o, eta, psi, 0.05, 10)
    s = zk.Zakharov(nx, nz, Lx, Lz, h, M=M, precision=1, eps=eps, taper=taper, filter=filt)
    s.set_state(eta, psi)
    s.step(0.05, 10)
    ge, gp = s.get_state()
    assert rel_l2(ge, e) < 1e-11 and rel_l2(gp, p) < 1e-11


def test_config1_fp64_200_steps(zk):
    """Config 1: 64^2, L = 100 m, h = 20 m, M = 3, RK4 dt = 0.02 s, 200 steps, FP64."""
    nx = nz = 64
    eta, psi = _sea(nx, nz, 100.0, 100.0, 20.0, 1.0, 8.0, seed=1)
    o = Oracle(Grid(nx, nz, 100.0, 100.0, 20.0), 3)
    eh, ph = o.spectrum(eta), o.spectrum(psi)
    H0 = o.energy(eh, ph)[0]
    e, p = run(o, eta, psi, 0.02, 200)
    H1 = o.energy(o.spectrum(e), o.spectrum(p))[0]
    s = zk.Zakharov(nx, nz, 100.0, 100.0, 20.0, M=3, precision=1)
    s.set_state(eta, psi)
    Hg0 = s.energy()[0]
    s.step(0.02, 200)
    ge, gp = s.get_state()
    Hg1 = s.energy()[0]
    assert rel_l2(ge, e) < 1e-10 and rel_l2(gp, p) < 1e-10
    assert abs(Hg0 - H0) / H0 < 1e-12 and abs(Hg1 - H1) / H0 < 1e-12


def test_config1_fp32_200_steps(zk):
    nx = nz = 64
    eta, psi = _sea(nx, nz, 100.0, 100.0, 20.0, 1.0, 8.0, seed=1)
    o = Oracle(Grid(nx, nz, 100.0, 100.0, 20.0), 3)
    e, p = run(o, eta, psi, 0.02, 200)
    s = zk.Zakharov(nx, nz, 100.0, 100.0, 20.0, M=3, precision=0)
    s.set_state(eta.astype(np.float32), psi.astype(np.float32))
    s.step(0.02, 200)
    ge, gp = s.get_state()
    tol = 4 * 200 * 2.0 ** -24
    assert rel_l2(ge, e) < tol and rel_l2(gp, p) < tol


@pytest.mark.parametrize("prec", [0, 1])
def test_energy_matches_oracle(zk, prec):
    nx, nz, Lx, Lz, h, M = 128, 64, 200.0, 100.0, 25.0, 5
    eta, psi = _sea(nx, nz, Lx, Lz, h, 2.0, 8.0, seed=9)
    o = Oracle(Grid(nx, nz, Lx, Lz, h), M)
    H, kin, pot, mean = o.energy(o.spectrum(eta), o.spectrum(psi))
    s = zk.Zakharov(nx, nz, Lx, Lz, h, M=M, precision=prec)
    s.set_state(eta, psi)
    gH, gk, gp, gm = s.energy()
    tol = 1e-12 if prec == 1 else 1e-6
    assert abs(gH - H) / H < tol and abs(gk - kin) / kin < tol and abs(gp - pot) / pot < tol
    assert abs(gm - mean) < 1e-6


def test_step_is_deterministic(zk):
    nx, nz = 128, 128
    eta, psi = _sea(nx, nz, 200.0, 200.0, 30.0, 3.0, 8.0, seed=3)
    out = []
    for _ in range(2):
        s = zk.Zakharov(nx, nz, 200.0, 200.0, 30.0, M=5)
        s.set_state(eta.astype(np.float32), psi.astype(np.float32))
        s.step(0.02, 20)
        out.append(s.get_state(np.float32))
        s.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_bad_arguments(zk):
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_create(48, 64, 1.0, 1.0, 1.0, 9.81, 3)
    assert ei.value.status == zk.ZK_EINVAL
    with pytest.raises(zk.ZkError):
        zk.zk_create(64, 64, 1.0, 1.0, 1.0, 9.81, 0)
    s = zk.Zakharov(16, 16, 1.0, 1.0, 1.0, M=2)
    with pytest.raises(zk.ZkError) as ei:
        s.step(0.01, 1)
    assert ei.value.status == zk.ZK_ESTATE
    with pytest.raises(zk.ZkError):
        zk.zk_set_options(s.ctx, eps=1.5)
