"""Reflecting walls by even extension (Sec. 3.3, Eq. 12) on the GPU.

The tank state is mirrored across each wall into the doubled periodic grid;
every operator of the step commutes with that reflection, so the doubled
state must stay mirror-symmetric and the tank is its corner. Checked against
the oracle run on the explicitly mirrored field (FP64, 1e-11).
"""
import numpy as np
import pytest

from oracle import Grid, Oracle, run
from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


def mirror(f):
    mz, mx = f.shape
    g = np.empty((2 * mz, 2 * mx), f.dtype)
    g[:mz, :mx] = f
    g[:mz, mx:] = f[:, ::-1]
    g[mz:, :] = g[:mz, :][::-1, :]
    return g


def _bump(m, L):
    # off-centre Gaussian bump of the paper's tank (sigma 1 m, truncated at R = 6 m), psi from a shifted mode
    x = (np.arange(m) + 0.5) * (L / m)
    Z, X = np.meshgrid(x, x, indexing="ij")
    r = np.hypot(X - 0.35 * L, Z - 0.6 * L)
    eta = np.where(r < 6.0, 0.3 * np.exp(-r * r / 2.0), 0.0)
    psi = 0.2 * np.cos(2 * np.pi * X / L) * np.sin(np.pi * Z / L)
    return eta, psi


@pytest.mark.parametrize("integrator", ["rk4", "ifab2", "ifrk4"])
def test_tank_matches_oracle_on_mirrored_grid(zk, integrator):
    m, L, h, M = 32, 20.0, 20.0, 3
    eta, psi = _bump(m, L)
    o = Oracle(Grid(2 * m, 2 * m, 2 * L, 2 * L, h), M)
    e, p = run(o, mirror(eta), mirror(psi), 0.01, 30, integrator=integrator)
    s = zk.Zakharov(2 * m, 2 * m, 2 * L, 2 * L, h, M=M, precision=1)
    code = {"rk4": zk.ZK_RK4, "ifab2": zk.ZK_IFAB2, "ifrk4": zk.ZK_IFRK4}[integrator]
    zk.zk_set_options(s.ctx, integrator=code)
    zk.zk_set_state_tank(s.ctx, eta, psi)
    s.step(0.01, 30)
    te, tp = np.empty_like(eta), np.empty_like(psi)
    zk.zk_get_state_tank(s.ctx, te, tp)
    assert np.linalg.norm(te - e[:m, :m]) / np.linalg.norm(e[:m, :m]) < 1e-11
    assert np.linalg.norm(tp - p[:m, :m]) / np.linalg.norm(p[:m, :m]) < 1e-11
    # the doubled state is still mirror-symmetric
    fe, fp = s.get_state()
    assert np.max(np.abs(fe - mirror(fe[:m, :m]))) < 1e-12 * max(1.0, np.max(np.abs(fe)))


def test_tank_device_io_fp32(zk):
    import torch
    m, L, h, M = 64, 20.0, 1.0, 2
    eta, psi = _bump(m, L)
    s = zk.Zakharov(2 * m, 2 * m, 2 * L, 2 * L, h, M=M, precision=0)
    de = torch.from_numpy(eta.astype(np.float32)).cuda()
    dp = torch.from_numpy(psi.astype(np.float32)).cuda()
    zk.zk_set_state_tank(s.ctx, de, dp)
    oe, op = torch.empty_like(de), torch.empty_like(dp)
    zk.zk_get_state_tank(s.ctx, oe, op)
    o = Oracle(Grid(2 * m, 2 * m, 2 * L, 2 * L, h), M)
    want = o.physical(o.spectrum(mirror(eta)))[:m, :m]   # Nyquist modes removed
    # FP32 forward + inverse 2D FFT: rounding grows like log2(n) per pass, u = 2^-24
    tol = 2 * np.log2((2 * m) ** 2) * 2.0 ** -24
    assert np.linalg.norm(oe.cpu().numpy() - want) / np.linalg.norm(want) < tol
