"""Integrating-factor RK4 in the oracle (CPU): exact linear flow at eps = 0,
fourth-order convergence, agreement with RK4 as dt -> 0, exact mean."""
import numpy as np

from oracle import Grid, Oracle
from paper_2608_25203_b300 import seas


def _setup(eps=1.0, filt=False):
    n, L, h = 32, 60.0, 10.0
    gr = Grid(n, n, L, L, h)
    o = Oracle(gr, 3, eps=eps, filt=filt)
    e, p, _ = seas.jonswap_sea(n, n, L, L, h, 1.5, 5.0, 9)
    return o, o.spectrum(e), o.spectrum(p)


def test_eps0_is_the_exact_rotation():
    o, eh, ph = _setup(eps=0.0)
    a = (eh, ph)
    for _ in range(7):
        a = o.step_ifrk4(*a, 0.3)                     # large steps: still exact
    b = o.linear_propagate(eh, ph, 2.1)
    assert np.abs(a[0] - b[0]).max() <= 1e-12 * np.abs(b[0]).max()
    assert np.abs(a[1] - b[1]).max() <= 1e-12 * np.abs(b[1]).max()


def test_fourth_order_and_agreement_with_rk4():
    o, eh, ph = _setup()
    T = 0.4

    def solve(step, n):
        a = (eh, ph)
        for _ in range(n):
            a = step(*a, T / n)
        return a

    ref = solve(o.step_rk4, 64)
    errs = []
    for n in (4, 8, 16):
        e, _ = solve(o.step_ifrk4, n)
        errs.append(np.linalg.norm(e - ref[0]))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 11 < r1 < 22 and 11 < r2 < 22, (r1, r2)
    assert errs[2] < 1e-6 * np.linalg.norm(ref[0])


def test_mean_eta_exact():
    o, eh, ph = _setup(filt=True)
    a = (eh, ph)
    for _ in range(10):
        a = o.step_ifrk4(*a, 0.05)
    assert abs(a[0][0, 0] - eh[0, 0]) <= 1e-12 * np.abs(eh).max()
