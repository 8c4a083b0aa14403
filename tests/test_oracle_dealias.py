"""Exact de-aliasing of the series (CPU): with the 3N padding every product of
the order-M series (M <= 5) has at most five band-limited factors, so no mode
folds back into the kept band. Pinned by comparison with an even larger
padding (4.5N), and by the mean of d eta / dt, which vanishes for the exact
operator and is only ~1e-6 under the 3/2 rule."""
import numpy as np
import pytest

from oracle import Grid, Oracle


def _state(n=32, L=40.0, h=8.0):
    # every kept mode populated (a band-limited sea aliases too little to tell the paddings apart)
    rng = np.random.default_rng(21)
    o = Oracle(Grid(n, n, L, L, h), 1)
    eta = o.physical(o.spectrum(0.05 * rng.standard_normal((n, n))))
    psi = o.physical(o.spectrum(0.2 * rng.standard_normal((n, n))))
    return eta, psi


@pytest.mark.parametrize("M", [2, 3, 4, 5])
def test_dno_exact_with_3n_padding(M):
    eta, psi = _state()
    outs = []
    for pad in (3.0, 4.5):
        o = Oracle(Grid(32, 32, 40.0, 40.0, 8.0, pad=pad), M, eps=1.0, taper=False)
        eh, ph = o.spectrum(eta), o.spectrum(psi)
        outs.append(o.dno(eh, ph))
    assert np.abs(outs[0] - outs[1]).max() <= 1e-12 * np.abs(outs[1]).max()
    # the 3/2 rule differs from the exact value by its aliasing error
    o = Oracle(Grid(32, 32, 40.0, 40.0, 8.0), M, eps=1.0, taper=False)
    d15 = o.dno(o.spectrum(eta), o.spectrum(psi))
    if M >= 3:   # G_2 and beyond hold cubic and higher products
        assert np.abs(d15 - outs[1]).max() > 1e3 * np.abs(outs[0] - outs[1]).max()
    else:        # G_1 is quadratic: the 3/2 rule is already exact
        assert np.abs(d15 - outs[1]).max() <= 1e-12 * np.abs(outs[1]).max()


def test_mean_residual_vanishes_with_3n_padding():
    eta, psi = _state()
    res = {}
    for pad in (1.5, 3.0):
        o = Oracle(Grid(32, 32, 40.0, 40.0, 8.0, pad=pad), 5, eps=1.0, taper=False)
        eh, ph = o.spectrum(eta), o.spectrum(psi)
        (Le, Lp), (Fe, Fp) = o.rhs_parts(eh, ph)
        res[pad] = o.last_mean_residual / np.abs(o.physical(Fe)).max() / (32 * 32)
    assert res[3.0] < 1e-14
    assert res[1.5] > 1e3 * res[3.0]


def test_padded_sizes():
    from oracle import padded_size
    assert padded_size(64) == 96 and padded_size(64, 3.0) == 192 and padded_size(1, 3.0) == 1
    with pytest.raises(ValueError):
        padded_size(64, 2.0)
