"""Pins of the closure oracle (CPU): brute-force convolution, shift equivariance,
finite-difference gradients, closed-form Adam steps, feature special cases."""
import numpy as np

from oracle import Grid, Oracle
from oracle import closure as cl


def brute_conv(x, W, b):
    n, ci, H, Wd = x.shape
    co, _, ks, _ = W.shape
    r = ks // 2
    y = np.zeros((n, co, H, Wd))
    for a in range(n):
        for o in range(co):
            for i in range(H):
                for j in range(Wd):
                    s = b[o]
                    for c in range(ci):
                        for p in range(ks):
                            for q in range(ks):
                                s += W[o, c, p, q] * x[a, c, (i + p - r) % H, (j + q - r) % Wd]
                    y[a, o, i, j] = s
    return y


def test_conv_matches_brute_force():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 4, 5))
    for ks in (1, 3):
        W = rng.standard_normal((4, 3, ks, ks))
        b = rng.standard_normal(4)
        assert np.allclose(cl.conv(x, W, b), brute_conv(x, W, b), atol=1e-12)


def test_conv_shift_equivariance_and_1x1_matmul():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 6, 8, 8))
    W = rng.standard_normal((5, 6, 3, 3))
    b = rng.standard_normal(5)
    y = cl.conv(x, W, b)
    ys = cl.conv(np.roll(x, (2, -3), axis=(2, 3)), W, b)
    assert np.allclose(ys, np.roll(y, (2, -3), axis=(2, 3)), atol=1e-12)
    W1 = rng.standard_normal((5, 6, 1, 1))
    assert np.allclose(cl.conv(x, W1, b), np.einsum("oc,ncij->noij", W1[:, :, 0, 0], x) + b[None, :, None, None])


def test_round16():
    assert cl.round16(np.array([1.0 + 2.0 ** -11]))[0] == 1.0          # tie to even
    assert cl.round16(np.array([1.0 + 3 * 2.0 ** -11]))[0] == 1.0 + 2.0 ** -9
    assert cl.round16(np.array([65504.0]))[0] == 65504.0


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    theta = cl.init_params(4) + 0.05 * rng.standard_normal(cl.param_count())
    x = rng.standard_normal((1, 6, 6, 8))
    t = rng.standard_normal((1, 2, 6, 8))

    def L(th, xx):
        y, _ = cl.forward(th, xx, fp16=False)
        return cl.mse(y, t)[0]

    y, cache = cl.forward(theta, x, fp16=False)
    _, dy = cl.mse(y, t)
    g, gx = cl.backward(theta, cache, dy)
    h = 1e-6
    idx = np.concatenate([rng.choice(cl.param_count(), 40, replace=False),
                          np.cumsum([int(np.prod(s)) for s in cl.param_shapes()]) - 1])
    for k in idx:
        e = np.zeros_like(theta)
        e[k] = h
        fd = (L(theta + e, x) - L(theta - e, x)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), k
    for _ in range(10):
        pos = tuple(rng.integers(0, s) for s in x.shape)
        e = np.zeros_like(x)
        e[pos] = h
        fd = (L(theta, x + e) - L(theta, x - e)) / (2 * h)
        assert abs(fd - gx[pos]) <= 1e-6 * max(1.0, abs(fd))


def test_adam_closed_forms():
    # first step: m_hat = g, v_hat = g^2, so the update is -lr g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = cl.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.1)
    assert np.allclose(th, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # constant gradient: m_hat = g and v_hat = g^2 at every step
    th = np.zeros(1); m = np.zeros(1); v = np.zeros(1)
    for t in range(1, 6):
        th, m, v = cl.adam(th, np.array([0.5]), m, v, t, lr=0.01, eps=0.0)
    assert abs(th[0] + 0.05) < 1e-12
    # minimises a quadratic
    th = np.array([3.0]); m = np.zeros(1); v = np.zeros(1)
    for t in range(1, 3001):
        th, m, v = cl.adam(th, 2 * (th - 1.0), m, v, t, lr=0.01)
    assert abs(th[0] - 1.0) < 1e-3


def test_features_and_target_special_cases():
    gr = Grid(16, 16, 20.0, 20.0, 5.0)
    o2, o6 = Oracle(gr, 2, eps=0.5), Oracle(gr, 6, eps=0.5)
    rng = np.random.default_rng(5)
    ph = o2.spectrum(rng.standard_normal((16, 16)) * 0.1)
    eh = np.zeros_like(ph)
    f = cl.features(o2, eh, ph)
    # flat surface: eta and its gradient vanish, both nonlinear parts vanish except the
    # Bernoulli -eps/2 |grad psi|^2 + eps/2 (G0 psi)^2 in d psi/dt
    assert np.abs(f[:3]).max() == 0.0 and np.abs(f[4]).max() < 1e-14
    assert np.allclose(f[3], o2.physical(gr.G0 * ph))
    assert np.abs(cl.target(o6, o2, eh, ph)).max() < 1e-14
    # small eta: f_6 - f_2 is O(eps^2 eta^2), the order-2 nonlinear part O(eps eta)
    eh = o2.spectrum(rng.standard_normal((16, 16)) * 1e-3)
    t = cl.target(o6, o2, eh, ph)
    eh2 = 2 * eh
    t2 = cl.target(o6, o2, eh2, ph)
    ratio = np.linalg.norm(t2[0]) / np.linalg.norm(t[0])
    assert 3.9 < ratio < 4.1


def test_closure_with_zero_net_is_base_rhs():
    gr = Grid(16, 16, 20.0, 20.0, 5.0)
    theta = np.zeros(cl.param_count())
    co = cl.ClosureOracle(gr, 2, theta, np.ones(6), np.ones(2), eps=0.5)
    o2 = Oracle(gr, 2, eps=0.5)
    rng = np.random.default_rng(6)
    eh = o2.spectrum(rng.standard_normal((16, 16)) * 0.05)
    ph = o2.spectrum(rng.standard_normal((16, 16)) * 0.1)
    a, b = co.rhs(eh, ph), o2.rhs(eh, ph)
    assert np.abs(a[0] - b[0]).max() == 0 and np.abs(a[1] - b[1]).max() == 0
    # a constant output bias adds only to the mean of d psi/dt (eta's mean is pinned to 0)
    theta = np.zeros(cl.param_count())
    theta[-2:] = [0.25, -0.5]
    co = cl.ClosureOracle(gr, 2, theta, np.ones(6), np.ones(2), eps=0.5)
    a = co.rhs(eh, ph)
    d0, d1 = a[0] - b[0], a[1] - b[1]
    assert np.abs(d0).max() < 1e-12
    assert abs(d1[0, 0] - (-0.5) * 16 * 16) < 1e-9 and np.abs(d1.ravel()[1:]).max() < 1e-9


def test_frozen_residual_step():
    """RK4 with the residual evaluated once per step (at the start state):
    * a residual that does not depend on the state (output bias only) gives the per-stage step;
    * otherwise the two steps differ by O(dt^2): the stage states move O(dt) from the start,
      and dt times an O(dt) change of the residual enters the step. Halving dt quarters it."""
    gr = Grid(16, 16, 20.0, 20.0, 5.0)
    o2 = Oracle(gr, 2, eps=0.5)
    rng = np.random.default_rng(8)
    eh = o2.spectrum(rng.standard_normal((16, 16)) * 0.05)
    ph = o2.spectrum(rng.standard_normal((16, 16)) * 0.1)
    theta = np.zeros(cl.param_count())
    theta[-2:] = [0.25, -0.5]
    co = cl.ClosureOracle(gr, 2, theta, np.ones(6), np.ones(2), eps=0.5)
    a, b = co.step_rk4_frozen(eh, ph, 0.05), co.step_rk4(eh, ph, 0.05)
    assert np.abs(a[0] - b[0]).max() < 1e-13 and np.abs(a[1] - b[1]).max() < 1e-13
    theta = cl.init_params(3) + 0.05 * rng.standard_normal(cl.param_count())
    co = cl.ClosureOracle(gr, 2, theta, np.full(6, 0.2), np.full(2, 0.05), eps=0.5)
    d = []
    for dt in (0.04, 0.02):
        a, b = co.step_rk4_frozen(eh, ph, dt), co.step_rk4(eh, ph, dt)
        d.append(np.linalg.norm(a[0] - b[0]) + np.linalg.norm(a[1] - b[1]))
    assert d[0] > 0 and 3.5 < d[0] / d[1] < 4.5, d
