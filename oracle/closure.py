"""FP64 CPU oracle of the learned closure (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module; the CUDA path shares no code with it.

The closure corrects a cheap low-order right-hand side towards the high-order
one. The paper's series (Sec. 3.2, Eq. 9) truncated at M terms gives the
right-hand side f_M(eta, psi) of Eqs. 4 and 10; a small network predicts the
residual f_6 - f_2 from local features of the state, and the corrected
right-hand side f_2 + R is integrated with the same RK4 and filter (Eq. 17).
The paper has no learned component; what is fixed here is this build's own
definition, restated by the CUDA kernels:

* features (6 channels, physical, unpadded grid): eta, d_x eta, d_z eta,
  G0 psi, and the nonlinear parts of f_2: (d eta/dt)_2 - G0 psi and
  (d psi/dt)_2 + g eta; each divided by its channel scale.
* target (2 channels): the physical f_6 - f_2 for eta and psi, divided by the
  output scales.
* network: three periodic 3x3 convolutions (6 -> 32 -> 32 -> 32 channels,
  tanh after each) and one 1x1 convolution (32 -> 2). Weights and the
  activations entering each convolution are rounded to FP16 (round to
  nearest even); products and sums are exact here (FP32 on the GPU).
* correction: R_hat = T(k) F[out_scale * y] per channel (unnormalised DFT,
  Nyquist modes zero, the taper T of the nonlinear terms), R_hat_eta(k=0) = 0;
  the corrected right-hand side is f_2 + R_hat.
* training: mean-squared error over all outputs, gradients by the chain rule
  through the network (rounding passed straight through), Adam (Kingma & Ba,
  2015) with bias correction.

The paper prints no learned component, so no pin comes from it; every
function below is pinned against its definition (brute-force sums, finite
differences, closed-form Adam steps, special cases of the features) by the
CPU tests, and the trained parameters are this build's own output.
"""
from __future__ import annotations

import numpy as np

from .zakharov import Oracle

CIN, WIDTH, COUT = 6, 32, 2
# (kernel size, input channels, output channels, tanh) per layer
LAYERS = ((3, CIN, WIDTH, True), (3, WIDTH, WIDTH, True), (3, WIDTH, WIDTH, True), (1, WIDTH, COUT, False))


def round16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest FP16 value (ties to even), returned as float64."""
    return np.asarray(a, dtype=np.float64).astype(np.float16).astype(np.float64)


def param_shapes():
    out = []
    for ks, ci, co, _ in LAYERS:
        out.append((co, ci, ks, ks))
        out.append((co,))
    return out


def param_count() -> int:
    return int(sum(np.prod(s) for s in param_shapes()))


def unpack(theta: np.ndarray):
    """Split the flat parameter vector into [W1, b1, ..., W4, b4] (views)."""
    parts, o = [], 0
    for s in param_shapes():
        n = int(np.prod(s))
        parts.append(theta[o:o + n].reshape(s))
        o += n
    return parts


def init_params(seed: int = 0) -> np.ndarray:
    """He-style uniform init: W ~ U(-a, a), a = sqrt(3 / fan_in); biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for ks, ci, co, _ in LAYERS:
        a = np.sqrt(3.0 / (ci * ks * ks))
        parts.append(rng.uniform(-a, a, size=(co, ci, ks, ks)).ravel())
        parts.append(np.zeros(co))
    return np.concatenate(parts)


def conv(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Periodic cross-correlation: y[n,o,i,j] = b[o] + sum_{c,p,q} W[o,c,p,q] x[n,c,i+p-r,j+q-r] (mod grid)."""
    ks = W.shape[2]
    r = ks // 2
    y = np.zeros((x.shape[0], W.shape[0]) + x.shape[2:]) + b[None, :, None, None]
    for p in range(ks):
        for q in range(ks):
            xs = np.roll(x, shift=(r - p, r - q), axis=(2, 3))      # xs[.., i, j] = x[.., i+p-r, j+q-r]
            y += np.einsum("oc,ncij->noij", W[:, :, p, q], xs)
    return y


def forward(theta: np.ndarray, x: np.ndarray, fp16: bool = True):
    """Network output y [n, 2, H, W] and the per-layer cache (input used, weights used, output)."""
    parts = unpack(theta)
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for l, (ks, ci, co, act) in enumerate(LAYERS):
        W, b = parts[2 * l], parts[2 * l + 1]
        hin = round16(h) if fp16 else h
        Wu = round16(W) if fp16 else W
        z = conv(hin, Wu, b)
        h = np.tanh(z) if act else z
        cache.append((hin, Wu, h))
    return h, cache


def backward(theta: np.ndarray, cache, dy: np.ndarray):
    """Gradient of a scalar loss w.r.t. the flat parameters and the input, given dL/dy."""
    grads = [None] * (2 * len(LAYERS))
    g = np.asarray(dy, dtype=np.float64)
    for l in reversed(range(len(LAYERS))):
        ks, ci, co, act = LAYERS[l]
        hin, Wu, h = cache[l]
        if act:
            g = g * (1.0 - h * h)                                   # d tanh
        r = ks // 2
        dW = np.zeros_like(Wu)
        dx = np.zeros_like(hin)
        for p in range(ks):
            for q in range(ks):
                xs = np.roll(hin, shift=(r - p, r - q), axis=(2, 3))
                dW[:, :, p, q] = np.einsum("noij,ncij->oc", g, xs)
                # transpose of the shift: y[i] += W x[i+p-r]  =>  dx[i] += W^T g[i-p+r]
                dx += np.roll(np.einsum("oc,noij->ncij", Wu[:, :, p, q], g), shift=(p - r, q - r), axis=(2, 3))
        grads[2 * l] = dW
        grads[2 * l + 1] = g.sum(axis=(0, 2, 3))
        g = dx
    return np.concatenate([a.ravel() for a in grads]), g


def mse(y: np.ndarray, t: np.ndarray):
    """Mean-squared error over every element and its gradient dL/dy."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1), returning new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ---- features, targets and the corrected right-hand side ---------------------
def features(o2: Oracle, eh: np.ndarray, ph: np.ndarray, in_scale=None) -> np.ndarray:
    """The 6 physical feature channels at spectral state (eh, ph) from the low-order oracle o2."""
    gr = o2.gr
    de, dp = Oracle.rhs(o2, eh, ph)          # the plain order-M right-hand side, never a closure's
    specs = [eh, 1j * gr.KX * eh, 1j * gr.KZ * eh, gr.G0 * ph, de - gr.G0 * ph, dp + gr.g * eh]
    f = np.stack([o2.physical(s) for s in specs])
    if in_scale is not None:
        f = f / np.asarray(in_scale, dtype=np.float64)[:, None, None]
    return f


def target(o6: Oracle, o2: Oracle, eh: np.ndarray, ph: np.ndarray, out_scale=None) -> np.ndarray:
    """Physical residual f_6 - f_2 (2 channels) at (eh, ph)."""
    e6, p6 = o6.rhs(eh, ph)
    e2, p2 = o2.rhs(eh, ph)
    t = np.stack([o2.physical(e6 - e2), o2.physical(p6 - p2)])
    if out_scale is not None:
        t = t / np.asarray(out_scale, dtype=np.float64)[:, None, None]
    return t


class ClosureOracle(Oracle):
    """Order-M oracle whose right-hand side adds the network's predicted residual."""

    def __init__(self, grid, M, theta, in_scale, out_scale, eps=1.0, taper=True, filt=True):
        super().__init__(grid, M, eps=eps, taper=taper, filt=filt)
        self.theta = np.asarray(theta, dtype=np.float64)
        self.in_scale = np.asarray(in_scale, dtype=np.float64)
        self.out_scale = np.asarray(out_scale, dtype=np.float64)

    def residual_hat(self, eh, ph):
        x = features(self, eh, ph, self.in_scale)
        y, _ = forward(self.theta, x[None])
        gr = self.gr
        R = [self.spectrum(self.out_scale[c] * y[0, c]) * (gr.taper if self.use_taper else 1.0) for c in range(2)]
        R[0][0, 0] = 0.0
        return R

    def rhs(self, eh, ph):
        de, dp = super().rhs(eh, ph)
        Re, Rp = self.residual_hat(eh, ph)
        return de + Re, dp + Rp

    def step_rk4_frozen(self, eh, ph, dt):
        """Classical RK4 in which the network's residual is evaluated once, at the step's start
        state, and added to the base-order right-hand side of every stage; then the filter."""
        Re, Rp = self.residual_hat(eh, ph)

        def f(e, p):
            de, dp = Oracle.rhs(self, e, p)
            return de + Re, dp + Rp

        k1e, k1p = f(eh, ph)
        k2e, k2p = f(eh + 0.5 * dt * k1e, ph + 0.5 * dt * k1p)
        k3e, k3p = f(eh + 0.5 * dt * k2e, ph + 0.5 * dt * k2p)
        k4e, k4p = f(eh + dt * k3e, ph + dt * k3p)
        eh = eh + dt / 6.0 * (k1e + 2 * k2e + 2 * k3e + k4e)
        ph = ph + dt / 6.0 * (k1p + 2 * k2p + 2 * k3p + k4p)
        return self.apply_filter(eh, ph)
