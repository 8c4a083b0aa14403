"""Training data and training loop of the learned closure, on the GPU.

Data: order-M (default 6) FP32 runs of the wave step on seeded JONSWAP seas;
every `every` steps the context's state gives one pair (features, target)
through ``zk_closure_features`` (the 6 feature channels and the residual
f_M - f_base of both equations). Scales: the RMS of each channel over the
data set. Training: mini-batches drawn with a seeded generator, each step one
``zk_net_train_step`` (forward, loss, backward and Adam in the library's own
kernels). PyTorch only holds the device arrays and gathers batches.
"""
from __future__ import annotations

import math

import numpy as np

from . import seas
from . import zk


def init_params(seed: int, nparam: int) -> np.ndarray:
    """Uniform fan-in init of the 6-32-32-32-2 network (biases zero)."""
    rng = np.random.default_rng(seed)
    out = []
    for ks, ci, co in ((3, 6, 32), (3, 32, 32), (3, 32, 32), (1, 32, 2)):
        a = math.sqrt(3.0 / (ci * ks * ks))
        out.append(rng.uniform(-a, a, size=co * ci * ks * ks))
        out.append(np.zeros(co))
    theta = np.concatenate(out).astype(np.float32)
    assert theta.size == nparam
    return theta


def sea_params(seed: int, hs=(1.0, 4.0), tp=(8.0, 12.0)):
    """Hs and Tp drawn uniformly for one training trajectory from its seed."""
    u = seas.uniform01(seed, np.arange(2, dtype=np.uint64))
    return hs[0] + (hs[1] - hs[0]) * float(u[0]), tp[0] + (tp[1] - tp[0]) * float(u[1])


def make_dataset(seeds, n=512, L=400.0, h=30.0, eps=0.5, dt=0.02, M=6, base=2, snaps=20, every=10,
                 hs=(1.0, 4.0), tp=(8.0, 12.0)):
    """(X [N][6][n][n], T [N][2][n][n]) unscaled device tensors and the kept seeds."""
    import torch
    X = torch.empty((len(seeds) * snaps, 6, n, n), device="cuda")
    T = torch.empty((len(seeds) * snaps, 2, n, n), device="cuda")
    k = 0
    kept = []
    for sd in seeds:
        Hs, Tp = sea_params(sd, hs, tp)
        eta, psi, _ = seas.jonswap_sea(n, n, L, L, h, Hs, Tp, sd)
        s = zk.Zakharov(n, n, L, L, h, M=M, eps=eps)
        s.set_state(eta.astype(np.float32), psi.astype(np.float32))
        k0 = k
        ok = True
        for j in range(snaps):
            zk.zk_closure_features(s.ctx, base, X[k], T[k])
            k += 1
            s.step(dt, every)
        torch.cuda.synchronize()
        if not (torch.isfinite(X[k0:k]).all() and torch.isfinite(T[k0:k]).all()):
            ok = False
        try:
            s.energy()
        except zk.ZkError:
            ok = False
        s.close()
        if ok:
            kept.append(sd)
        else:
            k = k0
    return X[:k], T[:k], kept


def channel_scales(X, T):
    """RMS of every feature and target channel over the data set (library reduction, FP64 sums)."""
    xs = zk.zk_net_channel_rms(X)
    ts = zk.zk_net_channel_rms(T)
    return np.maximum(xs, 1e-30), np.maximum(ts, 1e-30)


def apply_scales(X, scale):
    """Divide every channel of X by its scale, in place (library kernel)."""
    zk.zk_net_scale_channels(X, (1.0 / np.asarray(scale, np.float64)).astype(np.float32))


def train(X, T, in_scale, out_scale, iters=2000, batch=4, lr=2e-3, lr_end=2e-4, seed=0, log_every=0, net=None):
    """Train a network on the scaled data; returns (net, losses). X, T are scaled in place."""
    import torch
    apply_scales(X, in_scale)
    apply_scales(T, out_scale)
    if net is None:
        net = zk.Net()
        net.set_params(init_params(seed, net.nparam))
    rng = np.random.default_rng(seed + 1)
    losses = []
    N = X.shape[0]
    for it in range(iters):
        # cosine decay from lr to lr_end
        a = lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * it / max(1, iters - 1)))
        idx = torch.as_tensor(rng.choice(N, size=batch, replace=False), device=X.device)
        xb = X.index_select(0, idx).contiguous()
        tb = T.index_select(0, idx).contiguous()
        want = log_every and (it % log_every == 0 or it == iters - 1)
        loss = net.train_step(xb, tb, a, want_loss=bool(want))
        if want:
            losses.append((it, loss))
    return net, losses


def validation_loss(net, X, T):
    """Mean-squared error of the network on scaled data (lr-0 steps: the parameters stay, the Adam moments move)."""
    import torch
    tot = 0.0
    for k in range(X.shape[0]):
        tot += net.train_step(X[k:k + 1].contiguous(), T[k:k + 1].contiguous(), 0.0)
    torch.cuda.synchronize()
    return tot / max(1, X.shape[0])
