"""Closure network kernels (through the C ABI) against the FP64 oracle.

Tolerance: both sides round the same weights to FP16 and round each layer's
input to FP16, but the GPU rounds its FP32 activations, the oracle its FP64
ones; where the two straddle an FP16 rounding boundary (probability about
2^-24 / 2^-11 per value) one FP16 ulp (2^-11 relative) differs. With ~1e-4
of the values flipped and FP32 sums of <= 288 terms, relative L2 differences
stay below 1e-4, the bar used for outputs, gradients and input gradients.
"""
import numpy as np
import pytest

from oracle import closure as cl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _case(seed, B=2, H=32, W=48):
    rng = np.random.default_rng(seed)
    theta = (cl.init_params(seed) + 0.02 * rng.standard_normal(cl.param_count())).astype(np.float32)
    theta[-2:] = [0.1, -0.2]
    x = rng.standard_normal((B, 6, H, W)).astype(np.float32)
    return theta, x


def test_param_layout(zk):
    net = zk.Net()
    assert net.nparam == cl.param_count() == 20322
    theta = np.arange(net.nparam, dtype=np.float32)
    net.set_params(theta)
    assert np.array_equal(net.params(), theta)


def test_forward_matches_oracle(zk):
    import torch
    theta, x = _case(1)
    net = zk.Net(theta)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty((2, 2, 32, 48), device="cuda")
    net.forward(xd, y)
    torch.cuda.synchronize()
    yo, _ = cl.forward(theta.astype(np.float64), x.astype(np.float64))
    assert rel(y.cpu().numpy(), yo) < 1e-4


def test_backward_matches_oracle(zk):
    import torch
    theta, x = _case(2)
    rng = np.random.default_rng(9)
    dy = rng.standard_normal((2, 2, 32, 48)).astype(np.float32)
    net = zk.Net(theta)
    xd = torch.from_numpy(x).cuda()
    net.forward(xd)
    g = torch.empty(net.nparam, device="cuda")
    dx = torch.empty_like(xd)
    net.backward(torch.from_numpy(dy).cuda(), g, dx)
    torch.cuda.synchronize()
    yo, cache = cl.forward(theta.astype(np.float64), x.astype(np.float64))
    go, gxo = cl.backward(theta.astype(np.float64), cache, dy.astype(np.float64))
    gg = g.cpu().numpy()
    assert rel(gg, go) < 1e-4
    # every parameter block, including the biases, on its own
    o = 0
    for shp in cl.param_shapes():
        k = int(np.prod(shp))
        assert rel(gg[o:o + k], go[o:o + k]) < 1e-4, shp
        o += k
    assert rel(dx.cpu().numpy(), gxo) < 1e-4


def test_adam_matches_oracle(zk):
    import torch
    theta, _ = _case(3)
    rng = np.random.default_rng(4)
    net = zk.Net(theta)
    th, m, v = theta.astype(np.float64), np.zeros(theta.size), np.zeros(theta.size)
    for t in range(1, 4):
        g = rng.standard_normal(theta.size).astype(np.float32)
        net.adam(torch.from_numpy(g).cuda(), lr=1e-3)
        th, m, v = cl.adam(th, g.astype(np.float64), m, v, t, lr=1e-3)
    torch.cuda.synchronize()
    d = net.params().astype(np.float64) - th
    assert np.abs(d).max() < 1e-6 * (1 + np.abs(th).max())


def test_train_step_loss_and_descent(zk):
    import torch
    theta, x = _case(5, B=2, H=32, W=32)
    rng = np.random.default_rng(6)
    t = (0.3 * rng.standard_normal((2, 2, 32, 32))).astype(np.float32)
    net = zk.Net(theta)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    l0 = net.train_step(xd, td, lr=0.0)           # lr 0: loss of the current parameters
    yo, _ = cl.forward(theta.astype(np.float64), x.astype(np.float64))
    lo, _ = cl.mse(yo, t.astype(np.float64))
    assert abs(l0 - lo) < 1e-4 * lo
    net.set_params(theta)
    losses = [net.train_step(xd, td, lr=3e-3) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0]


def test_errors(zk):
    import torch
    net = zk.Net()
    with pytest.raises(zk.ZkError) as e:
        net.backward(torch.zeros((1, 2, 16, 16), device="cuda"))
    assert e.value.status == zk.ZK_ESTATE
    with pytest.raises(zk.ZkError) as e:
        net.forward(torch.zeros((1, 6, 24, 16), device="cuda"))
    assert e.value.status == zk.ZK_EINVAL
    with pytest.raises(zk.ZkError) as e:
        zk.zk_net_create(4, 32, 2)
    assert e.value.status == zk.ZK_EUNSUPPORTED
