"""Tensor-core (tcgen05) inference of the closure network against the oracle and
the SIMT kernels. Same rounding on both sides (FP16 weights and layer inputs,
FP32 sums), so the 1e-4 bar of the network tests applies (FP16 rounding-boundary
flips between FP32 and FP64 activations)."""
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


@pytest.mark.parametrize("H,W", [(16, 16), (32, 48), (64, 64)])
def test_tensor_core_inference_matches_oracle_and_simt(zk, H, W):
    import torch
    rng = np.random.default_rng(H * 1000 + W)
    theta = (cl.init_params(H) + 0.02 * rng.standard_normal(cl.param_count())).astype(np.float32)
    theta[-2:] = [0.05, -0.1]
    x = rng.standard_normal((1, 6, H, W)).astype(np.float32)
    net = zk.Net(theta)
    xd = torch.from_numpy(x[0]).cuda().contiguous()
    y_tc = torch.empty((2, H, W), device="cuda")
    y_simt = torch.empty((2, H, W), device="cuda")
    net.set_inference(1)
    net.predict(xd, y_tc)
    net.set_inference(0)
    net.predict(xd, y_simt)
    torch.cuda.synchronize()
    yo, _ = cl.forward(theta.astype(np.float64), x.astype(np.float64))
    assert rel(y_simt.cpu().numpy(), yo[0]) < 1e-4
    assert rel(y_tc.cpu().numpy(), yo[0]) < 1e-4
    assert rel(y_tc.cpu().numpy(), y_simt.cpu().numpy().astype(np.float64)) < 1e-4


def test_tensor_core_inference_is_deterministic(zk):
    import torch
    theta = cl.init_params(3).astype(np.float32)
    net = zk.Net(theta)
    net.set_inference(1)
    x = torch.randn((6, 128, 128), device="cuda")
    a = torch.empty((2, 128, 128), device="cuda")
    b = torch.empty_like(a)
    net.predict(x, a)
    net.predict(x, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    with pytest.raises(zk.ZkError):
        net.set_inference(3)


def test_tensor_core_wait_gives_up_with_etimeout_and_recovers(zk):
    """The bounded MMA waits of the tensor-core kernels run out (self-test mode 2: no MMA is
    issued, so nothing is in flight and no wait can complete); every block frees its TMEM and
    flags the call, zk_net_predict returns ZK_ETIMEOUT, and the same network then predicts
    correctly on the tensor cores: the device and the context stay usable."""
    import torch
    rng = np.random.default_rng(5)
    theta = cl.init_params(5).astype(np.float32)
    x = rng.standard_normal((1, 6, 32, 32)).astype(np.float32)
    net = zk.Net(theta)
    xd = torch.from_numpy(x[0]).cuda().contiguous()
    y = torch.empty((2, 32, 32), device="cuda")
    net.set_inference(2)
    for _ in range(2):
        with pytest.raises(zk.ZkError) as ei:
            net.predict(xd, y)
        assert ei.value.status == zk.ZK_ETIMEOUT
    net.set_inference(1)
    net.predict(xd, y)
    torch.cuda.synchronize()
    yo, _ = cl.forward(theta.astype(np.float64), x.astype(np.float64))
    assert rel(y.cpu().numpy(), yo[0]) < 1e-4
