"""Data preparation of the closure's training set in the library: per-channel RMS and channel
scaling of [n][c][h][w] device arrays, against numpy in FP64 on the same seeded data."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


def _data(n, c, h, w, seed):
    rng = np.random.default_rng(seed)
    # channels of very different magnitudes, as the closure's features are
    mags = 10.0 ** rng.uniform(-3, 1, size=c)
    return (rng.standard_normal((n, c, h, w)) * mags[None, :, None, None]).astype(np.float32)


@pytest.mark.parametrize("shape", [(3, 6, 16, 16), (5, 2, 32, 48), (1, 1, 16, 16)])
def test_channel_rms_matches_numpy(zk, shape):
    import torch
    x = _data(*shape, seed=sum(shape))
    want = np.sqrt(np.mean(x.astype(np.float64) ** 2, axis=(0, 2, 3)))
    got = zk.zk_net_channel_rms(torch.from_numpy(x).cuda())
    assert np.all(np.abs(got - want) <= 2.0 ** -23 * want), (got, want)
    # the same value on every call (fixed-order FP64 reduction)
    again = zk.zk_net_channel_rms(torch.from_numpy(x).cuda())
    assert np.array_equal(got, again)


def test_scale_channels_matches_numpy(zk):
    import torch
    x = _data(4, 6, 16, 32, seed=9)
    mul = np.array([0.5, 2.0, 1e-3, 7.0, -1.0, 3.25], np.float32)
    t = torch.from_numpy(x).cuda()
    zk.zk_net_scale_channels(t, mul)
    assert np.array_equal(t.cpu().numpy(), x * mul[None, :, None, None])


def test_bad_arguments_are_refused(zk):
    import torch
    t = torch.zeros((2, 3, 16, 16), device="cuda")
    with pytest.raises(ValueError):
        zk.zk_net_scale_channels(t, np.ones(2, np.float32))
    with pytest.raises(zk.ZkError):
        zk.zk_net_channel_rms(torch.zeros((0, 3, 16, 16), device="cuda"))
