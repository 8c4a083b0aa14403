"""Asynchronous state I/O (pinned host buffers, copy stream, two staging slots)
gives exactly what the synchronous calls give, over interleaved steps."""
import numpy as np
import pytest

from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_async_io_matches_sync(zk, dtype):
    import torch
    n, L = 128, 100.0
    prec = zk.ZK_F32 if dtype == np.float32 else zk.ZK_F64
    seqs = []
    for sd in (1, 2, 3):
        e, p, _ = seas.jonswap_sea(n, n, L, L, 20.0, 1.5, 6.0, sd)
        seqs.append((e.astype(dtype), p.astype(dtype)))
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    a = zk.Zakharov(n, n, L, L, 20.0, M=4, precision=prec)
    b = zk.Zakharov(n, n, L, L, 20.0, M=4, precision=prec)
    outs = [(torch.empty((n, n), dtype=tdt).pin_memory(), torch.empty((n, n), dtype=tdt).pin_memory()) for _ in seqs]
    ins = [(torch.from_numpy(e).pin_memory(), torch.from_numpy(p).pin_memory()) for e, p in seqs]
    for (he, hp), (oe, op) in zip(ins, outs):          # three round trips in flight, no host wait
        zk.zk_set_state_async(a.ctx, he, hp)
        a.step(0.02, 2)
        zk.zk_get_state_async(a.ctx, oe, op)
    zk.zk_sync(a.ctx)
    for (e, p), (oe, op) in zip(seqs, outs):
        b.set_state(e, p)
        b.step(0.02, 2)
        we, wp = b.get_state(dtype)
        assert np.array_equal(oe.numpy(), we) and np.array_equal(op.numpy(), wp)


def test_async_io_errors(zk):
    import torch
    s = zk.Zakharov(64, 64, 50.0, 50.0, 10.0, M=3)
    o = torch.empty((64, 64)).pin_memory()
    with pytest.raises(zk.ZkError) as e:
        zk.zk_get_state_async(s.ctx, o, o)
    assert e.value.status == zk.ZK_ESTATE
    zk.zk_io_join(s.ctx)                                 # nothing issued yet: a no-op
