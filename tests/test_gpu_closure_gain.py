"""What the trained closure gains over the method without it (GPU).

A small seeded training run (order-6 data on 16 seas at 256^2, 800 Adam
steps in the library's kernels) must cut the eta error of the order-2 series
against order 6 after 200 RK4 steps on an unseen sea by at least half, and
the network must be deterministic (same data, same seeds -> same parameters).
"""
import numpy as np
import pytest

from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu

N, L, H, EPS, DT = 256, 200.0, 30.0, 0.5, 0.02


@pytest.fixture(scope="module")
def trained():
    import torch
    from paper_2608_25203_b300 import closure_train as ct
    from paper_2608_25203_b300 import zk
    zk.load()
    nets = []
    for _ in range(2):
        X, T, kept = ct.make_dataset(list(range(300, 316)), n=N, L=L, h=H, eps=EPS, snaps=10, every=10)
        ins, outs = ct.channel_scales(X, T)
        net, losses = ct.train(X, T, ins, outs, iters=800, batch=4, lr=1e-3, lr_end=1e-5, seed=3)
        torch.cuda.synchronize()
        nets.append((net, ins, outs, kept))
    return zk, nets


def _run(zk, M, steps, net=None, ins=None, outs=None):
    eta, psi, _ = seas.jonswap_sea(N, N, L, L, H, 3.0, 10.0, 7)
    s = zk.Zakharov(N, N, L, L, H, M=6 if net else M, eps=EPS)
    s.set_state(eta.astype(np.float32), psi.astype(np.float32))
    if net:
        zk.zk_closure_set(s.ctx, net.n, 2, ins, outs, check_every=0)
    s.step(DT, steps)
    return s.get_state()[0]


def test_training_is_deterministic(trained):
    zk, nets = trained
    assert len(nets[0][3]) == 16
    assert np.array_equal(nets[0][0].params(), nets[1][0].params())


def test_closure_gain_over_base_order(trained):
    zk, nets = trained
    net, ins, outs, _ = nets[0]
    ref = _run(zk, 6, 200)
    e2 = np.linalg.norm(_run(zk, 2, 200) - ref) / np.linalg.norm(ref)
    ec = np.linalg.norm(_run(zk, 2, 200, net, ins, outs) - ref) / np.linalg.norm(ref)
    assert ec < 0.5 * e2, (ec, e2)
