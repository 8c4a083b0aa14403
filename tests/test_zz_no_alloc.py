"""zk_dno_static: the DNO for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (an embedding application owns the device
memory pool, or a latency-limited loop forbids allocation after start-up).
zk_dno_static serves them with a fixed scratch array inside the library. This
file is collected last on purpose. It checks, through the C ABI, that
consecutive calls with different sizes and orders agree with the context-based
zk_dno within the FP32 bar of the parity tests, so stale scratch contents from
a previous call never leak into a result; it also checks the size limit.
"""
import ctypes

import numpy as np
import pytest

from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu

CASES = [
    # nx, nz, Lx, Lz, h, M, eps, taper, Hs, Tp, seed
    (64, 64, 100.0, 100.0, 20.0, 3, 1.0, 1, 1.0, 8.0, 1),
    (128, 32, 200.0, 50.0, 15.0, 5, 0.7, 1, 1.0, 7.0, 2),
    (256, 256, 400.0, 400.0, 30.0, 6, 1.0, 0, 3.0, 10.0, 3),
    # the fullest layout the scratch array accepts: 256 x 256 with seven terms
    (256, 256, 400.0, 400.0, 30.0, 7, 0.5, 1, 2.0, 10.0, 4),
    (64, 64, 100.0, 100.0, 20.0, 3, 1.0, 1, 1.0, 8.0, 1),
]


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_dno_static_matches_dno_on_consecutive_calls():
    import torch
    from paper_2608_25203_b300 import zk
    lib = zk.load()
    torch.cuda.init()
    stream = torch.cuda.current_stream()
    for (nx, nz, Lx, Lz, h, M, eps, taper, Hs, Tp, seed) in CASES:
        eta, psi, _ = seas.jonswap_sea(nx, nz, Lx, Lz, h, Hs=Hs, Tp=Tp, seed=seed)
        eta32, psi32 = eta.astype(np.float32), psi.astype(np.float32)
        ref = zk.Zakharov(nx, nz, Lx, Lz, h, M=M, eps=eps, taper=bool(taper))
        ref.set_state(eta32, psi32)
        want = ref.dno()
        ref.close()
        d_eta = torch.from_numpy(eta32).cuda()
        d_psi = torch.from_numpy(psi32).cuda()
        d_v = torch.full_like(d_eta, float("nan"))
        torch.cuda.synchronize()
        st = lib.zk_dno_static(ctypes.c_void_p(d_eta.data_ptr()), ctypes.c_void_p(d_psi.data_ptr()),
                               ctypes.c_void_p(d_v.data_ptr()), nx, nz, Lx, Lz, h, 9.81, M, eps, taper,
                               ctypes.c_void_p(stream.cuda_stream))
        assert st == zk.ZK_OK, zk.load().zk_strerror(st)
        torch.cuda.synchronize()
        got = d_v.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        assert rel_l2(got, want) < 2e-5, (nx, nz, M)


def test_dno_static_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2608_25203_b300 import zk
    lib = zk.load()
    t = torch.zeros((512, 512), device="cuda", dtype=torch.float32)
    p = ctypes.c_void_p(t.data_ptr())
    assert lib.zk_dno_static(p, p, p, 512, 512, 1.0, 1.0, 1.0, 9.81, 3, 1.0, 1, None) == zk.ZK_EINVAL
    # 256 x 256 with 8 terms needs more than ZK_STATIC_SCRATCH_BYTES
    assert lib.zk_dno_static(p, p, p, 256, 256, 1.0, 1.0, 1.0, 9.81, 8, 1.0, 1, None) == zk.ZK_EINVAL
    assert lib.zk_dno_static(p, p, p, 48, 64, 1.0, 1.0, 1.0, 9.81, 3, 1.0, 1, None) == zk.ZK_EINVAL
