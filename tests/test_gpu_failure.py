"""Failure detection and checkpoint/resume on the GPU, without any GPU fault.

* A non-finite state is made on the host (a NaN planted in eta before upload); the energy
  reduction counts non-finite state entries in FP64 and zk_energy returns ZK_ENONFINITE, and the
  context stays usable: a finite state set afterwards evaluates normally.
* Checkpoint and resume include the IF-AB2 forcing history (Sec. 3.4, Eqs. 15-16): a run that is
  checkpointed after k steps and resumed in a fresh context continues bitwise identically to the
  uninterrupted run. Resuming from the state alone (zk_set_state) restarts the history with an
  IF-Euler step and differs, which shows the history matters.
* A checkpoint whose header does not match the context, or a short buffer, is refused with
  ZK_EINVAL before any device work.
"""
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


def _sea(n=64):
    e, p, _ = seas.jonswap_sea(n, n, 100.0, 100.0, 20.0, 1.0, 8.0, 1)
    return e, p


def test_nan_state_reports_enonfinite_and_context_recovers(zk):
    e, p = _sea()
    s = zk.Zakharov(64, 64, 100.0, 100.0, 20.0, M=3)
    bad = e.astype(np.float32).copy()
    bad[5, 7] = np.nan
    s.set_state(bad, p.astype(np.float32))
    with pytest.raises(zk.ZkError) as ei:
        s.energy()
    assert ei.value.status == zk.ZK_ENONFINITE
    # stepping a non-finite state is plain arithmetic: no fault, still non-finite
    s.step(0.02, 3)
    with pytest.raises(zk.ZkError) as ei:
        s.energy()
    assert ei.value.status == zk.ZK_ENONFINITE
    # the context is still usable
    s.set_state(e.astype(np.float32), p.astype(np.float32))
    H = s.energy()[0]
    assert np.isfinite(H) and H > 0
    s.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_ifab2_checkpoint_resume_is_bitwise(zk, prec):
    P = zk.ZK_F32 if prec == "f32" else zk.ZK_F64
    dt_np = np.float32 if prec == "f32" else np.float64
    e, p = _sea()
    e, p = e.astype(dt_np), p.astype(dt_np)

    def make():
        s = zk.Zakharov(64, 64, 100.0, 100.0, 20.0, M=3, precision=P, eps=0.8)
        zk.zk_set_options(s.ctx, eps=0.8, integrator=zk.ZK_IFAB2)
        return s

    ref = make()
    ref.set_state(e, p)
    ref.step(0.02, 7)
    ck = zk.zk_checkpoint_save(ref.ctx)
    ref.step(0.02, 9)
    want = ref.get_state()
    ref.close()

    res = make()
    zk.zk_checkpoint_load(res.ctx, ck)
    res.step(0.02, 9)
    got = res.get_state()
    res.close()
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])

    # resuming from the state alone restarts IF-AB2 with an IF-Euler step: not the same run
    alt = make()
    zk.zk_checkpoint_load(alt.ctx, ck)
    se, sp = alt.get_state(dtype=dt_np)
    alt.set_state(se, sp)
    alt.step(0.02, 9)
    other = alt.get_state()
    alt.close()
    d = np.linalg.norm(other[0] - want[0]) / np.linalg.norm(want[0])
    # far above the rounding of the state's round trip through physical space (~1e-7 in FP32)
    assert d > (1e-6 if prec == "f32" else 1e-9), d


def test_checkpoint_header_and_size_are_checked(zk):
    e, p = _sea()
    a = zk.Zakharov(64, 64, 100.0, 100.0, 20.0, M=3)
    a.set_state(e.astype(np.float32), p.astype(np.float32))
    ck = zk.zk_checkpoint_save(a.ctx)
    for kw in (dict(M=4), dict(precision=zk.ZK_F64)):
        b = zk.Zakharov(64, 64, 100.0, 100.0, 20.0, **dict(dict(M=3), **kw))
        with pytest.raises(zk.ZkError) as ei:
            zk.zk_checkpoint_load(b.ctx, ck)
        assert ei.value.status == zk.ZK_EINVAL
        b.close()
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_checkpoint_load(a.ctx, ck[:-8])
    assert ei.value.status == zk.ZK_EINVAL
    broken = bytearray(ck)
    broken[0] ^= 0xFF
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_checkpoint_load(a.ctx, bytes(broken))
    assert ei.value.status == zk.ZK_EINVAL
    # a fresh context without state cannot be checkpointed
    c = zk.Zakharov(64, 64, 100.0, 100.0, 20.0, M=3)
    with pytest.raises(zk.ZkError) as ei:
        zk.zk_checkpoint_save(c.ctx)
    assert ei.value.status == zk.ZK_ESTATE
    c.close()
    a.close()
