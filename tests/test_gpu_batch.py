"""Batched tiles on the GPU: bitwise equality with one context per tile, every
launch shape against the default one, the autotuner and its cache."""
import json
import os

import numpy as np
import pytest

from oracle import Grid, Oracle, run
from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


def _tiles():
    # three groups: (64^2, M=3) x 3 tiles with different depths, (128^2, M=4) x 2, (256^2, M=5) x 1
    T = []
    for j, h in enumerate((12.0, 30.0, 80.0)):
        T.append(dict(nx=64, nz=64, Lx=50.0, Lz=50.0, h=h, M=3, Hs=0.8, Tp=5.0, seed=500 + j))
    for j, h in enumerate((20.0, 45.0)):
        T.append(dict(nx=128, nz=128, Lx=100.0, Lz=100.0, h=h, M=4, Hs=1.0, Tp=6.0, seed=510 + j))
    T.append(dict(nx=256, nz=256, Lx=200.0, Lz=200.0, h=60.0, M=5, Hs=1.2, Tp=7.0, seed=520))
    return T


def _fields(t):
    e, p, _ = seas.jonswap_sea(t["nx"], t["nz"], t["Lx"], t["Lz"], t["h"], t["Hs"], t["Tp"], t["seed"])
    return e.astype(np.float32), p.astype(np.float32)


@pytest.mark.parametrize("name", ["rk4", "ifab2", "ifrk4"])
def test_batch_bitwise_equals_single_contexts(zk, name):
    integrator = {"rk4": zk.ZK_RK4, "ifab2": zk.ZK_IFAB2, "ifrk4": zk.ZK_IFRK4}[name]
    T = _tiles()
    b = zk.Batch(T, eps=0.5, integrator=integrator)
    assert b.info()[0] == 3
    singles = []
    for i, t in enumerate(T):
        e, p = _fields(t)
        b.set_state(i, e, p)
        s = zk.Zakharov(t["nx"], t["nz"], t["Lx"], t["Lz"], t["h"], M=t["M"], eps=0.5)
        zk.zk_set_options(s.ctx, eps=0.5, integrator=integrator)
        s.set_state(e, p)
        singles.append(s)
    b.step(0.02, 7)
    for s in singles:
        s.step(0.02, 7)
    for i, s in enumerate(singles):
        be, bp = b.get_state(i, np.float32)
        se, sp = s.get_state(np.float32)
        assert np.array_equal(be, se) and np.array_equal(bp, sp), f"tile {i}"
        assert np.isfinite(be).all()
        Hb = b.energy(i)[0]
        Hs_ = s.energy()[0]
        assert Hb == Hs_


def test_batch_tile_matches_oracle(zk):
    # the smallest group against the FP64 oracle (per-tile depth read by the kernels)
    T = _tiles()
    b = zk.Batch(T, eps=0.5)
    for i, t in enumerate(T):
        b.set_state(i, *_fields(t))
    b.step(0.02, 5)
    for i in range(3):
        t = T[i]
        e, p = _fields(t)
        o = Oracle(Grid(t["nx"], t["nz"], t["Lx"], t["Lz"], t["h"]), t["M"], eps=0.5)
        oe, op = run(o, e.astype(np.float64), p.astype(np.float64), 0.02, 5)
        ge, gp = b.get_state(i)
        n = 5
        tol = 4 * n * 2.0 ** -24          # the stepped FP32 bar of the parity tests
        assert np.linalg.norm(ge - oe) / np.linalg.norm(oe) < tol
        assert np.linalg.norm(gp - op) / np.linalg.norm(op) < tol


@pytest.mark.parametrize("n", [512, 1024, 2048])
def test_launch_shapes_agree(zk, n):
    # every plan variant / columns-per-block / row occupancy gives the same step
    # within FP32 rounding of the default shape (which the parity tests pin):
    # two runs, each within the one-step bar 4 * 2^-24 of the exact step
    tol = 8 * 2.0 ** -24
    L = n * 0.78125
    t = dict(nx=n, nz=n, Lx=L, Lz=L, h=40.0, M=3)
    e, p, _ = seas.jonswap_sea(n, n, L, L, 40.0, 1.5, 8.0, 77)
    b = zk.Batch([t], eps=0.5)
    b.set_state(0, e.astype(np.float32), p.astype(np.float32))
    b.step(0.02, 1)
    ref = b.get_state(0)
    for v in (0, 1):
        for ci in (0, 1, 2):
            for occ in (0, 1):
                b.set_state(0, e.astype(np.float32), p.astype(np.float32))
                try:
                    b.set_shape(0, v, ci, occ)
                    b.step(0.02, 1)
                except zk.ZkError as err:
                    # only shapes that exceed the block limits may refuse to launch
                    assert err.status == zk.ZK_ECUDA and ci == 2
                    continue
                ge, gp = b.get_state(0)
                assert np.linalg.norm(ge - ref[0]) / np.linalg.norm(ref[0]) < tol, (v, ci, occ)
                assert np.linalg.norm(gp - ref[1]) / np.linalg.norm(ref[1]) < tol, (v, ci, occ)
    b.close()


def test_autotune_and_cache(zk, tmp_path):
    T = _tiles()
    b = zk.Batch(T, eps=0.5)
    for i, t in enumerate(T):
        b.set_state(i, *_fields(t))
    before = [b.get_state(i, np.float32) for i in range(len(T))]
    path = str(tmp_path / "tune.json")
    tuned, cached = b.autotune(0.02, path)
    assert (tuned, cached) == (3, 0)
    after = [b.get_state(i, np.float32) for i in range(len(T))]
    for (e0, p0), (e1, p1) in zip(before, after):   # timing steps leave the state as it was
        assert np.array_equal(e0, e1) and np.array_equal(p0, p1)
    d = json.load(open(path))
    assert len(d["entries"]) == 3
    shapes = [(g["plan_v"], g["col_ci"], g["row_occ"]) for g in b.groups()]
    b2 = zk.Batch(T, eps=0.5)
    for i, t in enumerate(T):
        b2.set_state(i, *_fields(t))
    assert b2.autotune(0.02, path) == (0, 3)
    assert [(g["plan_v"], g["col_ci"], g["row_occ"]) for g in b2.groups()] == shapes
    b.step(0.02, 3)
    b2.step(0.02, 3)
    for i in range(len(T)):
        assert np.array_equal(b.get_state(i, np.float32)[0], b2.get_state(i, np.float32)[0])


def test_batch_errors(zk):
    T = _tiles()[:2]
    b = zk.Batch(T)
    with pytest.raises(zk.ZkError) as ei:
        b.step(0.02, 1)
    assert ei.value.status == zk.ZK_ESTATE
    with pytest.raises(zk.ZkError) as ei:
        b.set_state(5, *_fields(T[0]))
    assert ei.value.status == zk.ZK_EINVAL
    with pytest.raises(zk.ZkError):
        zk.zk_batch_create([64], [64], [50.0], [50.0], [-1.0], 9.81, [3])
