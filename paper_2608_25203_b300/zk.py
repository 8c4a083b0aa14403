"""Python binding of the zk C ABI (include/zk.h): argument marshalling only.

Every function named ``zk_*`` here forwards to the C entry point of the same
name in ``libzk.so``; ``Zakharov`` wraps a context for convenience. Arrays can
be numpy arrays (host memory) or torch CUDA tensors (device memory, passed by
pointer on the caller's current stream). The library must have been built for
sm_103a; importing works without a GPU, but every call fails loudly if the
shared library is missing - there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libzk.so")

ZK_OK, ZK_EINVAL, ZK_ENOMEM, ZK_ECUDA, ZK_ENONFINITE, ZK_ETIMEOUT, ZK_EUNSUPPORTED, ZK_ESTATE = range(8)
ZK_F32, ZK_F64 = 0, 1
ZK_RK4, ZK_IFRK4, ZK_IFAB2 = 0, 1, 2
ZK_PAD_3_2, ZK_PAD_3 = 0, 1
ZK_DFT_F32, ZK_DFT_BF16X3, ZK_DFT_FP16X3 = 0, 1, 2

# every symbol include/zk.h declares
EXPORTS = [
    "zk_create", "zk_create_ex", "zk_set_state_async", "zk_get_state_async", "zk_io_join",
    "zk_checkpoint_size", "zk_checkpoint_save", "zk_checkpoint_load", "zk_destroy", "zk_set_options", "zk_get_options", "zk_set_state", "zk_get_state",
    "zk_rhs", "zk_dno", "zk_step", "zk_energy", "zk_sync", "zk_device_bytes",
    "zk_launches_per_step", "zk_profile_step", "zk_dno_static", "zk_dno_inverse", "zk_relax",
    "zk_set_state_tank", "zk_get_state_tank", "zk_set_series_fp64", "zk_set_dft_precision",
    "zk_set_adaptive_order",
    "zk_adaptive_status",
    "zk_batch_create", "zk_batch_destroy", "zk_batch_set_options", "zk_batch_set_state", "zk_batch_get_state",
    "zk_batch_energy", "zk_batch_step", "zk_batch_sync", "zk_batch_info", "zk_batch_group", "zk_batch_set_shape",
    "zk_batch_autotune",
    "zk_net_create", "zk_net_destroy", "zk_net_param_count", "zk_net_set_params", "zk_net_get_params",
    "zk_net_forward", "zk_net_backward", "zk_net_adam", "zk_net_train_step", "zk_net_set_inference",
    "zk_net_channel_rms", "zk_net_scale_channels",
    "zk_net_predict",
    "zk_closure_features", "zk_closure_set", "zk_closure_set_once_per_step", "zk_closure_status",
    "zk_strerror", "zk_version",
]

ZK_K_COL_STATE, ZK_K_ROW_ROUND, ZK_K_COL_PHI, ZK_K_ROW_FINAL, ZK_K_COL_FINAL = range(5)
ZK_MAX_ORDER = 8
KERNEL_CLASSES = {ZK_K_COL_STATE: "col_state", ZK_K_ROW_ROUND: "row_round", ZK_K_COL_PHI: "col_phi",
                  ZK_K_ROW_FINAL: "row_final", ZK_K_COL_FINAL: "col_final"}


class ZkOptions(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("integrator", ctypes.c_int), ("taper", ctypes.c_int),
                ("filter", ctypes.c_int), ("stream", ctypes.c_void_p)]


class ZkError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn} failed: {msg} (status {status})")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libzk.so (once). Raises if it is missing: the path has no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libzk.so not built at {path}; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    pd = ctypes.POINTER(ctypes.c_double)
    sig = {
        "zk_create": ([ctypes.POINTER(vp), i, i, d, d, d, d, i, i], i),
        "zk_create_ex": ([ctypes.POINTER(vp), i, i, d, d, d, d, i, i, i], i),
        "zk_set_state_async": ([vp, vp, vp, i], i),
        "zk_get_state_async": ([vp, vp, vp, i], i),
        "zk_io_join": ([vp], i),
        "zk_checkpoint_size": ([vp, ctypes.POINTER(ctypes.c_size_t)], i),
        "zk_checkpoint_save": ([vp, vp, ctypes.c_size_t], i),
        "zk_checkpoint_load": ([vp, vp, ctypes.c_size_t], i),
        "zk_destroy": ([vp], None),
        "zk_set_options": ([vp, ctypes.POINTER(ZkOptions)], i),
        "zk_get_options": ([vp, ctypes.POINTER(ZkOptions)], i),
        "zk_set_state": ([vp, vp, vp, i, i], i),
        "zk_get_state": ([vp, vp, vp, i, i], i),
        "zk_rhs": ([vp, vp, vp, i, i], i),
        "zk_dno": ([vp, vp, i, i], i),
        "zk_step": ([vp, d, i], i),
        "zk_energy": ([vp, pd, pd, pd, pd], i),
        "zk_sync": ([vp], i),
        "zk_device_bytes": ([vp, ctypes.POINTER(ctypes.c_size_t)], i),
        "zk_launches_per_step": ([vp, ctypes.POINTER(i)], i),
        "zk_profile_step": ([vp, d, i, pd, ctypes.POINTER(i), pd, i, ctypes.POINTER(i)], i),
        "zk_dno_static": ([vp, vp, vp, i, i, d, d, d, d, i, d, i, vp], i),
        "zk_dno_inverse": ([vp, vp, i, i, i], i),
        "zk_set_state_tank": ([vp, vp, vp, i, i], i),
        "zk_get_state_tank": ([vp, vp, vp, i, i], i),
        "zk_relax": ([vp, vp, vp, i, i, d, i], i),
        "zk_set_series_fp64": ([vp, i], i),
        "zk_set_dft_precision": ([vp, i], i),
        "zk_set_adaptive_order": ([vp, i, d, i], i),
        "zk_adaptive_status": ([vp, ctypes.POINTER(i), ctypes.POINTER(i), pd], i),
        "zk_batch_create": ([ctypes.POINTER(vp), i, ctypes.POINTER(i), ctypes.POINTER(i), pd, pd, pd, d,
                             ctypes.POINTER(i), i], i),
        "zk_batch_destroy": ([vp], None),
        "zk_batch_set_options": ([vp, ctypes.POINTER(ZkOptions)], i),
        "zk_batch_set_state": ([vp, i, vp, vp, i, i], i),
        "zk_batch_get_state": ([vp, i, vp, vp, i, i], i),
        "zk_batch_energy": ([vp, i, pd, pd, pd, pd], i),
        "zk_batch_step": ([vp, d, i], i),
        "zk_batch_sync": ([vp], i),
        "zk_batch_info": ([vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_size_t)], i),
        "zk_batch_group": ([vp, i] + [ctypes.POINTER(i)] * 7, i),
        "zk_batch_set_shape": ([vp, i, i, i, i], i),
        "zk_batch_autotune": ([vp, d, ctypes.c_char_p, ctypes.POINTER(i), ctypes.POINTER(i)], i),
        "zk_net_create": ([ctypes.POINTER(vp), i, i, i], i),
        "zk_net_destroy": ([vp], None),
        "zk_net_param_count": ([vp, ctypes.POINTER(i)], i),
        "zk_net_set_params": ([vp, vp, i], i),
        "zk_net_get_params": ([vp, vp, i], i),
        "zk_net_forward": ([vp, vp, vp, i, i, i, vp], i),
        "zk_net_backward": ([vp, vp, vp, vp, vp], i),
        "zk_net_adam": ([vp, vp, d, vp], i),
        "zk_net_train_step": ([vp, vp, vp, i, i, i, d, pd, vp], i),
        "zk_net_channel_rms": ([vp, ctypes.c_longlong, i, i, vp, vp], i),
        "zk_net_scale_channels": ([vp, ctypes.c_longlong, i, i, vp, vp], i),
        "zk_net_set_inference": ([vp, i], i),
        "zk_net_predict": ([vp, vp, vp, i, i, vp], i),
        "zk_closure_features": ([vp, i, vp, vp, vp, vp], i),
        "zk_closure_set": ([vp, vp, i, vp, vp, i, d], i),
        "zk_closure_set_once_per_step": ([vp, i], i),
        "zk_closure_status": ([vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong), pd], i),
        "zk_strerror": ([i], ctypes.c_char_p),
        "zk_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(fn: str, st: int):
    if st != ZK_OK:
        raise ZkError(fn, st, load().zk_strerror(st).decode())


def _ptr(x, dtype_code):
    """(pointer, on_device) for a numpy array or a torch tensor of the expected dtype."""
    if isinstance(x, np.ndarray):
        want = np.float32 if dtype_code == ZK_F32 else np.float64
        if x.dtype != want or not x.flags["C_CONTIGUOUS"]:
            raise ValueError(f"expected C-contiguous {want.__name__} array")
        return x.ctypes.data, 0
    import torch
    if isinstance(x, torch.Tensor):
        want = torch.float32 if dtype_code == ZK_F32 else torch.float64
        if x.dtype != want or not x.is_contiguous():
            raise ValueError(f"expected contiguous {want} tensor")
        return x.data_ptr(), 1 if x.is_cuda else 0
    raise TypeError("expected numpy array or torch tensor")


# ---- thin wrappers with the C names -----------------------------------------
def zk_create(nx, nz, Lx, Lz, h, g, M, precision=ZK_F32):
    c = ctypes.c_void_p()
    _check("zk_create", load().zk_create(ctypes.byref(c), nx, nz, Lx, Lz, h, g, M, precision))
    return c


def zk_create_ex(nx, nz, Lx, Lz, h, g, M, precision=ZK_F32, pad=ZK_PAD_3_2):
    c = ctypes.c_void_p()
    _check("zk_create_ex", load().zk_create_ex(ctypes.byref(c), nx, nz, Lx, Lz, h, g, M, precision, pad))
    return c


def zk_destroy(ctx):
    load().zk_destroy(ctx)


def zk_set_options(ctx, eps=1.0, integrator=ZK_RK4, taper=1, filter=1, stream=None):
    o = ZkOptions(eps, integrator, taper, filter, stream)
    _check("zk_set_options", load().zk_set_options(ctx, ctypes.byref(o)))


def zk_get_options(ctx):
    o = ZkOptions()
    _check("zk_get_options", load().zk_get_options(ctx, ctypes.byref(o)))
    return o


def zk_set_state(ctx, eta, psi, dtype=None):
    dt = dtype if dtype is not None else _dtype_of(eta)
    pe, de = _ptr(eta, dt)
    pp, dp = _ptr(psi, dt)
    if de != dp:
        raise ValueError("eta and psi must both be host or both device arrays")
    _check("zk_set_state", load().zk_set_state(ctx, pe, pp, dt, de))


def zk_get_state(ctx, eta, psi, dtype=None):
    dt = dtype if dtype is not None else _dtype_of(eta)
    pe, de = _ptr(eta, dt)
    pp, _ = _ptr(psi, dt)
    _check("zk_get_state", load().zk_get_state(ctx, pe, pp, dt, de))


def zk_rhs(ctx, deta, dpsi, dtype=None):
    dt = dtype if dtype is not None else _dtype_of(deta)
    pe, de = _ptr(deta, dt)
    pp, _ = _ptr(dpsi, dt)
    _check("zk_rhs", load().zk_rhs(ctx, pe, pp, dt, de))


def zk_dno(ctx, v, dtype=None):
    dt = dtype if dtype is not None else _dtype_of(v)
    pv, dv = _ptr(v, dt)
    _check("zk_dno", load().zk_dno(ctx, pv, dt, dv))


def zk_step(ctx, dt, n=1):
    _check("zk_step", load().zk_step(ctx, float(dt), int(n)))


def zk_energy(ctx):
    H, k, p, m = (ctypes.c_double() for _ in range(4))
    _check("zk_energy", load().zk_energy(ctx, ctypes.byref(H), ctypes.byref(k), ctypes.byref(p), ctypes.byref(m)))
    return H.value, k.value, p.value, m.value


def zk_sync(ctx):
    _check("zk_sync", load().zk_sync(ctx))


def zk_device_bytes(ctx):
    b = ctypes.c_size_t()
    _check("zk_device_bytes", load().zk_device_bytes(ctx, ctypes.byref(b)))
    return b.value


def zk_checkpoint_save(ctx):
    """Checkpoint of the context (state spectra and IF-AB2 history) as host bytes."""
    n = ctypes.c_size_t()
    _check("zk_checkpoint_size", load().zk_checkpoint_size(ctx, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check("zk_checkpoint_save", load().zk_checkpoint_save(ctx, buf, n.value))
    return buf.raw


def zk_checkpoint_load(ctx, data):
    """Restore a checkpoint written by zk_checkpoint_save into a context of the same shape."""
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    _check("zk_checkpoint_load", load().zk_checkpoint_load(ctx, buf, len(data)))


def zk_launches_per_step(ctx):
    n = ctypes.c_int()
    _check("zk_launches_per_step", load().zk_launches_per_step(ctx, ctypes.byref(n)))
    return n.value


def zk_profile_step(ctx, dt, nsteps=1, cap=256):
    """Per-launch device times (ms, summed over nsteps), kernel classes and algorithmic bytes."""
    ms = (ctypes.c_double * cap)()
    kind = (ctypes.c_int * cap)()
    by = (ctypes.c_double * cap)()
    n = ctypes.c_int()
    _check("zk_profile_step", load().zk_profile_step(ctx, float(dt), int(nsteps), ms, kind, by, cap,
                                                     ctypes.byref(n)))
    k = n.value
    return list(ms[:k]), [KERNEL_CLASSES[x] for x in kind[:k]], list(by[:k])


def zk_set_state_async(ctx, eta, psi, dtype=None):
    """Upload from pinned host arrays (torch pinned tensors or numpy arrays) without waiting."""
    dt = dtype if dtype is not None else _dtype_of(eta)
    pe, de = _ptr(eta, dt)
    pp, dp = _ptr(psi, dt)
    if de or dp:
        raise ValueError("host arrays expected")
    _check("zk_set_state_async", load().zk_set_state_async(ctx, pe, pp, dt))


def zk_get_state_async(ctx, eta, psi, dtype=None):
    """Download into pinned host arrays without waiting (valid after zk_sync)."""
    dt = dtype if dtype is not None else _dtype_of(eta)
    pe, de = _ptr(eta, dt)
    pp, dp = _ptr(psi, dt)
    if de or dp:
        raise ValueError("host arrays expected")
    _check("zk_get_state_async", load().zk_get_state_async(ctx, pe, pp, dt))


def zk_io_join(ctx):
    _check("zk_io_join", load().zk_io_join(ctx))


def zk_set_state_tank(ctx, eta, psi, dtype=None):
    dt = dtype if dtype is not None else _dtype_of(eta)
    pe, de = _ptr(eta, dt)
    pp, dp = _ptr(psi, dt)
    if de != dp:
        raise ValueError("eta and psi must both be host or both device arrays")
    _check("zk_set_state_tank", load().zk_set_state_tank(ctx, pe, pp, dt, de))


def zk_get_state_tank(ctx, eta, psi, dtype=None):
    dt = dtype if dtype is not None else _dtype_of(eta)
    pe, de = _ptr(eta, dt)
    pp, _ = _ptr(psi, dt)
    _check("zk_get_state_tank", load().zk_get_state_tank(ctx, pe, pp, dt, de))


def zk_set_series_fp64(ctx, on=True):
    _check("zk_set_series_fp64", load().zk_set_series_fp64(ctx, 1 if on else 0))


def zk_set_dft_precision(ctx, mode):
    _check("zk_set_dft_precision", load().zk_set_dft_precision(ctx, int(mode)))


def zk_set_adaptive_order(ctx, m_min, tol, check_every):
    _check("zk_set_adaptive_order", load().zk_set_adaptive_order(ctx, int(m_min), float(tol), int(check_every)))


def zk_adaptive_status(ctx):
    o, c = ctypes.c_int(), ctypes.c_int()
    err = (ctypes.c_double * 8)()
    _check("zk_adaptive_status", load().zk_adaptive_status(ctx, ctypes.byref(o), ctypes.byref(c), err))
    return dict(order=o.value, checks=c.value, err=[err[m] for m in range(8)])


def zk_dno_inverse(ctx, v, iters=8, dtype=None):
    dt = dtype if dtype is not None else _dtype_of(v)
    pv, dv = _ptr(v, dt)
    _check("zk_dno_inverse", load().zk_dno_inverse(ctx, pv, dt, dv, int(iters)))


def zk_relax(ctx, sigma, eta_target, dt, iters=8, dtype=None):
    d = dtype if dtype is not None else _dtype_of(sigma)
    ps, ds = _ptr(sigma, d)
    pt, dtg = _ptr(eta_target, d)
    if ds != dtg:
        raise ValueError("sigma and eta_target must both be host or both device arrays")
    _check("zk_relax", load().zk_relax(ctx, ps, pt, d, ds, float(dt), int(iters)))


def zk_dno_static(eta, psi, v, Lx, Lz, h, g=9.81, M=5, eps=1.0, taper=1, stream=None):
    """G(eta) psi into v with no device allocation (scratch is a fixed array in the library).

    eta, psi, v: contiguous float32 CUDA tensors [nz][nx]. Queued on `stream`
    (a cudaStream_t handle, None = legacy default); returns without waiting.
    """
    nz, nx = eta.shape
    for t in (eta, psi, v):
        pt, dev = _ptr(t, ZK_F32)
        if not dev:
            raise ValueError("zk_dno_static takes device tensors")
    _check("zk_dno_static", load().zk_dno_static(eta.data_ptr(), psi.data_ptr(), v.data_ptr(), nx, nz,
                                                 float(Lx), float(Lz), float(h), float(g), int(M), float(eps),
                                                 int(taper), stream))


def zk_version():
    return load().zk_version().decode()


def _dtype_of(x):
    if isinstance(x, np.ndarray):
        return ZK_F64 if x.dtype == np.float64 else ZK_F32
    import torch
    return ZK_F64 if x.dtype == torch.float64 else ZK_F32


class Zakharov:
    """One simulation context on the current CUDA device."""

    def __init__(self, nx, nz, Lx, Lz, h, g=9.81, M=5, precision=ZK_F32, eps=1.0, taper=True,
                 filter=True, stream=None, pad=ZK_PAD_3_2):
        self.nx, self.nz, self.M, self.precision = nx, nz, M, precision
        self.ctx = zk_create_ex(nx, nz, Lx, Lz, h, g, M, precision, pad)
        self._stream = stream
        zk_set_options(self.ctx, eps=eps, taper=int(taper), filter=int(filter), stream=stream)

    def close(self):
        if self.ctx is not None:
            zk_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, eta, psi):
        if isinstance(eta, np.ndarray):
            eta = np.ascontiguousarray(eta)
            psi = np.ascontiguousarray(psi, dtype=eta.dtype)
        zk_set_state(self.ctx, eta, psi)

    def get_state(self, dtype=np.float64):
        e = np.empty((self.nz, self.nx), dtype)
        p = np.empty((self.nz, self.nx), dtype)
        zk_get_state(self.ctx, e, p)
        return e, p

    def rhs(self, dtype=np.float64):
        e = np.empty((self.nz, self.nx), dtype)
        p = np.empty((self.nz, self.nx), dtype)
        zk_rhs(self.ctx, e, p)
        return e, p

    def dno(self, dtype=np.float64):
        v = np.empty((self.nz, self.nx), dtype)
        zk_dno(self.ctx, v)
        return v

    def step(self, dt, n=1):
        zk_step(self.ctx, dt, n)

    def dno_inverse(self, v, iters=8):
        zk_dno_inverse(self.ctx, np.ascontiguousarray(v) if isinstance(v, np.ndarray) else v, iters)

    def relax(self, sigma, eta_target, dt, iters=8):
        if isinstance(sigma, np.ndarray):
            sigma = np.ascontiguousarray(sigma)
            eta_target = np.ascontiguousarray(eta_target, dtype=sigma.dtype)
        zk_relax(self.ctx, sigma, eta_target, dt, iters)

    def energy(self):
        return zk_energy(self.ctx)

    def sync(self):
        zk_sync(self.ctx)


# ---- batched tiles ----------------------------------------------------------
def zk_batch_create(nx, nz, Lx, Lz, h, g, M, precision=ZK_F32):
    n = len(nx)
    if not all(len(v) == n for v in (nz, Lx, Lz, h, M)):
        raise ValueError("per-tile lists must have equal length")
    ia = lambda v: (ctypes.c_int * n)(*[int(x) for x in v])
    da = lambda v: (ctypes.c_double * n)(*[float(x) for x in v])
    b = ctypes.c_void_p()
    _check("zk_batch_create", load().zk_batch_create(ctypes.byref(b), n, ia(nx), ia(nz), da(Lx), da(Lz), da(h),
                                                     float(g), ia(M), precision))
    return b


def zk_batch_destroy(b):
    load().zk_batch_destroy(b)


def zk_batch_set_options(b, eps=1.0, integrator=ZK_RK4, taper=1, filter=1, stream=None):
    o = ZkOptions(eps, integrator, taper, filter, stream)
    _check("zk_batch_set_options", load().zk_batch_set_options(b, ctypes.byref(o)))


def zk_batch_set_state(b, tile, eta, psi, dtype=None):
    dt = dtype if dtype is not None else _dtype_of(eta)
    pe, de = _ptr(eta, dt)
    pp, dp = _ptr(psi, dt)
    if de != dp:
        raise ValueError("eta and psi must both be host or both device arrays")
    _check("zk_batch_set_state", load().zk_batch_set_state(b, int(tile), pe, pp, dt, de))


def zk_batch_get_state(b, tile, eta, psi, dtype=None):
    dt = dtype if dtype is not None else _dtype_of(eta)
    pe, de = _ptr(eta, dt)
    pp, _ = _ptr(psi, dt)
    _check("zk_batch_get_state", load().zk_batch_get_state(b, int(tile), pe, pp, dt, de))


def zk_batch_energy(b, tile):
    v = [ctypes.c_double() for _ in range(4)]
    _check("zk_batch_energy", load().zk_batch_energy(b, int(tile), *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def zk_batch_step(b, dt, n=1):
    _check("zk_batch_step", load().zk_batch_step(b, float(dt), int(n)))


def zk_batch_sync(b):
    _check("zk_batch_sync", load().zk_batch_sync(b))


def zk_batch_info(b):
    ng, nl, by = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
    _check("zk_batch_info", load().zk_batch_info(b, ctypes.byref(ng), ctypes.byref(nl), ctypes.byref(by)))
    return ng.value, nl.value, by.value


def zk_batch_group(b, gi):
    v = [ctypes.c_int() for _ in range(7)]
    _check("zk_batch_group", load().zk_batch_group(b, int(gi), *[ctypes.byref(x) for x in v]))
    return dict(zip(("nx", "nz", "M", "ntiles", "plan_v", "col_ci", "row_occ"), (x.value for x in v)))


def zk_batch_set_shape(b, gi, plan_v, col_ci, row_occ):
    _check("zk_batch_set_shape", load().zk_batch_set_shape(b, int(gi), int(plan_v), int(col_ci), int(row_occ)))


def zk_batch_autotune(b, dt, cache_path=None):
    t, c = ctypes.c_int(), ctypes.c_int()
    path = cache_path.encode() if cache_path else None
    _check("zk_batch_autotune", load().zk_batch_autotune(b, float(dt), path, ctypes.byref(t), ctypes.byref(c)))
    return t.value, c.value


class Batch:
    """Many independent tiles advanced together (one graph, one launch per pass of each group)."""

    def __init__(self, tiles, g=9.81, precision=ZK_F32, eps=1.0, integrator=ZK_RK4, stream=None):
        """tiles: list of dicts with nx, nz, Lx, Lz, h, M."""
        self.tiles = [dict(t) for t in tiles]
        col = lambda k: [t[k] for t in self.tiles]
        self.b = zk_batch_create(col("nx"), col("nz"), col("Lx"), col("Lz"), col("h"), g, col("M"), precision)
        self.precision = precision
        zk_batch_set_options(self.b, eps=eps, integrator=integrator, stream=stream)

    def close(self):
        if self.b is not None:
            zk_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, tile, eta, psi):
        if isinstance(eta, np.ndarray):
            eta = np.ascontiguousarray(eta)
            psi = np.ascontiguousarray(psi, dtype=eta.dtype)
        zk_batch_set_state(self.b, tile, eta, psi)

    def get_state(self, tile, dtype=np.float64):
        t = self.tiles[tile]
        e = np.empty((t["nz"], t["nx"]), dtype)
        p = np.empty((t["nz"], t["nx"]), dtype)
        zk_batch_get_state(self.b, tile, e, p)
        return e, p

    def step(self, dt, n=1):
        zk_batch_step(self.b, dt, n)

    def sync(self):
        zk_batch_sync(self.b)

    def energy(self, tile):
        return zk_batch_energy(self.b, tile)

    def info(self):
        return zk_batch_info(self.b)

    def groups(self):
        return [zk_batch_group(self.b, gi) for gi in range(self.info()[0])]

    def set_shape(self, gi, plan_v, col_ci, row_occ):
        zk_batch_set_shape(self.b, gi, plan_v, col_ci, row_occ)

    def autotune(self, dt, cache_path=None):
        return zk_batch_autotune(self.b, dt, cache_path)


# ---- learned closure --------------------------------------------------------
def _dptr(t):
    """Device pointer of a contiguous float32 CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return t.data_ptr()


def _fvec(v, n):
    if v is None:
        return None
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float32).reshape(n))
    return a


def zk_net_create(cin=6, width=32, cout=2):
    n = ctypes.c_void_p()
    _check("zk_net_create", load().zk_net_create(ctypes.byref(n), cin, width, cout))
    return n


def zk_net_destroy(n):
    load().zk_net_destroy(n)


def zk_net_param_count(n):
    c = ctypes.c_int()
    _check("zk_net_param_count", load().zk_net_param_count(n, ctypes.byref(c)))
    return c.value


def zk_net_set_params(n, theta):
    if isinstance(theta, np.ndarray):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        _check("zk_net_set_params", load().zk_net_set_params(n, a.ctypes.data, 0))
    else:
        _check("zk_net_set_params", load().zk_net_set_params(n, _dptr(theta), 1))


def zk_net_get_params(n):
    a = np.empty(zk_net_param_count(n), np.float32)
    _check("zk_net_get_params", load().zk_net_get_params(n, a.ctypes.data, 0))
    return a


def zk_net_forward(n, x, y=None, stream=None):
    B, C, H, W = x.shape
    _check("zk_net_forward", load().zk_net_forward(n, _dptr(x), _dptr(y), B, H, W, stream))


def zk_net_backward(n, dy, grad=None, dx=None, stream=None):
    _check("zk_net_backward", load().zk_net_backward(n, _dptr(dy), _dptr(grad), _dptr(dx), stream))


def zk_net_adam(n, grad=None, lr=1e-3, stream=None):
    _check("zk_net_adam", load().zk_net_adam(n, _dptr(grad), float(lr), stream))


def zk_net_train_step(n, x, target, lr, stream=None, want_loss=True):
    B, C, H, W = x.shape
    loss = ctypes.c_double(float("nan"))
    _check("zk_net_train_step", load().zk_net_train_step(n, _dptr(x), _dptr(target), B, H, W, float(lr),
                                                         ctypes.byref(loss) if want_loss else None, stream))
    return loss.value


def zk_net_channel_rms(x, stream=None):
    """Per-channel RMS over samples and positions of a [n][c][h][w] float32 CUDA tensor (numpy float32 [c])."""
    n, c = x.shape[0], x.shape[1]
    hw = int(np.prod(x.shape[2:]))
    out = np.empty(c, np.float32)
    _check("zk_net_channel_rms", load().zk_net_channel_rms(_dptr(x), int(n), int(c), hw, out.ctypes.data, stream))
    return out


def zk_net_scale_channels(x, mul, stream=None):
    """x[:, ch] *= mul[ch] in place on a [n][c][h][w] float32 CUDA tensor."""
    n, c = x.shape[0], x.shape[1]
    hw = int(np.prod(x.shape[2:]))
    m = np.ascontiguousarray(mul, dtype=np.float32)
    if m.shape != (c,):
        raise ValueError("one factor per channel expected")
    _check("zk_net_scale_channels", load().zk_net_scale_channels(_dptr(x), int(n), int(c), hw, m.ctypes.data, stream))


def zk_net_set_inference(n, mode):
    _check("zk_net_set_inference", load().zk_net_set_inference(n, int(mode)))


def zk_net_predict(n, x, y, stream=None):
    C, H, W = x.shape[-3:]
    _check("zk_net_predict", load().zk_net_predict(n, _dptr(x), _dptr(y), H, W, stream))


def zk_closure_features(ctx, base_order, feat, target=None, in_scale=None, out_scale=None):
    a, b = _fvec(in_scale, 6), _fvec(out_scale, 2)
    _check("zk_closure_features", load().zk_closure_features(
        ctx, int(base_order), None if a is None else a.ctypes.data, None if b is None else b.ctypes.data,
        _dptr(feat), _dptr(target)))


def zk_closure_set(ctx, net, base_order=2, in_scale=None, out_scale=None, check_every=50, check_tol=0.2):
    a, b = _fvec(in_scale, 6), _fvec(out_scale, 2)
    _check("zk_closure_set", load().zk_closure_set(
        ctx, net, int(base_order), None if a is None else a.ctypes.data, None if b is None else b.ctypes.data,
        int(check_every), float(check_tol)))


def zk_closure_set_once_per_step(ctx, on):
    _check("zk_closure_set_once_per_step", load().zk_closure_set_once_per_step(ctx, int(on)))


def zk_closure_status(ctx):
    a, c, f, e = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong(), ctypes.c_double()
    _check("zk_closure_status", load().zk_closure_status(ctx, ctypes.byref(a), ctypes.byref(c), ctypes.byref(f),
                                                         ctypes.byref(e)))
    return dict(active=a.value, checks=c.value, fallback_step=f.value, last_err=e.value)


class Net:
    """The closure network (6 -> 32 -> 32 -> 32 -> 2 periodic conv net) on the current CUDA device."""

    def __init__(self, theta=None):
        self.n = zk_net_create()
        self.nparam = zk_net_param_count(self.n)
        if theta is not None:
            self.set_params(theta)

    def close(self):
        if self.n is not None:
            zk_net_destroy(self.n)
            self.n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        zk_net_set_params(self.n, theta)

    def params(self):
        return zk_net_get_params(self.n)

    def forward(self, x, y=None, stream=None):
        zk_net_forward(self.n, x, y, stream)

    def backward(self, dy, grad=None, dx=None, stream=None):
        zk_net_backward(self.n, dy, grad, dx, stream)

    def adam(self, grad=None, lr=1e-3, stream=None):
        zk_net_adam(self.n, grad, lr, stream)

    def train_step(self, x, target, lr, stream=None, want_loss=True):
        return zk_net_train_step(self.n, x, target, lr, stream, want_loss)

    def set_inference(self, mode):
        zk_net_set_inference(self.n, mode)

    def predict(self, x, y, stream=None):
        zk_net_predict(self.n, x, y, stream)
