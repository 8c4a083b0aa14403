"""Config 3 (the 2048^2 sea workload: L = 1600 m, h = 50 m, M = 5, eps = 0.5, JONSWAP Hs 4 m,
Tp 12 s, seed 3) over 20 RK4 steps, every precision form against the FP64 oracle.

The expected values are the oracle's own run of the same case (FP64 numpy, 20 RK4 steps from the
FP32-rounded initial state), stored on every 8th grid point of each axis by
tests/golden/make_oracle_runs.py (it imports only the oracle and the sea generator), together with
the full-grid L2 norms of eta and psi and the Hamiltonian at both ends. The GPU end state is
compared on the same sample points:
  * relative L2 over the sample, scaled to the full field: |e_sample| / |o_sample|;
  * relative max-norm over the sample: max|e| / max|o|.
Bars: FP32 rounding accumulates at most linearly, 2^-24 per step and transform chain with a
factor 4 of headroom (the stepped-run bar of the other FP32 tests): 4 n 2^-24. The FP64 series
sums leave the transforms in FP32, so they share that bar. The split DFT-GEMM stages add their own
rounding, bounded per product by u^2 of the 16-bit format (BF16: 128 times, FP16: 8 times the FP32
unit roundoff, pinned by test_split_roundoff.py): 4 n (ratio + 1) 2^-24. The max-norm bars are four
times the L2 bars. Each form's errors are printed, so the table of results can be restated.
"""
import os

import numpy as np
import pytest

from paper_2608_25203_b300 import seas

pytestmark = pytest.mark.gpu

N, L, H, M, EPS, DT = 2048, 1600.0, 50.0, 5, 0.5, 0.02
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config3_rk4_20_sub8.npz")


@pytest.fixture(scope="module")
def zk():
    import torch  # noqa: F401
    from paper_2608_25203_b300 import zk as _zk
    _zk.load()
    return _zk


@pytest.fixture(scope="module")
def golden():
    d = np.load(GOLDEN)
    return {k: d[k] for k in d.files}


@pytest.fixture(scope="module")
def initial():
    e, p, _ = seas.jonswap_sea(N, N, L, L, H, 4.0, 12.0, 3)
    return e.astype(np.float32), p.astype(np.float32)


FORMS = {"fp32": 1.0, "fp32_series64": 1.0, "bf16x3": 129.0, "fp16x3": 9.0}


@pytest.mark.parametrize("form", list(FORMS))
def test_config3_20_steps_against_oracle(zk, golden, initial, form):
    steps, sub = int(golden["steps"]), int(golden["sub"])
    s = zk.Zakharov(N, N, L, L, H, M=M, eps=EPS)
    if form == "fp32_series64":
        zk.zk_set_series_fp64(s.ctx, True)
    elif form == "bf16x3":
        zk.zk_set_dft_precision(s.ctx, zk.ZK_DFT_BF16X3)
    elif form == "fp16x3":
        zk.zk_set_dft_precision(s.ctx, zk.ZK_DFT_FP16X3)
    s.set_state(*initial)
    H0 = s.energy()[0]
    s.step(DT, steps)
    ge, gp = s.get_state()
    H1 = s.energy()[0]
    s.close()
    oe, op = golden["eta"], golden["psi"]
    ge, gp = ge[::sub, ::sub], gp[::sub, ::sub]
    errs = {
        "eta_l2": float(np.linalg.norm(ge - oe) / np.linalg.norm(oe)),
        "psi_l2": float(np.linalg.norm(gp - op) / np.linalg.norm(op)),
        "eta_max": float(np.max(np.abs(ge - oe)) / np.max(np.abs(oe))),
        "psi_max": float(np.max(np.abs(gp - op)) / np.max(np.abs(op))),
        "H0": abs(H0 - float(golden["H0"])) / float(golden["H0"]),
        "H1": abs(H1 - float(golden["H1"])) / float(golden["H1"]),
    }
    bar = 4 * steps * FORMS[form] * 2.0 ** -24
    print(f"config 3 {form} vs oracle after {steps} steps: " + " ".join(f"{k} {v:.3e}" for k, v in errs.items())
          + f" (bar {bar:.3e})")
    assert errs["eta_l2"] < bar and errs["psi_l2"] < bar, (errs, bar)
    assert errs["eta_max"] < 4 * bar and errs["psi_max"] < 4 * bar, (errs, bar)
    # the Hamiltonian (FP64 reduction of the FP32 state) at both ends
    assert errs["H0"] < 1e-6 and errs["H1"] < 1e-6 + bar, errs
