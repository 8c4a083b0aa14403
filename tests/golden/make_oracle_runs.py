"""Write the oracle runs that the GPU parity tests of configs 2 and 3 compare against.

Only the FP64 oracle (``oracle/``) and the seeded sea generator are used; nothing here calls the
CUDA path. Run from the repository root:

    python tests/golden/make_oracle_runs.py [config2] [config3]

config2: 512^2, L = 400 m, h = 30 m, M = 5, eps = 1, JONSWAP Hs 3 m, Tp 10 s, seed 2, classical
    RK4 at dt = 0.02 s with the Eq. 17 filter, 1000 steps, from the FP32-rounded initial state.
    Also the twin run from that state perturbed by 1e-7 (relative, seeded direction), whose
    end-state difference gives the amplification A of the tolerance rule
    tol = max(1e-4, 10 A 6e-8 sqrt(steps)). Stored: final eta, psi (float64), H at the start and
    the end, A.
config3: the 2048^2 sea workload (L = 1600 m, h = 50 m, M = 5, eps = 0.5, Hs 4 m, Tp 12 s,
    seed 3), RK4 at dt = 0.02 s, 20 steps, from the FP32-rounded state. Stored: eta, psi after
    20 steps on every 8th grid point of each axis (float64), their full-grid L2 norms, and H.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import Grid, Oracle  # noqa: E402
from paper_2608_25203_b300 import seas  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def oracle_run(gr, M, eps, eta, psi, dt, steps, log=""):
    o = Oracle(gr, M, eps=eps)
    eh, ph = o.spectrum(eta), o.spectrum(psi)
    H0 = o.energy(eh, ph)[0]
    t = time.time()
    for n in range(steps):
        eh, ph = o.step_rk4(eh, ph, dt)
        if (n + 1) % 100 == 0:
            print(f"{log} step {n + 1} ({time.time() - t:.0f} s)", flush=True)
    H1 = o.energy(eh, ph)[0]
    return o.physical(eh), o.physical(ph), H0, H1


def twin_perturbation(e64, p64):
    rng = np.random.default_rng(2)
    de, dp = rng.standard_normal(e64.shape), rng.standard_normal(p64.shape)
    de *= 1e-7 * np.linalg.norm(e64) / np.linalg.norm(de)
    dp *= 1e-7 * np.linalg.norm(p64) / np.linalg.norm(dp)
    return de, dp


def config2():
    N, L, h, M, eps, dt, steps = 512, 400.0, 30.0, 5, 1.0, 0.02, 1000
    e, p, _ = seas.jonswap_sea(N, N, L, L, h, 3.0, 10.0, 2)
    e64 = e.astype(np.float32).astype(np.float64)
    p64 = p.astype(np.float32).astype(np.float64)
    gr = Grid(N, N, L, L, h)
    fe, fp, H0, H1 = oracle_run(gr, M, eps, e64, p64, dt, steps, "config2")
    de, dp = twin_perturbation(e64, p64)
    te, tp, _, _ = oracle_run(gr, M, eps, e64 + de, p64 + dp, dt, steps, "config2 twin")
    A = max(np.linalg.norm(te - fe) / np.linalg.norm(fe), np.linalg.norm(tp - fp) / np.linalg.norm(fp)) / 1e-7
    np.savez_compressed(os.path.join(HERE, "config2_rk4_1000.npz"), eta=fe, psi=fp, H0=H0, H1=H1, A=A,
                        steps=steps)
    print(f"config2: H0 {H0:.12e} H1 {H1:.12e} A {A:.4g}")


def config3():
    N, L, h, M, eps, dt, steps, sub = 2048, 1600.0, 50.0, 5, 0.5, 0.02, 20, 8
    e, p, _ = seas.jonswap_sea(N, N, L, L, h, 4.0, 12.0, 3)
    e64 = e.astype(np.float32).astype(np.float64)
    p64 = p.astype(np.float32).astype(np.float64)
    fe, fp, H0, H1 = oracle_run(Grid(N, N, L, L, h), M, eps, e64, p64, dt, steps, "config3")
    np.savez_compressed(os.path.join(HERE, "config3_rk4_20_sub8.npz"), eta=fe[::sub, ::sub], psi=fp[::sub, ::sub],
                        eta_norm=np.linalg.norm(fe), psi_norm=np.linalg.norm(fp), H0=H0, H1=H1, steps=steps,
                        sub=sub)
    print(f"config3: H0 {H0:.12e} H1 {H1:.12e}")


if __name__ == "__main__":
    which = sys.argv[1:] or ["config2", "config3"]
    for w in which:
        {"config2": config2, "config3": config3}[w]()
