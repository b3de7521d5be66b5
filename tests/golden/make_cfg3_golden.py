"""Write the oracle's first two steps of the N = 65536 free-expansion workload to cfg3_oracle_start.npz.

Workload: N = 65536 electrons, Gaussian bunch with sigma = 20 um, gamma0 = 3 along +z, relative energy
spread 1e-3, transverse momentum spread 1e-4 u0 (seed 0); no external field; dt = 1e-15 s; history depth
1024. A full 500-step oracle run of 65536 particles is out of reach of a host (about 2e12 pair
evaluations), so the oracle's reference is its first full step (all 65536 targets) and, from the state it
reaches, the fields and push of sampled targets:
  E_0, B_0, M_0     self fields (and sum_j |F_ij|) of TARGETS at step 0 (the fields of the step 0 -> 1);
  x_1, u_1          positions and proper velocities of TARGETS after one step;
  E_1, B_1, M_1     self fields of TARGETS at step 1;
  x_2, u_2          positions and proper velocities of TARGETS after two steps (their push with E_1, B_1);
  targets, meta.

Only the oracle and the seeded bunch sampler run here; no value comes from the CUDA library.
Run: ``python tests/golden/make_cfg3_golden.py`` (about 5-10 minutes on 8 cores).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2605_05543_gb300 import inputs  # noqa: E402

N, SIGMA, GAMMA0, SEED = 65536, 20e-6, 3.0, 0
D, DT = 1024, 1e-15
NTARGETS = 64
OUT = os.path.join(HERE, "cfg3_oracle_start.npz")


def sampled_targets():
    rng = np.random.default_rng(3)
    return np.sort(np.concatenate([[0, N - 1], rng.choice(np.arange(1, N - 1), NTARGETS - 2, replace=False)]))


def main():
    b = inputs.gaussian_bunch(N, SIGMA, GAMMA0, seed=SEED)
    tg = sampled_targets()
    t0 = time.time()
    run = oracle.Run(b.x, b.u, D, DT, nmax=1)
    _, _, _, M0 = oracle.self_fields(run.T, run.W, run.V, 0, D, targets=tg, mags=True)
    run.step(1)  # all targets: the state at step 1
    out = dict(targets=tg.astype(np.int64), E_0=run.E[tg].copy(), B_0=run.B[tg].copy(), M_0=M0,
               x_1=run.x[tg].copy(), u_1=run.u[tg].copy())
    print(f"step 1 after {time.time() - t0:.0f} s", flush=True)
    E1, B1, _, M1 = oracle.self_fields(run.T, run.W, run.V, 1, D, targets=tg, mags=True)
    x2, u2, _ = oracle.push(run.x[tg], run.u[tg], E1, B1, DT)
    out.update(E_1=E1, B_1=B1, M_1=M1, x_2=x2, u_2=u2)
    meta = dict(N=N, sigma=SIGMA, gamma0=GAMMA0, seed=SEED, D=D, dt=DT, oracle_threads=oracle.num_threads(),
                seconds=round(time.time() - t0, 1), sigma_rms_1=float(np.sqrt(np.mean(np.sum(
                    (run.x - run.x.mean(axis=0)) ** 2, axis=1)))))
    out["meta"] = np.array(json.dumps(meta))
    np.savez_compressed(OUT, **out)
    print(f"wrote {OUT}", flush=True)


if __name__ == "__main__":
    main()
