"""Write the oracle's reference run of the N = 4096 uniform-field workload to cfg2_oracle_run.npz.

Workload: N = 4096 electrons, Gaussian bunch with sigma = 10 um, gamma0 = 3 along +z, relative energy
spread 1e-3, transverse momentum spread 1e-4 u0 (seed 0); uniform external B = 5e-5 T along x;
dt = 1e-15 s; history depth D = 512 (the history window slides from step 512 on); 2000 steps.

Only the oracle (``oracle/``) and the seeded bunch sampler run here; no value comes from the CUDA
library. Stored:
  x_<k>, u_<k>      positions (m) and proper velocities (m/s) of all particles after k steps,
                    k in POS_STEPS;
  E_<k>, B_<k>      self fields (E) and the push's total B on TARGETS at state k (the fields the
                    step from k to k+1 uses), k in FIELD_STEPS;
  M_<k>             sum_j |E_ij| and sum_j |B_ij| of those targets (the error scale);
  t_<k>             the time stamp after k steps;
  targets           the sampled target indices;
  meta              the workload as a JSON string.

Run: ``python tests/golden/make_cfg2_golden.py`` (about 15-20 minutes on 8 cores).
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

N, SIGMA, GAMMA0, SEED = 4096, 10e-6, 3.0, 0
D, DT, STEPS = 512, 1e-15, 2000
B_UNIFORM = (5e-5, 0.0, 0.0)
POS_STEPS = (1, 100, 511, 512, 1000, 1500, 2000)
FIELD_STEPS = (0, 1, 511, 512, 1000, 1999)
NTARGETS = 256
OUT = os.path.join(HERE, "cfg2_oracle_run.npz")


def sampled_targets():
    rng = np.random.default_rng(20260)
    rest = rng.choice(np.arange(1, N - 1), NTARGETS - 2, replace=False)
    return np.sort(np.concatenate([[0, N - 1], rest])).astype(np.int64)


def main():
    b = inputs.gaussian_bunch(N, SIGMA, GAMMA0, seed=SEED)
    par = oracle.bext_params(1, b=B_UNIFORM)
    tg = sampled_targets()
    run = oracle.Run(b.x, b.u, D, DT, nmax=STEPS)
    out = dict(targets=tg)
    t0 = time.time()
    for k in range(STEPS):
        run.step(1, bkind=1, bpar=par)
        if k in FIELD_STEPS:
            # run.E / run.B are the fields the step from k used; the error scale needs sum_j |F_ij|
            _, _, _, M = oracle.self_fields(run.T, run.W, run.V, k, D, targets=tg, mags=True)
            out[f"E_{k}"] = run.E[tg].copy()
            out[f"B_{k}"] = run.B[tg].copy()
            out[f"M_{k}"] = M
        if run.n in POS_STEPS:
            out[f"x_{run.n}"] = run.x.copy()
            out[f"u_{run.n}"] = run.u.copy()
            out[f"t_{run.n}"] = np.array([run.t])
        if run.n % 100 == 0:
            print(f"step {run.n}  {time.time() - t0:.0f} s", flush=True)
    meta = dict(N=N, sigma=SIGMA, gamma0=GAMMA0, seed=SEED, D=D, dt=DT, steps=STEPS, B=list(B_UNIFORM),
                pos_steps=list(POS_STEPS), field_steps=list(FIELD_STEPS), oracle_threads=oracle.num_threads(),
                seconds=round(time.time() - t0, 1))
    out["meta"] = np.array(json.dumps(meta))
    np.savez_compressed(OUT, **out)
    print(f"wrote {OUT}", flush=True)


if __name__ == "__main__":
    main()
