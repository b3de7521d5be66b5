"""Shared helpers of the GPU tests: seeded inputs, oracle references and error metrics."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2605_05543_gb300 import inputs

DT = 1e-15


def history_case(N, n, sigma=10e-6, gamma0=3.0, seed=0, dt=DT, wiggle=1e-4, period_steps=160.0):
    b = inputs.gaussian_bunch(N, sigma, gamma0, seed=seed)
    return inputs.synthetic_history(b.x, b.u, n, dt, wiggle=wiggle, period_steps=period_steps, seed=seed + 100)


def window(h, D):
    """The most recent min(n+1, D) slots, as emppp_set_history takes them."""
    k0 = max(0, h.n - D + 1)
    return (np.ascontiguousarray(h.T[k0:]), np.ascontiguousarray(h.W[k0:]), np.ascontiguousarray(h.V[k0:]),
            np.ascontiguousarray(h.u))


def field_errors(E, B, E_ref, B_ref, M):
    """Per-component errors normalised by sum_j |E_ij| (resp. |B_ij|) of the target: (max_E, max_B)."""
    sE = np.maximum(M[:, 0:1], 1e-300)
    sB = np.maximum(M[:, 1:2], 1e-300)
    return float(np.max(np.abs(E - E_ref) / sE)), float(np.max(np.abs(B - B_ref) / sB))


def gpu_fields_from_history(Solver, h, D, dt=DT, **kw):
    """Fields and stats of one GPU step evaluated on history h (and the state after the step)."""
    T, W, V, u = window(h, D)
    with Solver(W.shape[1], D, dt, **kw) as s:
        s.set_history(h.n, T, W, V, u)
        s.step(1)
        E, B = s.get_fields()
        st = s.stats()
        x, uu, t, n = s.get_state()
    return E, B, st, x, uu


def oracle_step_from_history(h, D, dt=DT, bkind=0, bpar=None):
    run = oracle.Run(None, h.u, D, dt, nmax=1, T0=h.T, W0=h.W, V0=h.V)
    run.step(1, bkind=bkind, bpar=bpar)
    return run
