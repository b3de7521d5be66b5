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


def gpu_fields_from_history(Solver, h, D, dt=DT, tuning=None, **kw):
    """Fields and stats of one GPU step evaluated on history h (and the state after the step); tuning:
    keyword arguments of Solver.set_tuning (work split and tile shape), else the defaults."""
    T, W, V, u = window(h, D)
    with Solver(W.shape[1], D, dt, **kw) as s:
        s.set_history(h.n, T, W, V, u)
        if tuning:
            s.set_tuning(**tuning)
        s.step(1)
        E, B = s.get_fields()
        st = s.stats()
        x, uu, t, n = s.get_state()
    return E, B, st, x, uu


def oracle_step_from_history(h, D, dt=DT, bkind=0, bpar=None):
    run = oracle.Run(None, h.u, D, dt, nmax=1, T0=h.T, W0=h.W, V0=h.V)
    run.step(1, bkind=bkind, bpar=bpar)
    return run


def sigma_rms(x):
    """rms distance of the particles from their centroid: the bunch size of the position bar."""
    return float(np.sqrt(np.mean(np.sum((x - x.mean(axis=0)) ** 2, axis=1))))


def record(name, values):
    """Append measured numbers of a test to $EMPPP_TEST_RECORD_DIR/test_record.jsonl when that variable
    names a directory (the tests' numbers on record); otherwise do nothing."""
    import json
    import os

    d = os.environ.get("EMPPP_TEST_RECORD_DIR")
    if not d or not os.path.isdir(d):
        return
    with open(os.path.join(d, "test_record.jsonl"), "a") as f:
        f.write(json.dumps({"test": name, **values}) + "\n")


def light_sphere_case(nb=64, n=40, seed=70, oldest=False):
    """nb two-particle bunches (history n + 1 slots, step DT): in each, a resting target sits on the light
    sphere of one stored slot k of its source, c (t_n - t_k) from w_k to within 0 to 1e-12 relative, and
    the source moves with constant acceleration. Every node test at that slot falls inside the mixed path's
    FP32 guard band. With oldest, k is the oldest slot and the target lies ahead of the source along its
    motion, so that the uniform-motion guess falls at the edge of the history and the mixed path's
    oldest-slot bound is tried on pairs it must not decide. Returns (T, W, V, u)."""
    rng = np.random.default_rng(seed)
    C = inputs.C_LIGHT
    T = np.array([k * DT for k in range(n + 1)])
    W = np.zeros((n + 1, 2 * nb, 3))
    V = np.zeros((n + 1, 2 * nb, 3))
    eps = [0.0, 1e-16, -1e-16, 1e-15, -1e-15, 1e-14, -1e-14, 1e-12, -1e-12]
    for b in range(nb):
        beta = rng.uniform(0.3, 0.9)
        vdir = rng.normal(size=3)
        v0 = beta * C * vdir / np.linalg.norm(vdir)
        acc = rng.normal(size=3) * 1e18
        w00 = rng.normal(size=3) * 1e-6
        k = 0 if oldest else int(rng.integers(1, n - 1))
        nhat = rng.normal(size=3)
        if oldest:
            nhat = 0.3 * nhat + vdir / np.linalg.norm(vdir)
        nhat /= np.linalg.norm(nhat)
        wk = w00 + v0 * T[k] + 0.5 * acc * T[k] ** 2
        r = wk + C * (T[n] - T[k]) * (1.0 + eps[b % len(eps)]) * nhat
        W[:, 2 * b] = r  # the target rests on the sphere
        W[:, 2 * b + 1] = w00 + v0[None] * T[:, None] + 0.5 * acc[None] * T[:, None] ** 2
        V[:, 2 * b + 1] = v0[None] + acc[None] * T[:, None]
    u = np.zeros((2 * nb, 3))
    g = 1.0 / np.sqrt(1.0 - np.sum(V[n, 1::2] ** 2, axis=1) / C ** 2)
    u[1::2] = V[n, 1::2] * g[:, None]
    return T, W, V, u
