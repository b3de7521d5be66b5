"""Adaptive time step (Sec. 2.4) on the GPU against the oracle's rule (GB300).

Every step takes dt = clip(c_dt eta_min / v_max, dt_min, dt_max) from the interaction scale of its own
retarded solve. The oracle runs the same rule on the same seeded bunch. Bar:
- FP64 path: over a run, each step's (dt, eta_min, v_max), the time stamps and the positions within the
  run bar of 1e-9 (relative; positions relative to the bunch size), the first step's within 1e-12; one
  step from an unevenly spaced history: fields within 1e-12 of sum_j |E_ij|, the oracle's branch
  counts, and (dt, eta_min, v_max) within 1e-12;
- mixed path (FP32 interaction scale): the same quantities within 1e-5, brackets exact.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import field_errors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2605_05543_gb300 import emppp, inputs  # noqa: E402

DT0 = 1e-15
PAPER = dict(oracle.ADAPTIVE_PAPER)


def _rel(a, b):
    return abs(a - b) / abs(b)


def _sigma_rms(x):
    return float(np.sqrt(np.mean(np.sum((x - x.mean(axis=0)) ** 2, axis=1))))


def _oracle_run(bunch, D, steps, adaptive):
    run = oracle.Run(bunch.x, bunch.u, D, DT0, nmax=steps)
    run.step(steps, adaptive=adaptive)
    return run


def _gpu_run(bunch, D, steps, adaptive, precision="fp64", proposal="bisect"):
    """Steps one at a time, logging (dt, eta_min, v_max) of each; returns the log, the final state and the
    stored history."""
    N = bunch.x.shape[0]
    log = []
    with emppp.Solver(N, D, DT0, precision=precision, proposal=proposal) as s:
        s.set_particles(bunch.x.copy(), bunch.u.copy())
        s.set_adaptive_dt(**adaptive)
        for _ in range(steps):
            s.step(1)
            st = s.stats()
            log.append((st["dt_last"], st["eta_min"], st["v_max"]))
        x, u, t, n = s.get_state()
        hist = s.get_history()
    return np.array(log), x, u, t, n, hist


@pytest.mark.parametrize("proposal", ["bisect", "closed_form"])
def test_fp64_adaptive_run_matches_oracle(proposal):
    """N = 200 Gaussian bunch (sigma = 5 um, gamma0 = 3), the paper's rule (C = 0.05, dt in [1e-15,
    1e-12] s), 30 steps: the chosen steps lie inside the clamps and change every step."""
    b = inputs.gaussian_bunch(200, 5e-6, 3.0, seed=1)
    D, steps = 64, 30
    run = _oracle_run(b, D, steps, PAPER)
    log, x, u, t, n, (nh, T, W, V, uh) = _gpu_run(b, D, steps, PAPER, proposal=proposal)
    ref = np.array(run.adaptive_log)
    assert ref[:, 0].min() > 1e-15 and ref[:, 0].max() < 1e-12  # the formula, not a clamp, sets dt
    assert len(np.unique(ref[:, 0])) == steps
    # the first step's inputs are identical on both sides: the field bar; after it, the two runs carry
    # rounding-level differences in positions, which the run's bar (1e-9) bounds
    assert all(_rel(log[0, c], ref[0, c]) <= 1e-12 for c in range(3)), (log[0], ref[0])
    worst = max(_rel(log[k, c], ref[k, c]) for k in range(steps) for c in range(3))
    err = np.max(np.linalg.norm(x - run.x, axis=1)) / _sigma_rms(run.x)
    print(f"fp64 adaptive run ({proposal}): worst relative error of (dt, eta_min, v_max) {worst:.2e}, "
          f"positions {err:.2e}")
    assert worst <= 1e-9, worst
    assert n == steps and _rel(t, run.t) <= 1e-9
    assert np.max(np.abs(T - run.T[n - T.shape[0] + 1:n + 1]) / run.T[n]) <= 1e-9
    assert err <= 1e-9, err
    assert np.max(np.abs(u - run.u)) <= 1e-9 * np.max(np.abs(run.u))


def _history(kind, N=300, steps=24, seed=2):
    """Oracle history with unevenly spaced slots: 'cycled' steps through dt = (1, 2.5, 0.6, 1.7) fs;
    'adaptive' takes the rule's own steps (about 70 fs here, so that most close pairs fall in the
    near-field shortcut bracket, where c (t_n - t_r) is far below c (t_n - t_{n-1}))."""
    b = inputs.gaussian_bunch(N, 5e-6, 3.0, seed=seed)
    run = oracle.Run(b.x, b.u, 64, DT0, nmax=steps)
    if kind == "adaptive":
        run.step(steps, adaptive=PAPER)
    else:
        for k in range(steps):
            run.dt = DT0 * (1.0, 2.5, 0.6, 1.7)[k % 4]
            run.step(1)
    return run


@pytest.mark.parametrize("kind", ["cycled", "adaptive"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("proposal", ["bisect", "closed_form"])
def test_one_step_from_uneven_history(kind, precision, tol, proposal):
    """Fields, interaction scale and step of one adaptive step evaluated on a history whose slots are
    unevenly spaced, against the oracle at the same step (depth 16 of 25 stored slots)."""
    run = _history(kind)
    n, D, N = run.n, 16, run.N
    T, W, V = run.T[:n + 1], run.W[:n + 1], run.V[:n + 1]
    if kind == "cycled":
        assert np.ptp(np.diff(T)) > np.mean(np.diff(T))  # the spacing varies
    E_ref, B_ref, st_ref, M = oracle.self_fields(T, W, V, n, D, mags=True)
    eta_ref, vmax_ref = oracle.interaction_scale(T, W, V, n, D, 0.0)
    dt_ref = oracle.adaptive_dt(eta_ref, vmax_ref)
    k0 = n - D + 1
    with emppp.Solver(N, D, DT0, precision=precision, proposal=proposal) as s:
        s.set_history(n, T[k0:].copy(), W[k0:].copy(), V[k0:].copy(), run.u.copy())
        s.set_adaptive_dt(**PAPER)
        s.step(1)
        E, B = s.get_fields()
        st = s.stats()
        x, u, t, nn = s.get_state()
    eE, eB = field_errors(E, B, E_ref, B_ref, M)
    print(f"{kind} {precision} {proposal}: field err E {eE:.2e} B {eB:.2e}; dt {_rel(st['dt_last'], dt_ref):.1e} "
          f"eta {_rel(st['eta_min'], eta_ref):.1e} v {_rel(st['v_max'], vmax_ref):.1e}; branches "
          f"{st['out_of_history']}/{st['shortcut']}/{st['bisection']}")
    assert eE <= tol and eB <= tol, (eE, eB)
    for k in ("out_of_history", "shortcut", "bisection"):
        assert st[k] == st_ref[k], (k, st, st_ref)
    assert _rel(st["eta_min"], eta_ref) <= tol and _rel(st["v_max"], vmax_ref) <= tol
    assert _rel(st["dt_last"], dt_ref) <= tol
    assert nn == n + 1 and _rel(t - T[n], dt_ref) <= tol


def test_mixed_adaptive_run_tracks_oracle():
    """Mixed path over a 30-step adaptive run: every step's size within 1e-5 of the oracle's."""
    b = inputs.gaussian_bunch(200, 5e-6, 3.0, seed=1)
    run = _oracle_run(b, 64, 30, PAPER)
    log, x, u, t, n, _ = _gpu_run(b, 64, 30, PAPER, precision="mixed", proposal="closed_form")
    ref = np.array(run.adaptive_log)
    worst = max(_rel(log[k, c], ref[k, c]) for k in range(30) for c in range(3))
    print(f"mixed adaptive run: worst relative error of (dt, eta_min, v_max) {worst:.2e}")
    assert worst <= 1e-5, worst
    assert _rel(t, run.t) <= 1e-5


def test_cutoff_and_clamps():
    """eta_allow removes the closest pairs from the scale; dt_min and dt_max clamp the step."""
    b = inputs.gaussian_bunch(128, 1e-6, 3.0, seed=3)
    D = 32
    run = _oracle_run(b, D, 6, PAPER)
    n = run.n
    T, W, V = run.T[:n + 1], run.W[:n + 1], run.V[:n + 1]
    eta0, _ = oracle.interaction_scale(T, W, V, n, D, 0.0)
    cut = 3.0 * eta0
    eta_c, v_c = oracle.interaction_scale(T, W, V, n, D, cut)
    cases = [
        dict(PAPER, eta_allow=cut),                       # cutoff: a larger eta_min
        dict(PAPER, dt_min=1e-13, dt_max=1e-12),         # the formula's step is below dt_min
        dict(PAPER, dt_min=1e-16, dt_max=2e-15),         # ... and above dt_max
        dict(PAPER, eta_allow=1.0),                       # no pair qualifies: dt_max
    ]
    for cfg in cases:
        eta_r, v_r = oracle.interaction_scale(T, W, V, n, D, cfg["eta_allow"])
        dt_r = oracle.adaptive_dt(eta_r, v_r, cfg["c_dt"], cfg["dt_min"], cfg["dt_max"])
        with emppp.Solver(128, D, DT0) as s:
            s.set_history(n, T.copy(), W.copy(), V.copy(), run.u.copy())
            s.set_adaptive_dt(**cfg)
            s.step(1)
            st = s.stats()
            _, _, t, _ = s.get_state()
        assert _rel(st["dt_last"], dt_r) <= 1e-12, (cfg, st["dt_last"], dt_r)
        assert _rel(t - T[n], dt_r) <= 1e-12
        if np.isfinite(eta_r):
            assert _rel(st["eta_min"], eta_r) <= 1e-12 and _rel(st["v_max"], v_r) <= 1e-12
        else:
            assert st["eta_min"] == 0.0 and st["v_max"] == 0.0 and st["dt_last"] == cfg["dt_max"]
    assert eta_c > cut > eta0 and v_c > 0.0


def test_disable_returns_to_fixed_step():
    b = inputs.gaussian_bunch(64, 2e-6, 3.0, seed=4)
    with emppp.Solver(64, 16, DT0) as s:
        s.set_particles(b.x.copy(), b.u.copy())
        s.set_adaptive_dt(**PAPER)
        s.step(3)
        _, _, t3, _ = s.get_state()
        assert t3 > 3 * DT0
        s.set_adaptive_dt(enable=False)
        s.step(2)
        _, _, t5, n5 = s.get_state()
        assert n5 == 5 and t5 == (t3 + DT0) + DT0
        assert s.stats()["dt_last"] == DT0
    with pytest.raises(emppp.EmpppError) as ei:
        with emppp.Solver(8, 8, DT0) as s:
            s.set_adaptive_dt(c_dt=0.05, dt_min=1e-12, dt_max=1e-15)
    assert ei.value.status == emppp.ERR_ARG


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_is_bitwise_identical(precision):
    """Captured and replayed steps (the device picks each step's size inside the graph) give the eager
    steps' state bit for bit."""
    b = inputs.gaussian_bunch(300, 5e-6, 3.0, seed=5)
    out = []
    for graphs in (False, True):
        stream = torch.cuda.Stream()
        with emppp.Solver(300, 32, DT0, precision=precision, proposal="closed_form", graphs=graphs,
                          stream=stream) as s:
            s.set_particles(b.x.copy(), b.u.copy())
            s.set_adaptive_dt(**PAPER)
            s.step(12)
            x, u, t, n = s.get_state()
            _, T, _, _, _ = s.get_history()
        out.append((x, u, t, T))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] and np.array_equal(out[0][3], out[1][3])


def test_adaptive_with_ring_wrap_and_batch():
    """Adaptive steps over a history ring that wraps (depth 8 for 20 steps) and in a two-bunch batch: each
    bunch's state equals its own single-bunch run driven by the batch's common steps (the smaller of the
    two bunches' steps), and the single-bunch FP64 run with depth 8 matches the oracle's."""
    b1 = inputs.gaussian_bunch(150, 3e-6, 3.0, seed=21)
    b2 = inputs.gaussian_bunch(90, 1e-6, 5.0, seed=22)
    D, steps = 8, 20
    # ring wrap, single bunch, against the oracle
    run = _oracle_run(b1, D, steps, PAPER)
    log, x, u, t, n, _ = _gpu_run(b1, D, steps, PAPER)
    ref = np.array(run.adaptive_log)
    worst = max(_rel(log[k, c], ref[k, c]) for k in range(steps) for c in range(3))
    err = np.max(np.linalg.norm(x - run.x, axis=1)) / _sigma_rms(run.x)
    assert worst <= 1e-9 and err <= 1e-9, (worst, err)
    # the batch takes the smaller step of the two bunches at every step
    with emppp.Solver(0, D, DT0, bunches=[150, 90]) as s:
        s.set_particles(np.concatenate([b1.x, b2.x]), np.concatenate([b1.u, b2.u]))
        s.set_adaptive_dt(**PAPER)
        dts = []
        for _ in range(steps):
            s.step(1)
            dts.append(s.stats()["dt_last"])
        xb, ub, tb, nb = s.get_state()
    log1 = _gpu_run(b1, D, steps, PAPER)[0]
    log2 = _gpu_run(b2, D, steps, PAPER)[0]
    assert _rel(dts[0], min(log1[0, 0], log2[0, 0])) <= 1e-15
    # replaying the batch's steps on each bunch alone gives the batch's states
    for (bb, lo, hi) in ((b1, 0, 150), (b2, 150, 240)):
        r = oracle.Run(bb.x, bb.u, D, DT0, nmax=steps)
        for dt in dts:
            r.dt = dt
            r.step(1)
        e = np.max(np.linalg.norm(xb[lo:hi] - r.x, axis=1)) / _sigma_rms(r.x)
        assert e <= 1e-9, e


def test_adaptive_with_learned_proposal():
    """The network proposal under the adaptive step: same states as the bisection proposal, bit for bit."""
    b = inputs.gaussian_bunch(200, 5e-6, 3.0, seed=23)
    params = inputs.mlp_init_params(0)
    out = []
    for proposal in ("bisect", "mlp"):
        with emppp.Solver(200, 32, DT0, proposal=proposal) as s:
            if proposal == "mlp":
                s.set_proposal(params)
            s.set_particles(b.x.copy(), b.u.copy())
            s.set_adaptive_dt(**PAPER)
            s.step(10)
            x, u, t, n = s.get_state()
        out.append((x, u, t))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2]
