"""The comparison variants of the step on the GPU against the oracle (GB300): the midpoint
reconstruction of eq:mid, and the self fields evaluated at the pusher's half-step point (Sec. 2.3).

Bar (FP64 path): fields within 1e-12 of sum_j |E_ij| of each target, branch counts equal to the
oracle's, positions within 1e-9 of the bunch size after full runs; every proposal gives the same state
bit for bit, and graph replay gives the eager steps' state bit for bit.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import DT, field_errors, history_case, window

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2605_05543_gb300 import emppp, inputs  # noqa: E402


def _sigma(x):
    return float(np.sqrt(np.mean(np.sum((x - x.mean(axis=0)) ** 2, axis=1))))


@pytest.mark.parametrize("proposal", ["bisect", "closed_form", "mlp"])
@pytest.mark.parametrize("N,n,D", [(300, 30, 16), (257, 40, 64)])
def test_midpoint_fields_match_oracle(proposal, N, n, D):
    """One step on a stored history: several target tiles, a ragged last tile, every branch."""
    h = history_case(N, n, sigma=5e-6, seed=41)
    E_ref, B_ref, st_ref, M = oracle.self_fields(h.T, h.W, h.V, n, D, mags=True, variant=oracle.MIDPOINT)
    T, W, V, u = window(h, D)
    with emppp.Solver(N, D, DT, proposal=proposal, reconstruction="midpoint") as s:
        if proposal == "mlp":
            s.set_proposal(inputs.mlp_init_params(0))
        s.set_history(n, T, W, V, u)
        s.step(1)
        E, B = s.get_fields()
        st = s.stats()
    eE, eB = field_errors(E, B, E_ref, B_ref, M)
    assert eE <= 1e-12 and eB <= 1e-12, (eE, eB)
    for k in ("out_of_history", "shortcut", "bisection"):
        assert st[k] == st_ref[k], (k, st, st_ref)
    assert st_ref["bisection"] > 0
    # the variant differs from the method by far more than the tolerance
    E_lin, _, _ = oracle.self_fields(h.T, h.W, h.V, n, D)
    assert np.max(np.abs(E_lin - E_ref) / M[:, 0:1]) > 1e-6


def _run_pair(N, D, steps, variant, bkind=0, bpar=None, seed=42, **solver_kw):
    b = inputs.gaussian_bunch(N, 3e-6, 3.0, seed=seed)
    run = oracle.Run(b.x, b.u, D, DT, nmax=steps)
    run.step(steps, bkind=bkind, bpar=bpar, variant=variant)
    return b, run


@pytest.mark.parametrize("variant,kw", [
    (oracle.MIDPOINT, dict(reconstruction="midpoint")),
    (oracle.HALF_STEP, dict(field_point="half_step")),
    (oracle.MIDPOINT | oracle.HALF_STEP, dict(reconstruction="midpoint", field_point="half_step")),
])
def test_variant_runs_match_oracle(variant, kw):
    """Full runs of a gamma0 = 3 bunch past the ring's wrap (40 steps, depth 12) in a uniform field:
    positions, velocities, time and the last step's fields against the oracle's run."""
    N, D, steps = 200, 12, 40
    par = oracle.bext_params(1, b=(5e-5, 0.0, 0.0))
    b, run = _run_pair(N, D, steps, variant, bkind=1, bpar=par)
    with emppp.Solver(N, D, DT, proposal="closed_form", **kw) as s:
        s.set_particles(b.x.copy(), b.u.copy())
        s.step(steps, emppp.bext_uniform((5e-5, 0.0, 0.0)))
        x, u, t, n = s.get_state()
        E, B = s.get_fields()
    assert n == steps and t == run.t
    err = np.max(np.linalg.norm(x - run.x, axis=1)) / _sigma(run.x)
    assert err <= 1e-9, err
    assert np.max(np.abs(u - run.u)) <= 1e-9 * np.max(np.abs(run.u))
    scale = np.max(np.linalg.norm(run.E, axis=1))
    assert np.max(np.abs(E - run.E)) <= 1e-9 * scale
    assert np.max(np.abs(B - run.B)) <= 1e-9 * np.max(np.linalg.norm(run.B, axis=1))


def test_half_step_first_step_fields():
    """The first step's fields (one stored slot plus the provisional one) against the oracle to the
    field bar, so that the half-step point itself is checked before any trajectory error builds up."""
    b = inputs.gaussian_bunch(150, 2e-6, 3.0, seed=43)
    run = oracle.Run(b.x, b.u, 8, DT, nmax=1)
    run.step(1, variant=oracle.HALF_STEP)
    T = np.array([0.0, 0.5 * DT])
    x_half = b.x + 0.5 * DT * oracle.velocity(b.u)
    W = np.stack([b.x, x_half])
    V = np.stack([oracle.velocity(b.u)] * 2)
    _, _, _, M = oracle.self_fields(T, W, V, 1, 8, mags=True)
    with emppp.Solver(150, 8, DT, field_point="half_step") as s:
        s.set_particles(b.x.copy(), b.u.copy())
        s.step(1)
        E, B = s.get_fields()
        st = s.stats()
    eE, eB = field_errors(E, B, run.E, run.B, M)
    assert eE <= 1e-12 and eB <= 1e-12, (eE, eB)
    assert st["out_of_history"] + st["shortcut"] + st["bisection"] == 150 * 149


def test_variants_all_proposals_and_graphs_agree():
    """Bisection, closed-form and network proposals, eager and graph-replayed, give one state."""
    b = inputs.gaussian_bunch(160, 3e-6, 3.0, seed=44)
    params = inputs.mlp_init_params(0)
    out = []
    for proposal in ("bisect", "closed_form", "mlp"):
        for graphs in (False, True):
            stream = torch.cuda.Stream()
            with emppp.Solver(160, 10, DT, proposal=proposal, graphs=graphs, stream=stream,
                              reconstruction="midpoint", field_point="half_step") as s:
                if proposal == "mlp":
                    s.set_proposal(params)
                s.set_particles(b.x.copy(), b.u.copy())
                s.step(25)
                x, u, t, n = s.get_state()
            out.append((x, u, t))
    for x, u, t in out[1:]:
        assert np.array_equal(x, out[0][0]) and np.array_equal(u, out[0][1]) and t == out[0][2]


def test_half_step_batch_matches_single_bunches():
    """Two bunches in one handle with the half-step point: each is its own single-bunch oracle run."""
    b1 = inputs.gaussian_bunch(90, 2e-6, 3.0, seed=45)
    b2 = inputs.gaussian_bunch(37, 1e-6, 2.0, seed=46)
    steps, D = 15, 8
    with emppp.Solver(0, D, DT, bunches=[90, 37], field_point="half_step") as s:
        s.set_particles(np.concatenate([b1.x, b2.x]), np.concatenate([b1.u, b2.u]))
        s.step(steps)
        x, u, t, n = s.get_state()
    off = 0
    for bb in (b1, b2):
        run = oracle.Run(bb.x, bb.u, D, DT, nmax=steps)
        run.step(steps, variant=oracle.HALF_STEP)
        N = bb.x.shape[0]
        err = np.max(np.linalg.norm(x[off:off + N] - run.x, axis=1)) / _sigma(run.x)
        assert err <= 1e-9, err
        off += N


def _exact_fields(h, omega, A, targets):
    """Self fields of the analytic trajectories behind inputs.synthetic_history at the present slot:
    w_j(s) = x_j + v_j s + (A_j / omega^2)(1 - cos omega s), s = t - t_n; the retarded s_r < 0 of each
    pair solved by Newton on c^2 s^2 = |r - w_j(s)|^2 from the uniform-motion delay, then the
    Lienard-Wiechert field (the oracle's pinned eq:LW_E) with the exact w, v, a. Returns (E, sum |E_ij|)."""
    c = oracle.constants()["c"]
    x, v = h.W[h.n], h.V[h.n]
    N = x.shape[0]
    E = np.zeros((len(targets), 3))
    M = np.zeros(len(targets))
    for ii, i in enumerate(targets):
        js = np.array([j for j in range(N) if j != i])
        d = x[i] - x[js]
        dv = np.sum(d * v[js], axis=1)
        c2v2 = c * c - np.sum(v[js] ** 2, axis=1)
        s = -(dv + np.sqrt(dv * dv + c2v2 * np.sum(d * d, axis=1))) / c2v2
        for _ in range(30):
            w = x[js] + v[js] * s[:, None] + (A[js] / omega ** 2) * (1.0 - np.cos(omega * s))[:, None]
            vs = v[js] + (A[js] / omega) * np.sin(omega * s)[:, None]
            e = x[i] - w
            g = c * c * s * s - np.sum(e * e, axis=1)
            dg = 2.0 * c * c * s + 2.0 * np.sum(e * vs, axis=1)
            s = s - g / dg
        w = x[js] + v[js] * s[:, None] + (A[js] / omega ** 2) * (1.0 - np.cos(omega * s))[:, None]
        vs = v[js] + (A[js] / omega) * np.sin(omega * s)[:, None]
        acc = A[js] * np.cos(omega * s)[:, None]
        assert np.max(np.abs(np.linalg.norm(x[i] - w, axis=1) + c * s) / (-c * s)) <= 1e-13
        for k, j in enumerate(js):
            Ej, _ = oracle.lw_fields(x[i] - w[k], vs[k], acc[k], -inputs.Q_E)
            E[ii] += Ej
            M[ii] += np.linalg.norm(Ej)
    return E, M


def test_accuracy_linear_versus_midpoint():
    """The accuracy comparison the variant exists for: on trajectories with a known closed form (the
    synthetic history's), with every retarded time inside the stored history, the GPU fields of the
    linear reconstruction and of eq:mid against the exact Lienard-Wiechert fields. The linear form's error
    is second order in dt and the midpoint's first order; the printed numbers are the comparison."""
    N, n, D, dt, period = 512, 150, 256, 1e-15, 160.0
    b = inputs.gaussian_bunch(N, 1e-6, 1.5, seed=47)
    h = inputs.synthetic_history(b.x, b.u, n, dt, wiggle=1e-4, period_steps=period, seed=48)
    omega = 2.0 * np.pi / (period * dt)
    dirs = inputs.normals(48, 3 * N).reshape(N, 3)
    A = dirs / np.linalg.norm(dirs, axis=1, keepdims=True) * (1e-4 * oracle.constants()["c"] * omega)
    targets = np.random.default_rng(49).choice(N, 48, replace=False)
    E_ex, M = _exact_fields(h, omega, A, targets)
    err, med = {}, {}
    for recon in ("linear", "midpoint"):
        with emppp.Solver(N, D, dt, proposal="closed_form", reconstruction=recon) as s:
            s.set_history(n, h.T, h.W, h.V, h.u)
            s.step(1)
            E, _ = s.get_fields()
            st = s.stats()
        assert st["out_of_history"] == 0
        e = np.max(np.abs(E[targets] - E_ex) / M[:, None], axis=1)
        err[recon], med[recon] = float(np.max(e)), float(np.median(e))
    print(f"field error against the exact trajectories (dt = {dt:g} s), median / max over targets: linear "
          f"{med['linear']:.2e} / {err['linear']:.2e}, midpoint {med['midpoint']:.2e} / {err['midpoint']:.2e}")
    assert err["linear"] <= 1e-5 and err["linear"] <= 1e-3 * err["midpoint"], err


def test_variant_option_errors():
    with pytest.raises(emppp.EmpppError) as ei:
        emppp.Solver(8, 8, DT, precision="mixed", reconstruction="midpoint")
    assert ei.value.status == emppp.ERR_ARG
    with pytest.raises(emppp.EmpppError) as ei:
        emppp.Solver(8, 8, DT, precision="mixed", field_point="half_step")
    assert ei.value.status == emppp.ERR_ARG
    with emppp.Solver(8, 8, DT, field_point="half_step") as s:
        with pytest.raises(emppp.EmpppError) as ei:
            s.set_adaptive_dt()
        assert ei.value.status == emppp.ERR_STATE
    with emppp.Solver(8, 8, DT) as s:
        s.set_adaptive_dt()
        with pytest.raises(emppp.EmpppError) as ei:
            s.set_options(reconstruction="midpoint")
        assert ei.value.status == emppp.ERR_STATE
