"""The paper's own workload (Sec. 2.5, Sec. 3.1) on the GPU against the oracle (GB300): a 2 mm bunch of
N_p macroparticles at 1-100 MeV, injected at 10 Earth radii in the centred dipole with a tilt, advanced
with the adaptive time step and the energy monitor.

The bunch is simulated in its own frame: it is centred at the origin and the dipole's centre sits at
-r0 = (+10 R_E, 0, 0), which is the paper's geometry translated by -r0. In absolute coordinates at
6.4e7 m a double resolves 7.5 nm, so every push would round positions to that grain; in the bunch frame
positions keep their full relative precision.

Bar (FP64 path): each step's size within 1e-12 relative of the oracle's on the first step and within
the run bar 1e-9 after it, positions within 1e-9 of the bunch size, mean energy within 1e-12 relative.
Mixed path: step sizes within 1e-5.
"""
import math
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2605_05543_gb300 import emppp, inputs  # noqa: E402

ADAPT = dict(oracle.ADAPTIVE_PAPER)
CENTER = tuple(-c for c in inputs.PAPER_R0)


def _rel(a, b):
    return abs(a - b) / abs(b)


def _runs(Np, E0, weight, steps, D, precision="fp64"):
    b = inputs.paper_bunch(Np, E0, theta=math.radians(30), phi=math.radians(45), seed=7, weight=weight)
    par = oracle.bext_params(2, m0=inputs.PAPER_M0, center=CENTER)
    run = oracle.Run(b.x, b.u, D, 1e-15, weights=b.weights, nmax=steps)
    T, E = [0.0], [oracle.mean_kinetic_energy(b.u, b.weights)]
    for _ in range(steps):
        run.step(1, bkind=2, bpar=par, adaptive=ADAPT)
        T.append(run.t)
        E.append(oracle.mean_kinetic_energy(run.u, b.weights))
    log = []
    with emppp.Solver(Np, D, 1e-15, precision=precision, proposal="closed_form") as s:
        s.set_particles(b.x.copy(), b.u.copy(), b.weights.copy())
        s.set_adaptive_dt(**ADAPT)
        s.set_energy_monitor(30e3 * emppp.EV)
        Eg = [s.get_energy()[0]["ebar"]]
        for _ in range(steps):
            s.step(1, emppp.bext_dipole(inputs.PAPER_M0, CENTER))
            st = s.stats()
            log.append((st["dt_last"], st["eta_min"], st["v_max"]))
            Eg.append(s.get_energy()[0]["ebar"])
        x, u, t, n = s.get_state()
    return b, run, np.array(run.adaptive_log), np.array(log), np.array(E), np.array(Eg), x, u, t


@pytest.mark.parametrize("Np,E0,weight", [(400, 1.0, 1e6), (800, 10.0, 1e6), (400, 100.0, 1e7)])
def test_paper_workload_fp64(Np, E0, weight):
    steps = 25
    b, run, ref, log, E, Eg, x, u, t = _runs(Np, E0, weight, steps, 64)
    assert all(_rel(log[0, c], ref[0, c]) <= 1e-12 for c in range(3))
    worst = max(_rel(log[k, c], ref[k, c]) for k in range(steps) for c in range(3))
    assert worst <= 1e-9, worst
    assert _rel(t, run.t) <= 1e-9
    sig = float(np.sqrt(np.mean(np.sum((run.x - run.x.mean(axis=0)) ** 2, axis=1))))
    err = np.max(np.linalg.norm(x - run.x, axis=1)) / sig
    assert err <= 1e-9, err
    assert np.max(np.abs(Eg - E) / E) <= 1e-12
    print(f"paper Np={Np} E0={E0} MeV w={weight:g}: dt {ref[0, 0]:.3e}..{ref[-1, 0]:.3e} s, worst step err "
          f"{worst:.1e}, positions {err:.1e}")


def test_paper_workload_mixed():
    steps = 25
    b, run, ref, log, E, Eg, x, u, t = _runs(800, 1.0, 1e6, steps, 64, precision="mixed")
    worst = max(_rel(log[k, c], ref[k, c]) for k in range(steps) for c in range(3))
    print(f"paper mixed: worst step err {worst:.1e}")
    assert worst <= 1e-5, worst


@pytest.mark.parametrize("E0", [10.0, 100.0])
def test_paper_workload_high_energy(E0):
    """The paper's higher beam energies (gamma 20.6 and 196.7), one step from a 30-step history of the
    paper's bunch, against the oracle. The retarded solve of a source moving towards the target is
    conditioned like 1 / (1 - beta cos psi), up to 2 gamma^2: both the oracle and the FP64 path lose
    digits in proportion (at gamma 196.7 the oracle itself is 2.4e-11 from a 40-digit evaluation of
    the same formulas), so the FP64 bar is 1e-12 scaled by (gamma0 / 3)^2. The mixed path keeps 1e-5:
    its C0 = L1^2 - |d|^2 is formed again in FP64 for the pairs where FP32 would lose that."""
    b = inputs.paper_bunch(800, E0, theta=math.radians(30), phi=math.radians(45), seed=8, weight=1e6)
    par = oracle.bext_params(2, m0=inputs.PAPER_M0, center=CENTER)
    run = oracle.Run(b.x, b.u, 64, 1e-12, weights=b.weights, nmax=30)
    run.step(29, bkind=2, bpar=par)
    n = run.n
    T, W, V = run.T[:n + 1], run.W[:n + 1], run.V[:n + 1]
    E_ref, B_ref, st_ref, M = oracle.self_fields(T, W, V, n, 64, weights=b.weights, mags=True)
    step = oracle.Run(None, run.u, 64, 1e-12, weights=b.weights, nmax=1, T0=T, W0=W, V0=V)
    step.step(1, bkind=2, bpar=par)  # B of the step: self field plus the dipole at x^{n+1/2}
    gamma0 = inputs.beam_kinematics(E0 * 1e6 * inputs.Q_E)[0]
    tol = {"fp64": 1e-12 * max(1.0, (gamma0 / 3.0) ** 2), "mixed": 1e-5}
    out = {}
    for precision in ("fp64", "mixed"):
        with emppp.Solver(800, 64, 1e-12, precision=precision, proposal="closed_form") as s:
            s.set_history(n, T.copy(), W.copy(), V.copy(), run.u.copy(), b.weights.copy())
            s.step(1, emppp.bext_dipole(inputs.PAPER_M0, CENTER))
            E, B = s.get_fields()
            st = s.stats()
        eE = float(np.max(np.abs(E - E_ref) / np.maximum(M[:, 0:1], 1e-300)))
        eB = float(np.max(np.abs(B - step.B) / np.maximum(M[:, 1:2], 1e-300)))
        out[precision] = (eE, eB, st["guard_fallbacks"])
        for k in ("out_of_history", "shortcut", "bisection"):
            assert st[k] == st_ref[k], (precision, k, st, st_ref)
    print(f"paper E0={E0} MeV (gamma {gamma0:.1f}): fp64 err {out['fp64'][0]:.1e}/{out['fp64'][1]:.1e}, mixed err "
          f"{out['mixed'][0]:.1e}/{out['mixed'][1]:.1e} ({out['mixed'][2]} FP64 fallbacks); branches {st_ref}")
    for p in ("fp64", "mixed"):
        assert max(out[p][:2]) <= tol[p], (p, out[p], tol[p])


def _golden_centroids():
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_centroid_steps.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                Np, step, t, z = line.split()
                rows.append((int(Np), int(step), float(t), float(z)))
    return rows


def test_centroid_speed_matches_the_printed_states():
    """The printed states of the baseline run give zbar / t = 2.276 m / 8.07e-9 s and 2.270 m / 8.04e-9 s:
    the centroid moves along the field-aligned injection direction at the beam speed. The N_p = 400 run
    of the paper's bunch (adaptive step, dipole) to the printed step gives the same centroid speed within
    the printed digits. (The time at a given step depends on the macroparticle weight, which follows from
    a peak density the paper does not give, so t itself is not compared.)"""
    Np, step, t_ref, z_ref = _golden_centroids()[0]
    b = inputs.paper_bunch(Np, 1.0, seed=11, weight=1e6)
    with emppp.Solver(Np, 1024, 1e-15, precision="mixed", proposal="closed_form") as s:
        s.set_particles(b.x.copy(), b.u.copy(), b.weights.copy())
        s.set_adaptive_dt(**ADAPT)
        s.step(step, emppp.bext_dipole(inputs.PAPER_M0, CENTER))
        x, u, t, n = s.get_state()
    zbar = float(np.average(x[:, 2], weights=b.weights) - np.average(b.x[:, 2], weights=b.weights))
    speed, speed_ref = zbar / t, z_ref / t_ref
    # the printed values carry 3-4 digits: 8.07e-9 is known to 0.07 %, 2.276 m to 0.03 %
    assert abs(speed / speed_ref - 1.0) <= 1.5e-3, (speed, speed_ref)
    for Np2, step2, t2, z2 in _golden_centroids()[1:]:
        assert abs((z2 / t2) / speed_ref - 1.0) <= 1.5e-3  # the two printed states agree with each other
