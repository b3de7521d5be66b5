"""Stage switch by the energy criterion (Sec. 2.7) on the GPU against the oracle (GB300).

Bar: the mean kinetic energy per electron of every bunch within 1e-12 relative of the oracle's at every
step (FP64 path), the rate dE/dt within the rounding that its backward difference amplifies, the switch
step equal to the oracle's, and the two-stage procedure's re-run identical, bit for bit, to a plain run
of the same number of steps.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2605_05543_gb300 import emppp, inputs  # noqa: E402

QE = 1.602176634e-19
ME = 9.1093837015e-31
K_C = 1.0 / (4.0 * math.pi * 8.8541878128e-12)


def _pair_at_rest(d0=1e-8):
    x = np.array([[0.0, 0.0, -d0 / 2], [0.0, 0.0, d0 / 2]])
    return x, np.zeros((2, 3)), d0


def _oracle_record(x, u, D, dt, steps, weights=None, bkind=0, bpar=None):
    run = oracle.Run(x, u, D, dt, weights=weights, nmax=steps)
    T, E = [0.0], [oracle.mean_kinetic_energy(u, weights)]
    for _ in range(steps):
        run.step(1, bkind=bkind, bpar=bpar)
        T.append(run.t)
        E.append(oracle.mean_kinetic_energy(run.u, weights))
    return run, np.array(T), np.array(E)


def _gpu_record(s, steps, bext=None):
    out = [s.get_energy()]
    for _ in range(steps):
        s.step(1, bext)
        out.append(s.get_energy())
    return out


def test_coulomb_pair_record_and_switch():
    """Two electrons released at rest 10 nm apart (FP64 path): the record and the switch step."""
    x, u, d0 = _pair_at_rest()
    ke2 = K_C * QE * QE
    t_dyn = d0 / math.sqrt(ke2 / d0 / ME)
    dt, steps = 2e-3 * t_dyn, 3000
    run, T, E = _oracle_record(x, u, 16, dt, steps)
    rates = np.diff(E) / np.diff(T)
    eps = 0.2 * rates.max()
    n_ref, _ = oracle.energy_switch(T, E, eps, 1)
    assert 10 < n_ref < steps
    with emppp.Solver(2, 16, dt) as s:
        s.set_particles(x.copy(), u.copy())
        s.set_energy_monitor(eps, hold=1)
        rec = _gpu_record(s, steps)
    eb = np.array([r[0]["ebar"] for r in rec])
    assert np.max(np.abs(eb[1:] - E[1:]) / E[1:]) <= 1e-12
    assert eb[0] == 0.0
    # the rate amplifies the energy's rounding by E / (dE per step)
    rg = np.array([r[0]["rate"] for r in rec[1:]])
    tol = 1e-13 * np.abs(E[1:]) / dt + 1e-12 * np.abs(rates)
    assert np.all(np.abs(rg - rates) <= tol)
    last = rec[-1][0]
    assert last["switched"] == 1 and last["armed"] == 1
    assert last["n_sw"] == n_ref and last["t_sw"] == T[n_ref]


@pytest.mark.parametrize("hold", [1, 5])
def test_bunch_record_matches_oracle(hold):
    """N = 256 Gaussian bunch (sigma = 10 um, gamma0 = 3) in a uniform field, 60 steps: every step's mean
    energy, and the switch step of a threshold the decaying rate crosses."""
    b = inputs.gaussian_bunch(256, 10e-6, 3.0, seed=0)
    dt, steps = 1e-15, 60
    par = oracle.bext_params(1, b=(5e-5, 0.0, 0.0))
    run, T, E = _oracle_record(b.x, b.u, 64, dt, steps, bkind=1, bpar=par)
    rates = np.diff(E) / np.diff(T)
    with emppp.Solver(256, 64, dt) as s:
        s.set_particles(b.x.copy(), b.u.copy())
        s.set_energy_monitor(1.0, hold=hold)  # any threshold; the record does not depend on it
        rec = _gpu_record(s, steps, emppp.bext_uniform((5e-5, 0.0, 0.0)))
    eb = np.array([r[0]["ebar"] for r in rec])
    assert np.max(np.abs(eb - E) / E) <= 1e-12, np.max(np.abs(eb - E) / E)
    rg = np.array([r[0]["rate"] for r in rec[1:]])
    assert np.all(np.abs(rg - rates) <= 1e-13 * E[1:] / dt + 1e-12 * np.abs(rates))
    # a threshold between the rate's extremes, away from any step's rate by a margin
    lo, hi = np.abs(rates).min(), np.abs(rates).max()
    cands = np.linspace(lo, hi, 41)[1:-1]
    margin = np.array([np.min(np.abs(np.abs(rates) - c)) / c for c in cands])
    eps = float(cands[np.argmax(margin)])
    n_ref, _ = oracle.energy_switch(T, E, eps, hold)
    with emppp.Solver(256, 64, dt) as s:
        s.set_particles(b.x.copy(), b.u.copy())
        s.set_energy_monitor(eps, hold=hold)
        s.step(steps, emppp.bext_uniform((5e-5, 0.0, 0.0)))
        st = s.get_energy()[0]
    assert st["n_sw"] == n_ref and (n_ref < 0 or st["t_sw"] == T[n_ref])
    assert st["switched"] == (1 if n_ref >= 0 else 0)


def test_batch_records_per_bunch():
    """Two bunches of different sizes in one handle: each bunch's record is its own oracle record."""
    b1 = inputs.gaussian_bunch(100, 3e-6, 3.0, seed=1)
    b2 = inputs.gaussian_bunch(37, 1e-6, 2.0, seed=2)
    dt, steps = 1e-15, 20
    refs = [_oracle_record(bb.x, bb.u, 32, dt, steps)[2] for bb in (b1, b2)]
    with emppp.Solver(0, 32, dt, bunches=[100, 37]) as s:
        s.set_particles(np.concatenate([b1.x, b2.x]), np.concatenate([b1.u, b2.u]))
        s.set_energy_monitor(1.0)
        rec = _gpu_record(s, steps)
    for b in range(2):
        eb = np.array([r[b]["ebar"] for r in rec])
        assert np.max(np.abs(eb - refs[b]) / refs[b]) <= 1e-12


def test_two_stage_procedure():
    """emppp_two_stage on the Coulomb pair: the threshold step is the monitoring run's, the switch comes
    t_after later, the re-run's state at the switch is a plain run's bit for bit, and stage 2 is the
    handoff plus the dipole transport."""
    x, u, d0 = _pair_at_rest()
    ke2 = K_C * QE * QE
    dt = 2e-3 * d0 / math.sqrt(ke2 / d0 / ME)
    _, T, E = _oracle_record(x, u, 16, dt, 2000)
    eps = 0.2 * (np.diff(E) / np.diff(T)).max()
    n_ref, _ = oracle.energy_switch(T, E, eps, 1)
    RE = inputs.R_EARTH
    m0 = 3.1e-5 * 4 * math.pi * RE ** 3 / 1.25663706212e-6
    center = (-4 * RE, 0.0, 0.0)
    extra = 37  # the coupled model stays on 37 steps past the threshold (t_sw > t_th)
    with emppp.Solver(2, 16, dt) as s:
        rep = s.two_stage(x.copy(), u.copy(), eps, max_stage1_steps=2000, dt2=1e-9, steps2=100, check_every=64,
                          t_after=(extra - 0.5) * dt, bext2=emppp.bext_dipole(m0), center=center)
        x2, u2, t2, n2 = s.get_state()
    assert rep["switched"] == 1 and rep["n_th"] == n_ref and rep["t_th"] == T[n_ref]
    assert rep["n_sw"] == n_ref + extra and rep["t_sw"] == T[n_ref + extra]
    assert rep["stage1_steps_first_run"] >= n_ref
    n_sw = n_ref + extra
    with emppp.Solver(2, 16, dt) as s:
        s.set_particles(x.copy(), u.copy())
        s.step(n_sw)
        xs, us, ts, ns = s.get_state()
        s.handoff(center)
        s.transport(100, 1e-9, emppp.bext_dipole(m0))
        x3, u3, t3, n3 = s.get_state()
    assert np.array_equal(x2, x3) and np.array_equal(u2, u3) and t2 == t3 and n2 == n3 == n_sw + 100
    # stage 2 against the oracle: the translated pair pushed in the dipole alone
    xt = xs + (np.asarray(center) - xs.mean(axis=0))
    run = oracle.Run(xt, us, 4, 1e-9, nmax=100)
    run.step(100, bkind=2, bpar=oracle.bext_params(2, m0=m0), self_on=False)
    assert np.max(np.abs(x3 - run.x)) <= 1e-9 * RE
    assert np.max(np.abs(u3 - run.u)) <= 1e-9 * np.max(np.abs(run.u))


def test_graph_replay_keeps_the_record():
    b = inputs.gaussian_bunch(200, 5e-6, 3.0, seed=3)
    out = []
    for graphs in (False, True):
        stream = torch.cuda.Stream()
        with emppp.Solver(200, 32, 1e-15, graphs=graphs, stream=stream) as s:
            s.set_particles(b.x.copy(), b.u.copy())
            s.set_energy_monitor(1.0, hold=2)
            s.step(15)
            out.append(s.get_energy()[0])
    assert out[0] == out[1]


def test_monitor_errors():
    with emppp.Solver(4, 8, 1e-15) as s:
        with pytest.raises(emppp.EmpppError) as ei:
            s.set_energy_monitor(-1.0)
        assert ei.value.status == emppp.ERR_ARG
        with pytest.raises(emppp.EmpppError) as ei:
            s.set_energy_monitor(1.0, hold=0)
        assert ei.value.status == emppp.ERR_ARG
        b = inputs.gaussian_bunch(4, 1e-6, 3.0, seed=4)
        s.set_particles(b.x.copy(), b.u.copy())
        with pytest.raises(emppp.EmpppError) as ei:
            s.get_energy()
        assert ei.value.status == emppp.ERR_STATE


@pytest.mark.parametrize("N", [300, 20000])
def test_monitor_on_both_launch_forms(N):
    """Systems of up to 16384 particles evaluate the monitor in the post-pair launch's last block from
    terms the pushing threads formed; larger ones in the monitor's own launch. Both against the oracle's
    mean energy of the GPU's own state after each step."""
    b = inputs.gaussian_bunch(N, 20e-6, 3.0, seed=5)
    w = np.linspace(0.5, 2.0, N)
    with emppp.Solver(N, 8, 1e-15, precision="mixed", proposal="closed_form") as s:
        s.set_particles(b.x.copy(), b.u.copy(), w.copy())
        s.set_energy_monitor(1.0)
        for _ in range(3):
            s.step(1)
            x, u, t, n = s.get_state()
            e = s.get_energy()[0]
            ref = oracle.mean_kinetic_energy(u, w)
            assert abs(e["ebar"] - ref) <= 1e-12 * ref, (N, e["ebar"], ref)
