"""Batched bunches, the stage-1 -> stage-2 handoff, stage-2 transport and CUDA-graph replay (GB300).

- A batch of independent bunches gives, bunch by bunch, exactly (bit for bit) what separate solvers give
  with the same source chunking, and matches the oracle.
- The handoff puts each bunch's weighted centroid at the requested point and keeps the momenta.
- Stage-2 transport in the centred dipole agrees with the oracle's push with the pair fields off, and
  conserves |u| in a static magnetic field.
- One step captured in a CUDA graph and replayed gives the same state, bit for bit, as eager launches.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import DT, field_errors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2605_05543_gb300 import emppp, inputs  # noqa: E402

RE = inputs.R_EARTH
MU0 = 1.25663706212e-6
M0_CFG = 3.1e-5 * 4 * math.pi * RE ** 3 / MU0  # dipole with B = 3.1e-5 T at 1 Earth radius


def _bunches(spec):
    xs, us = [], []
    for N, sigma, g0, seed in spec:
        b = inputs.gaussian_bunch(N, sigma, g0, seed=seed)
        xs.append(b.x)
        us.append(b.u)
    return xs, us


SPEC = [(300, 5e-6, 3.0, 1), (129, 20e-6, 2.0, 2), (517, 10e-6, 8.0, 3)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_separate_solvers(precision):
    xs, us = _bunches(SPEC)
    steps, D = 12, 8
    sizes = [x.shape[0] for x in xs]
    with emppp.Solver(0, D, DT, precision=precision, source_split=2, bunches=sizes) as s:
        s.set_particles(np.concatenate(xs), np.concatenate(us))
        s.step(steps)
        xb, ub, tb, nb = s.get_state()
        Eb, Bb = s.get_fields()
        stb = s.stats()
    off = 0
    pairs = 0
    for x, u in zip(xs, us):
        N = x.shape[0]
        with emppp.Solver(N, D, DT, precision=precision, source_split=2) as s1:
            s1.set_particles(x.copy(), u.copy())
            s1.step(steps)
            x1, u1, t1, n1 = s1.get_state()
            E1, B1 = s1.get_fields()
        assert np.array_equal(xb[off:off + N], x1) and np.array_equal(ub[off:off + N], u1)
        assert np.array_equal(Eb[off:off + N], E1) and np.array_equal(Bb[off:off + N], B1)
        off += N
        pairs += N * (N - 1)
    assert stb["pairs"] == steps * pairs
    assert nb == steps and tb == t1


def test_batch_fields_match_oracle():
    from gpu_helpers import history_case, window

    hs = [history_case(N, 40, sigma=sig, gamma0=g0, seed=sd) for N, sig, g0, sd in SPEC]
    D = 32
    wins = [window(h, D) for h in hs]
    T = wins[0][0]
    W = np.concatenate([w[1] for w in wins], axis=1)
    V = np.concatenate([w[2] for w in wins], axis=1)
    u = np.concatenate([w[3] for w in wins])
    for h in hs[1:]:
        assert np.array_equal(h.T, hs[0].T)
    with emppp.Solver(0, D, DT, bunches=[w[1].shape[1] for w in wins]) as s:
        s.set_history(40, T, np.ascontiguousarray(W), np.ascontiguousarray(V), u)
        s.step(1)
        E, B = s.get_fields()
    off = 0
    for h in hs:
        N = h.W.shape[1]
        E_ref, B_ref, _, M = oracle.self_fields(h.T, h.W, h.V, 40, D, mags=True)
        eE, eB = field_errors(E[off:off + N], B[off:off + N], E_ref, B_ref, M)
        assert eE <= 1e-12 and eB <= 1e-12
        off += N


def test_handoff_places_centroids():
    xs, us = _bunches(SPEC)
    center = np.array([-4 * RE, 0.0, 0.0])
    sizes = [x.shape[0] for x in xs]
    w = np.concatenate([np.linspace(0.5, 1.5, n) for n in sizes])
    with emppp.Solver(0, 8, DT, bunches=sizes) as s:
        s.set_particles(np.concatenate(xs), np.concatenate(us), w)
        s.step(3)
        x0, u0, _, n0 = s.get_state()
        s.handoff(center)
        x1, u1, t1, n1 = s.get_state()
        n, T, W, V, uh = s.get_history()
    assert n1 == n0 and np.array_equal(u1, u0)
    assert T.shape[0] == 1 and np.array_equal(W[0], x1)
    off = 0
    for N in sizes:
        ww = w[off:off + N, None]
        cen = np.sum(ww * x1[off:off + N], axis=0) / np.sum(ww)
        assert np.max(np.abs(cen - center)) <= 1e-9 * RE
        # a rigid translation: relative positions unchanged
        d1 = x1[off:off + N] - x1[off]
        d0 = x0[off:off + N] - x0[off]
        assert np.max(np.abs(d1 - d0)) <= 1e-6  # metres; the translation adds rounding at |x| ~ 2.5e7 m
        off += N


def test_transport_matches_oracle_in_dipole():
    """Stage 2 from 4 Earth radii on the equator, dipole B = 3.1e-5 T at 1 Earth radius, dt = 1e-9 s."""
    b = inputs.gaussian_bunch(200, 20e-6, 3.0, seed=5)
    center = np.array([-4 * RE, 0.0, 0.0])
    x_host = b.x - b.x.mean(axis=0) + center  # the same translation, formed on the host for the oracle
    steps = 5000
    run = oracle.Run(x_host, b.u, 4, 1e-9, nmax=steps)
    run.step(steps, bkind=2, bpar=oracle.bext_params(2, m0=M0_CFG), self_on=False)
    with emppp.Solver(200, 8, DT) as s:
        s.set_particles(b.x.copy(), b.u.copy())
        s.handoff(center)
        s.transport(steps, 1e-9, emppp.bext_dipole(M0_CFG))
        x, u, t, n = s.get_state()
        E, B = s.get_fields()
    assert n == steps and abs(t - run.t) <= 1e-15 * run.t
    assert np.all(E == 0.0)
    assert np.max(np.abs(x - run.x)) <= 1e-9 * RE
    assert np.max(np.abs(u - run.u)) <= 1e-9 * np.max(np.abs(run.u))


def test_transport_conserves_speed_in_magnetic_field():
    b = inputs.gaussian_bunch(64, 1e-3, 20.0, seed=6)
    with emppp.Solver(64, 4, DT) as s:
        s.set_particles(b.x.copy() + np.array([-3 * RE, 0.0, 0.0]), b.u.copy())
        s.transport(20000, 1e-8, emppp.bext_dipole(M0_CFG))
        x, u, t, n = s.get_state()
    s0 = np.linalg.norm(b.u, axis=1)
    s1 = np.linalg.norm(u, axis=1)
    assert np.max(np.abs(s1 - s0) / s0) <= 1e-11


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_equals_eager(precision):
    b = inputs.gaussian_bunch(700, 8e-6, 3.0, seed=7)
    stream = torch.cuda.Stream()
    res = []
    for graphs in (False, True):
        with emppp.Solver(700, 16, DT, precision=precision, proposal="closed_form", stream=stream,
                          graphs=graphs) as s:
            s.set_particles(b.x.copy(), b.u.copy())
            s.step(30, emppp.bext_uniform((5e-5, 0.0, 0.0)))
            x, u, _, n = s.get_state()
            st = s.stats()
            res.append((x, u, n, st["kernel_launches"]))
    assert res[0][2] == res[1][2] == 30
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert res[0][3] == res[1][3]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_target_order_refresh_changes_no_result(precision):
    """The spatial target order is recomputed every 16 steps: an older order is still a permutation of the
    bunch, and each target's sum runs over the sources in a fixed order, so 40 replayed steps with the order
    equal 40 with the identity order bit for bit; the ordered run launches the order kernel at steps 0, 16
    and 32 only."""
    b = inputs.gaussian_bunch(3000, 8e-6, 3.0, seed=9)
    stream = torch.cuda.Stream()
    res = []
    for order in (0, 1):
        with emppp.Solver(3000, 64, DT, precision=precision, proposal="closed_form", stream=stream,
                          graphs=True) as s:
            s.set_particles(b.x.copy(), b.u.copy())
            s.set_tuning(items_per_block=16, target_order=order)
            s.reset_stats()
            s.step(40)
            x, u, _, n = s.get_state()
            E, B = s.get_fields()
            res.append((x, u, E, B, s.stats()["kernel_launches"]))
    for k in range(4):
        assert np.array_equal(res[0][k], res[1][k])
    assert res[1][4] - res[0][4] == 3


def test_two_stage_pipeline_batched_equals_single():
    """Stage 1 (mixed, 20 steps) -> handoff to 4 Earth radii -> stage 2 (dipole, 2000 steps) for a small
    batch of bunches, against the same pipeline run bunch by bunch."""
    spec = [(513, 10e-6, 3.0, 11), (256, 40e-6, 12.0, 12), (1024, 5e-6, 2.0, 13)]
    xs, us = _bunches(spec)
    sizes = [x.shape[0] for x in xs]
    center = (-4 * RE, 0.0, 0.0)
    dip = emppp.bext_dipole(M0_CFG)

    def pipeline(solver, x, u):
        solver.set_particles(x, u)
        solver.step(20)
        solver.handoff(center)
        solver.transport(2000, 1e-9, dip)
        return solver.get_state()

    with emppp.Solver(0, 32, DT, precision="mixed", proposal="closed_form", source_split=2, bunches=sizes) as s:
        xb, ub, tb, nb = pipeline(s, np.concatenate(xs), np.concatenate(us))
    off = 0
    for x, u in zip(xs, us):
        N = x.shape[0]
        with emppp.Solver(N, 32, DT, precision="mixed", proposal="closed_form", source_split=2) as s1:
            x1, u1, t1, n1 = pipeline(s1, x.copy(), u.copy())
        assert np.array_equal(xb[off:off + N], x1) and np.array_equal(ub[off:off + N], u1)
        off += N
    assert nb == 2020


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_keeps_state_and_results(precision):
    from gpu_helpers import history_case, window

    h = history_case(3000, 80, sigma=10e-6, seed=21)
    T, W, V, u = window(h, 128)
    # (targets per block, sources per sum, staged history window)
    shapes = [(128, 8, 0), (64, 8, 0), (256, 8, 0)] + ([(128, 16, 0), (128, 32, 0), (128, 32, 1)]
                                                       if precision == "mixed" else [])
    fields = []
    with emppp.Solver(3000, 128, DT, precision=precision, proposal="closed_form") as s:
        s.set_history(80, T, W, V, u)
        rep = s.autotune()
        _, _, t0, n0 = s.get_state()
        # 5 splits x both target orders at the default shape, then the other tile shapes
        assert n0 == 80 and len(rep["candidates"]) == 10 + len(shapes) - 1
        assert all(c["ms"] > 0 for c in rep["candidates"])
        assert {(c["targets_per_block"], c["sources_per_sum"], int(c["history_window"] > 0))
                for c in rep["candidates"]} == set(shapes)
        s.step(1)
        fields.append(s.get_fields())
        for tpb, sps, hw in shapes:
            for ipb, order in ((4, 0), (16, 1)):
                s.set_history(80, T, W, V, u)
                s.set_tuning(items_per_block=ipb, target_order=order, targets_per_block=tpb, sources_per_sum=sps,
                             history_window=hw)
                s.step(1)
                fields.append(s.get_fields())
                st = s.stats()
                assert st["pairs"] == 3000 * 2999
        with pytest.raises(emppp.EmpppError):
            s.set_tuning(targets_per_block=96)
        with pytest.raises(emppp.EmpppError):
            s.set_tuning(targets_per_block=64, sources_per_sum=16)
        with pytest.raises(emppp.EmpppError):
            s.set_tuning(targets_per_block=128, sources_per_sum=64)
    E_ref, B_ref, _, M = oracle.self_fields(h.T, h.W, h.V, 80, 128, mags=True)
    tol = 1e-12 if precision == "fp64" else 1e-5
    for E, B in fields:
        eE, eB = field_errors(E, B, E_ref, B_ref, M)
        assert eE <= tol and eB <= tol
