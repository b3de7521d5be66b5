"""FP64 CUDA path against the FP64 oracle, element by element, on seeded inputs (GB300).

Bar: every field component within 1e-12 of sum_j |E_ij| (resp. |B_ij|) of its target, identical
bracket decisions (branch counts equal the oracle's exactly), positions within 1e-9 of the bunch
size after the stated step counts.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import DT, field_errors, gpu_fields_from_history, history_case, oracle_step_from_history, window

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2605_05543_gb300 import emppp, inputs  # noqa: E402

FIELD_TOL = 1e-12
POS_TOL = 1e-9

# (N, n, D, sigma, seed): several 128-target tiles with ragged tails, every branch, ring wrap
CASES = [
    (2, 0, 16, 1e-6, 0),
    (3, 5, 16, 0.3e-6, 1),
    (17, 40, 32, 2e-6, 2),
    (129, 12, 64, 1e-6, 3),
    (256, 100, 64, 10e-6, 4),
    (300, 30, 256, 5e-6, 5),
    (1000, 600, 512, 10e-6, 6),
]


@pytest.mark.parametrize("proposal", ["bisect", "closed_form"])
@pytest.mark.parametrize("N,n,D,sigma,seed", CASES)
def test_fields_match_oracle(N, n, D, sigma, seed, proposal):
    h = history_case(N, n, sigma=sigma, seed=seed)
    E_ref, B_ref, st_ref, M = oracle.self_fields(h.T, h.W, h.V, n, D, mags=True)
    E, B, st, x, u = gpu_fields_from_history(emppp.Solver, h, D, proposal=proposal)
    eE, eB = field_errors(E, B, E_ref, B_ref, M)
    assert eE <= FIELD_TOL and eB <= FIELD_TOL, (eE, eB)
    for k in ("out_of_history", "shortcut", "bisection"):
        assert st[k] == st_ref[k], (k, st, st_ref)
    if proposal == "bisect":
        assert st["node_tests"] == st_ref["node_tests"]
    # the push from these fields
    run = oracle_step_from_history(h, D)
    scale = max(sigma, 1e-9)
    assert np.max(np.abs(x - run.x)) <= 1e-12 * scale
    assert np.max(np.abs(u - run.u)) <= 1e-12 * np.max(np.abs(run.u))


@pytest.mark.parametrize("split", [1, 3, 7])
def test_source_split_gives_same_fields(split):
    h = history_case(300, 50, sigma=5e-6, seed=9)
    E_ref, B_ref, _, M = oracle.self_fields(h.T, h.W, h.V, 50, 64, mags=True)
    E, B, st, _, _ = gpu_fields_from_history(emppp.Solver, h, 64, source_split=split)
    eE, eB = field_errors(E, B, E_ref, B_ref, M)
    assert eE <= FIELD_TOL and eB <= FIELD_TOL


def test_deterministic_repeat():
    h = history_case(500, 80, seed=10)
    a = gpu_fields_from_history(emppp.Solver, h, 128)
    b = gpu_fields_from_history(emppp.Solver, h, 128)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[3], b[3])


def _run_both(N, sigma, gamma0, D, steps, bkind=0, b=(0.0, 0.0, 0.0), m0=0.0, seed=0, dt=DT, pair_fields=True,
              center=(0.0, 0.0, 0.0), proposal="bisect"):
    bunch = inputs.gaussian_bunch(N, sigma, gamma0, seed=seed, center=center)
    par = oracle.bext_params(bkind, b=b, m0=m0)
    run = oracle.Run(bunch.x, bunch.u, D, dt, nmax=steps)
    run.step(steps, bkind=bkind, bpar=par, self_on=pair_fields)
    bext = [emppp.bext_none(), emppp.bext_uniform(b), emppp.bext_dipole(m0)][bkind]
    with emppp.Solver(N, D, dt, pair_fields=pair_fields, proposal=proposal) as s:
        s.set_particles(bunch.x.copy(), bunch.u.copy())
        s.step(steps, bext)
        x, u, t, n = s.get_state()
        E, B = s.get_fields()
    return run, x, u, t, n, E, B


def _sigma_rms(x):
    return float(np.sqrt(np.mean(np.sum((x - x.mean(axis=0)) ** 2, axis=1))))


def test_free_expansion_256_full_run():
    """N = 256, sigma = 10 um, gamma0 = 3, no external field, dt = 1e-15 s, 200 steps, depth 256."""
    run, x, u, t, n, E, B = _run_both(256, 10e-6, 3.0, 256, 200)
    assert n == 200 and t == run.t
    err = np.max(np.linalg.norm(x - run.x, axis=1)) / _sigma_rms(run.x)
    assert err <= POS_TOL, err
    assert np.max(np.abs(u - run.u)) <= 1e-9 * np.max(np.abs(run.u))


def test_uniform_field_run_with_ring_wrap():
    """N = 512 in B = 5e-5 T along x, depth 32 so that the ring wraps many times."""
    run, x, u, t, n, E, B = _run_both(512, 10e-6, 3.0, 32, 80, bkind=1, b=(5e-5, 0.0, 0.0), seed=2,
                                      proposal="closed_form")
    err = np.max(np.linalg.norm(x - run.x, axis=1)) / _sigma_rms(run.x)
    assert err <= POS_TOL, err
    scale = np.max(np.abs(run.B))
    assert np.max(np.abs(B - run.B)) <= 1e-12 * scale


def test_dipole_transport_without_pair_fields():
    """Stage-2 style: pair fields off, centred dipole with B = 3.1e-5 T at 1 Earth radius, bunch at
    4 Earth radii on the equator moving along +z, dt = 1e-9 s, 2000 steps."""
    RE = inputs.R_EARTH
    m0 = 3.1e-5 * 4 * math.pi * RE ** 3 / 1.25663706212e-6
    run, x, u, t, n, E, B = _run_both(64, 20e-6, 3.0, 4, 2000, bkind=2, m0=m0, dt=1e-9, pair_fields=False,
                                      center=(-4 * RE, 0.0, 0.0), seed=3)
    assert np.all(E == 0.0)
    assert np.max(np.abs(x - run.x)) <= 1e-9 * RE
    assert np.max(np.abs(u - run.u)) <= 1e-9 * np.max(np.abs(run.u))
    assert np.max(np.abs(B - run.B)) <= 1e-12 * np.max(np.abs(run.B))


@pytest.mark.parametrize("shape", [(128, 8), (64, 8)])
def test_full_size_sampled_targets(shape):
    """N = 65536, sigma = 20 um, gamma0 = 3, depth 1024, history of 251 slots: the benchmark's workload,
    at the default tile shape and at (64, 8), which the autotuner can choose on the FP64 path. The oracle
    evaluates 48 sampled targets against all sources."""
    N, n, D = 65536, 250, 1024
    h = history_case(N, n, sigma=20e-6, seed=0)
    tuning = dict(items_per_block=16, target_order=1, targets_per_block=shape[0], sources_per_sum=shape[1])
    E, B, st, x, u = gpu_fields_from_history(emppp.Solver, h, D, tuning=tuning, proposal="closed_form")
    rng = np.random.default_rng(0)
    tg = np.unique(np.concatenate([[0, 1, N - 1], rng.choice(N, 45, replace=False)]))
    E_ref, B_ref, st_ref, M = oracle.self_fields(h.T, h.W, h.V, n, D, targets=tg, mags=True)
    eE, eB = field_errors(E[tg], B[tg], E_ref, B_ref, M)
    assert eE <= FIELD_TOL and eB <= FIELD_TOL, (eE, eB)
    assert st["pairs"] == N * (N - 1)
    assert st["out_of_history"] + st["shortcut"] + st["bisection"] == N * (N - 1)


def test_single_particle_has_no_self_field():
    b = inputs.gaussian_bunch(1, 1e-6, 3.0, seed=0)
    with emppp.Solver(1, 8, DT) as s:
        s.set_particles(b.x.copy(), b.u.copy())
        s.step(3)
        E, B = s.get_fields()
        st = s.stats()
    assert np.all(E == 0) and np.all(B == 0) and st["pairs"] == 0


def test_device_pointer_inputs_and_outputs():
    h = history_case(200, 30, seed=11)
    T, W, V, u = window(h, 64)
    dev = torch.device("cuda:0")
    with emppp.Solver(200, 64, DT, stream=torch.cuda.current_stream()) as s:
        s.set_history(30, *(torch.from_numpy(a).to(dev) for a in (T, W, V, u)))
        s.step(1)
        Ed = torch.zeros(200, 3, dtype=torch.float64, device=dev)
        Bd = torch.zeros_like(Ed)
        s.get_fields(Ed, Bd)
        xd = torch.zeros_like(Ed)
        ud = torch.zeros_like(Ed)
        s.get_state(xd, ud)
        Eh, Bh = s.get_fields()
    assert np.array_equal(Ed.cpu().numpy(), Eh)
    E_ref, B_ref, _, M = oracle.self_fields(h.T, h.W, h.V, 30, 64, mags=True)
    assert field_errors(Eh, Bh, E_ref, B_ref, M)[0] <= FIELD_TOL


def test_history_round_trip():
    h = history_case(100, 70, seed=12)
    T, W, V, u = window(h, 32)
    with emppp.Solver(100, 32, DT) as s:
        s.set_history(70, T, W, V, u)
        n, T2, W2, V2, u2 = s.get_history()
        assert n == 70 and np.array_equal(T2, T) and np.array_equal(W2, W) and np.array_equal(V2, V)
        s.step(5)
        n, T3, W3, V3, u3 = s.get_history()
        x, uu, t, nn = s.get_state()
    assert n == 75 and T3.shape[0] == 32 and np.array_equal(W3[-1], x)


def test_resume_is_bitwise_identical():
    b = inputs.gaussian_bunch(300, 5e-6, 3.0, seed=13)
    with emppp.Solver(300, 16, DT) as s:
        s.set_particles(b.x.copy(), b.u.copy())
        s.step(40)
        x_ref, u_ref, _, _ = s.get_state()
    with emppp.Solver(300, 16, DT) as s:
        s.set_particles(b.x.copy(), b.u.copy())
        s.step(25)
        ckpt = s.get_history()
    with emppp.Solver(300, 16, DT) as s2:
        n, T, W, V, u = ckpt
        s2.set_history(n, T, W, V, u)
        s2.step(15)
        x, uu, _, _ = s2.get_state()
    assert np.array_equal(x, x_ref) and np.array_equal(uu, u_ref)


# ---- error paths: numeric faults are flagged by the kernels and reported, never trapped --------
def test_coincident_particles_reported():
    x = np.zeros((2, 3))
    u = np.array([[0.0, 0.0, 1e8], [0.0, 0.0, 1e8]])
    with emppp.Solver(2, 8, DT) as s:
        s.set_particles(x, u)
        s.step(1)
        with pytest.raises(emppp.EmpppError) as ei:
            s.get_fields()
    assert ei.value.status == emppp.ERR_NUMERIC


def test_superluminal_history_reported():
    h = history_case(8, 10, seed=14)
    T, W, V, u = window(h, 16)
    V = V.copy()
    V[:, 3] *= 1.2 * inputs.C_LIGHT / np.linalg.norm(V[:, 3], axis=1, keepdims=True)
    with emppp.Solver(8, 16, DT) as s:
        s.set_history(10, T, W, V, u)
        s.step(1)
        with pytest.raises(emppp.EmpppError) as ei:
            s.synchronize()
    assert ei.value.status == emppp.ERR_NUMERIC


def test_argument_errors():
    with pytest.raises(emppp.EmpppError) as ei:
        emppp.Solver(0, 8, DT)
    assert ei.value.status == emppp.ERR_ARG
    with pytest.raises(emppp.EmpppError):
        emppp.Solver(8, 1, DT)
    with pytest.raises(emppp.EmpppError):
        emppp.Solver(8, 8, -1.0)
    with emppp.Solver(8, 8, DT) as s:
        with pytest.raises(emppp.EmpppError) as ei:
            s.step(1)
        assert ei.value.status == emppp.ERR_STATE
        h = history_case(8, 3, seed=15)
        T, W, V, u = window(h, 8)
        with pytest.raises(emppp.EmpppError):
            s.set_history(3, T[::-1].copy(), W, V, u)  # time stamps not increasing
