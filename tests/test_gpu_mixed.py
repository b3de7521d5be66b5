"""Mixed-precision CUDA path against the FP64 oracle on seeded inputs (GB300).

Bar: every field component within 1e-5 of sum_j |E_ij| (resp. |B_ij|) of its target; the bracket of
every pair equal to the FP64 one (branch counts equal the oracle's exactly, because the FP32 node
test defers to the FP64 test inside its guard band); positions within 1e-9 of the bunch size after a
full run. The achieved error of each case is printed (pytest -s) and kept in the assertion message.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import DT, field_errors, gpu_fields_from_history, history_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2605_05543_gb300 import emppp, inputs  # noqa: E402

MIXED_TOL = 1e-5

CASES = [
    (2, 0, 16, 1e-6, 0),
    (3, 5, 16, 0.3e-6, 1),
    (17, 40, 32, 2e-6, 2),
    (129, 12, 64, 1e-6, 3),
    (256, 100, 64, 10e-6, 4),
    (300, 30, 256, 5e-6, 5),
    (1000, 600, 512, 10e-6, 6),
    (4096, 300, 512, 10e-6, 7),
]


@pytest.mark.parametrize("proposal", ["bisect", "closed_form"])
@pytest.mark.parametrize("N,n,D,sigma,seed", CASES)
def test_mixed_fields_match_fp64_oracle(N, n, D, sigma, seed, proposal):
    h = history_case(N, n, sigma=sigma, seed=seed)
    E_ref, B_ref, st_ref, M = oracle.self_fields(h.T, h.W, h.V, n, D, mags=True)
    E, B, st, x, u = gpu_fields_from_history(emppp.Solver, h, D, precision="mixed", proposal=proposal)
    eE, eB = field_errors(E, B, E_ref, B_ref, M)
    print(f"mixed N={N} n={n} D={D} {proposal}: err E {eE:.2e} B {eB:.2e}, guard fallbacks "
          f"{st['guard_fallbacks']} of {st['node_tests']} node tests")
    assert eE <= MIXED_TOL and eB <= MIXED_TOL, (eE, eB)
    for k in ("out_of_history", "shortcut", "bisection"):
        assert st[k] == st_ref[k], (k, st, st_ref)
    if proposal == "bisect":
        assert st["node_tests"] == st_ref["node_tests"]


@pytest.mark.parametrize("shape", [(128, 8), (128, 32)])
def test_mixed_full_size_sampled_targets(shape):
    """N = 65536, sigma = 20 um, depth 1024, 251-slot history: the benchmark's workload, at the default
    tile shape and at the one the benchmark's autotuner chooses (128 targets per block, 32 sources per
    FP32 partial sum)."""
    N, n, D = 65536, 250, 1024
    h = history_case(N, n, sigma=20e-6, seed=0)
    tuning = dict(items_per_block=16, target_order=1, targets_per_block=shape[0], sources_per_sum=shape[1])
    E, B, st, x, u = gpu_fields_from_history(emppp.Solver, h, D, tuning=tuning, precision="mixed",
                                             proposal="closed_form")
    rng = np.random.default_rng(1)
    tg = np.unique(np.concatenate([[0, N - 1], rng.choice(N, 62, replace=False)]))
    E_ref, B_ref, _, M = oracle.self_fields(h.T, h.W, h.V, n, D, targets=tg, mags=True)
    eE, eB = field_errors(E[tg], B[tg], E_ref, B_ref, M)
    print(f"mixed N=65536: err E {eE:.2e} B {eB:.2e}; fallbacks {st['guard_fallbacks']} / {st['node_tests']}")
    assert eE <= MIXED_TOL and eB <= MIXED_TOL, (eE, eB)


def test_mixed_full_run_positions():
    """N = 256, sigma = 10 um, gamma0 = 3, 200 steps, depth 256: positions against the FP64 oracle."""
    b = inputs.gaussian_bunch(256, 10e-6, 3.0, seed=0)
    run = oracle.Run(b.x, b.u, 256, DT, nmax=200)
    run.step(200)
    with emppp.Solver(256, 256, DT, precision="mixed", proposal="closed_form") as s:
        s.set_particles(b.x.copy(), b.u.copy())
        s.step(200)
        x, u, t, n = s.get_state()
        E, B = s.get_fields()
    sig = float(np.sqrt(np.mean(np.sum((run.x - run.x.mean(axis=0)) ** 2, axis=1))))
    err_x = np.max(np.linalg.norm(x - run.x, axis=1)) / sig
    scale = np.max(np.abs(run.E))
    err_E = np.max(np.abs(E - run.E)) / scale
    print(f"mixed 256x200: position err {err_x:.2e} of sigma, last-step field err {err_E:.2e} of max |E|")
    assert err_x <= 1e-9
    assert err_E <= 1e-4


def test_mixed_uniform_field_with_wrap():
    b = inputs.gaussian_bunch(512, 10e-6, 3.0, seed=2)
    par = oracle.bext_params(1, b=(5e-5, 0.0, 0.0))
    run = oracle.Run(b.x, b.u, 32, DT, nmax=80)
    run.step(80, bkind=1, bpar=par)
    with emppp.Solver(512, 32, DT, precision="mixed") as s:
        s.set_particles(b.x.copy(), b.u.copy())
        s.step(80, emppp.bext_uniform((5e-5, 0.0, 0.0)))
        x, u, t, n = s.get_state()
    sig = float(np.sqrt(np.mean(np.sum((run.x - run.x.mean(axis=0)) ** 2, axis=1))))
    assert np.max(np.linalg.norm(x - run.x, axis=1)) / sig <= 1e-9


def test_mixed_and_fp64_paths_agree():
    h = history_case(2000, 150, sigma=8e-6, seed=31)
    E64, B64, st64, _, _ = gpu_fields_from_history(emppp.Solver, h, 256)
    E32, B32, st32, _, _ = gpu_fields_from_history(emppp.Solver, h, 256, precision="mixed")
    _, _, _, M = oracle.self_fields(h.T, h.W, h.V, 150, 256, mags=True)
    eE, eB = field_errors(E32, B32, E64, B64, M)
    assert eE <= MIXED_TOL and eB <= MIXED_TOL
    for k in ("out_of_history", "shortcut", "bisection", "node_tests"):
        assert st32[k] == st64[k]
