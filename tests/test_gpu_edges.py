"""Edge cases of the CUDA path against the oracle (GB300): tiny and ragged bunches in one batch, the
smallest history depth, and a bunch spread so wide that the mixed path's FP32 split cannot hold it.

Bar: FP64 fields within 1e-12 of sum_j |E_ij|, mixed within 1e-5, branch counts equal to the oracle's,
positions within 1e-9 of the bunch size after full runs.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import DT, field_errors, history_case, light_sphere_case, window

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2605_05543_gb300 import emppp, inputs  # noqa: E402

TOL = {"fp64": 1e-12, "mixed": 1e-5}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("proposal", ["bisect", "closed_form"])
def test_tiny_and_ragged_bunches_in_one_batch(precision, proposal):
    """Bunches of 1, 2, 3, 129 and 130 particles share one launch; each gets its own oracle fields (the
    single particle none), and the batch's branch counts are the sum of the oracle's."""
    spec = [(1, 1e-6, 3.0, 31), (2, 1e-6, 3.0, 32), (3, 2e-6, 5.0, 33), (129, 5e-6, 3.0, 34), (130, 8e-6, 2.0, 35)]
    n, D = 30, 16
    hs = [history_case(N, n, sigma=s, gamma0=g, seed=sd) for N, s, g, sd in spec]
    wins = [window(h, D) for h in hs]
    W = np.ascontiguousarray(np.concatenate([w[1] for w in wins], axis=1))
    V = np.ascontiguousarray(np.concatenate([w[2] for w in wins], axis=1))
    u = np.concatenate([w[3] for w in wins])
    with emppp.Solver(0, D, DT, precision=precision, proposal=proposal, bunches=[N for N, *_ in spec]) as s:
        s.set_history(n, wins[0][0], W, V, u)
        s.step(1)
        E, B = s.get_fields()
        st = s.stats()
    off, counts = 0, dict(out_of_history=0, shortcut=0, bisection=0)
    for (N, *_), h in zip(spec, hs):
        E_ref, B_ref, st_ref, M = oracle.self_fields(h.T, h.W, h.V, n, D, mags=True)
        if N == 1:
            assert np.all(E[off] == 0.0) and np.all(B[off] == 0.0)
        else:
            eE, eB = field_errors(E[off:off + N], B[off:off + N], E_ref, B_ref, M)
            assert eE <= TOL[precision] and eB <= TOL[precision], (N, eE, eB)
        for k in counts:
            counts[k] += st_ref[k]
        off += N
    for k in counts:
        assert st[k] == counts[k], (k, st, counts)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_smallest_history_depth(precision):
    """Depth 2 (the present slot and one more): 12 steps of free expansion against the oracle."""
    b = inputs.gaussian_bunch(100, 2e-6, 3.0, seed=36)
    run = oracle.Run(b.x, b.u, 2, DT, nmax=12)
    run.step(12)
    with emppp.Solver(100, 2, DT, precision=precision) as s:
        s.set_particles(b.x.copy(), b.u.copy())
        s.step(12)
        x, u, t, n = s.get_state()
        E, B = s.get_fields()
    sig = float(np.sqrt(np.mean(np.sum((run.x - run.x.mean(axis=0)) ** 2, axis=1))))
    assert np.max(np.linalg.norm(x - run.x, axis=1)) / sig <= (1e-9 if precision == "fp64" else 1e-6)
    scale = np.max(np.linalg.norm(run.E, axis=1))
    assert np.max(np.abs(E - run.E)) <= TOL[precision] * scale * 100


def test_mixed_path_far_from_the_split_origin():
    """Particles spread over 1.5 m: beyond 0.5 m from the bunch's FP32 split origin the mixed path takes
    every node test in FP64, and its brackets and fields still follow the oracle."""
    b = inputs.gaussian_bunch(64, 2e-6, 3.0, seed=37)
    x = b.x.copy()
    x[32:] += np.array([1.5, 0.0, 0.0])  # a second cluster 1.5 m away
    h = inputs.synthetic_history(x, b.u, 20, DT, seed=38)
    D = 32
    E_ref, B_ref, st_ref, M = oracle.self_fields(h.T, h.W, h.V, 20, D, mags=True)
    T, W, V, u = window(h, D)
    with emppp.Solver(64, D, DT, precision="mixed", proposal="closed_form") as s:
        s.set_history(20, T, W, V, u)
        s.step(1)
        E, B = s.get_fields()
        st = s.stats()
    eE, eB = field_errors(E, B, E_ref, B_ref, M)
    assert eE <= 1e-5 and eB <= 1e-5, (eE, eB)
    for k in ("out_of_history", "shortcut", "bisection"):
        assert st[k] == st_ref[k]
    assert st["guard_fallbacks"] > 0  # the far cluster's tests ran in FP64


@pytest.mark.parametrize("oldest", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("proposal", ["bisect", "closed_form"])
def test_node_tests_at_the_light_sphere(precision, proposal, oldest):
    """Targets placed on the light sphere of one stored slot of their source, to within 1e-16 to 1e-12 of
    its radius (64 two-particle bunches in one batch): every such node test falls inside the FP32 guard
    band, the FP64 test decides it, and the brackets must be the oracle's (branch counts equal) with
    fields within each path's bar. With oldest the slot is the oldest one and the target lies ahead of
    the source: the mixed path's oldest-slot bound must leave those tests to the guard band."""
    C = oracle.constants()["c"]
    n, D, nb = 40, 64, 64
    T, W, V, u = light_sphere_case(nb, n, oldest=oldest)
    with emppp.Solver(0, D, DT, precision=precision, proposal=proposal, bunches=[2] * nb) as s:
        s.set_history(n, T, W, V, u)
        s.step(1)
        E, B = s.get_fields()
        st = s.stats()
    counts = dict(out_of_history=0, shortcut=0, bisection=0)
    tol = 1e-12 if precision == "fp64" else 1e-5
    for b in range(nb):
        sl = slice(2 * b, 2 * b + 2)
        E_ref, B_ref, st_ref, M = oracle.self_fields(T, W[:, sl], V[:, sl], n, D, mags=True)
        # the resting target's own B at the source is zero up to rounding: B is measured against the
        # E scale (over c) where sum_j |B_ij| is only that rounding
        M = M.copy()
        M[:, 1] = np.maximum(M[:, 1], M[:, 0] / C)
        eE, eB = field_errors(E[sl], B[sl], E_ref, B_ref, M)
        assert eE <= tol and eB <= tol, (b, eE, eB)
        for key in counts:
            counts[key] += st_ref[key]
    for key in counts:
        assert st[key] == counts[key], (key, st, counts)
    assert st["guard_fallbacks"] >= nb // 2  # the band was exercised
