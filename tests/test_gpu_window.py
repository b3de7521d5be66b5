"""Staged history windows of the mixed pair kernel (GB300): each warp copies, one source ahead, the run of
history slots its targets' guessed brackets of the next source fall in (Sec. 2.2 node reads) from the FP32
ring into shared memory by bulk copy, and reads the predicted bracket's two records there.

The window changes where records are read, not the search or the arithmetic, and it splits the work like
the same tile shape without it. So against (128 targets, 32 sources per sum) without the window, on the
same state:
  - the fields are identical bit for bit, and the branch and node-test counts are equal;
  - both agree with the FP64 oracle within the mixed path's 1e-5 of sum_j |F_ij|.
Cases: several target tiles with a ragged tail, a ring window that has wrapped (copies in two runs), an
untrained learned proposal (guesses all over the history, windows cut at their slot limit), targets on the
light sphere of a stored slot, a single-slot history (nothing to stage), and the benchmark's N = 65536
workload.
A wait limit of zero makes every warp's first wait give up: the kernel then gathers from the ring, the
fields stay identical and the next status read is EMPPP_ERR_TIMEOUT.
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

STAT_KEYS = ("pairs", "out_of_history", "shortcut", "bisection", "node_tests", "guard_fallbacks")


def _fields(T, W, V, u, n, D, proposal, window_on, bunches=None, wait_limit=None):
    N = W.shape[1]
    with emppp.Solver(N if bunches is None else 0, D, DT, precision="mixed", proposal=proposal,
                      bunches=bunches) as s:
        s.set_history(n, T, W, V, u)
        if proposal == "mlp":
            s.set_proposal(inputs.mlp_init_params(5))
        s.set_tuning(items_per_block=16, target_order=1, targets_per_block=128, sources_per_sum=32,
                     history_window=1 if window_on else 0)
        if wait_limit is not None:
            s.set_wait_limit(wait_limit)
        s.reset_stats()
        s.step(1)
        status = emppp.OK
        try:
            s.get_state()
        except emppp.EmpppError as e:
            status = e.status
        E, B = s.get_fields()
        st = s.stats()
        return E, B, {k: st[k] for k in STAT_KEYS}, status


CASES = {
    # N, n, D, sigma: 2 tiles + ragged tail; a wrapped ring (n > D); a deep history of a small bunch
    "tiles": (300, 60, 128, 10e-6),
    "wrapped": (517, 90, 48, 5e-6),
    "deep": (200, 250, 256, 20e-6),
}


@pytest.mark.parametrize("proposal", ["closed_form", "mlp"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_window_fields_identical_and_match_oracle(case, proposal):
    N, n, D, sigma = CASES[case]
    h = history_case(N, n, sigma=sigma, seed=31 + N)
    T, W, V, u = window(h, D)
    E0, B0, s0, st0 = _fields(T, W, V, u, n, D, proposal, False)
    E1, B1, s1, st1 = _fields(T, W, V, u, n, D, proposal, True)
    assert st0 == emppp.OK and st1 == emppp.OK
    assert np.array_equal(E0, E1) and np.array_equal(B0, B1)
    assert s0 == s1
    E_ref, B_ref, _, M = oracle.self_fields(h.T, h.W, h.V, n, D, mags=True)
    eE, eB = field_errors(E1, B1, E_ref, B_ref, M)
    assert eE <= 1e-5 and eB <= 1e-5, (eE, eB)


def test_window_light_sphere_and_single_slot():
    T, W, V, u = light_sphere_case()
    n = T.shape[0] - 1
    sizes = [2] * (W.shape[1] // 2)
    E0, B0, s0, _ = _fields(T, W, V, u, n, 64, "closed_form", False, bunches=sizes)
    E1, B1, s1, _ = _fields(T, W, V, u, n, 64, "closed_form", True, bunches=sizes)
    assert np.array_equal(E0, E1) and np.array_equal(B0, B1) and s0 == s1
    assert s1["guard_fallbacks"] > 0
    # a single stored slot: every pair is out of history, no window is staged
    h = history_case(300, 0, seed=5)
    T, W, V, u = window(h, 16)
    E0, B0, s0, _ = _fields(T, W, V, u, 0, 16, "closed_form", False)
    E1, B1, s1, _ = _fields(T, W, V, u, 0, 16, "closed_form", True)
    assert np.array_equal(E0, E1) and np.array_equal(B0, B1) and s0 == s1
    assert s1["out_of_history"] == s1["pairs"]


def test_window_wait_limit_zero_reports_timeout_with_exact_fields():
    N, n, D, sigma = CASES["tiles"]
    h = history_case(N, n, sigma=sigma, seed=31 + N)
    T, W, V, u = window(h, D)
    E0, B0, s0, _ = _fields(T, W, V, u, n, D, "closed_form", False)
    E1, B1, s1, st = _fields(T, W, V, u, n, D, "closed_form", True, wait_limit=0)
    assert st == emppp.ERR_TIMEOUT
    assert np.array_equal(E0, E1) and np.array_equal(B0, B1) and s0 == s1
    # the status is reported once; the next step with the default limit runs clean
    with emppp.Solver(N, D, DT, precision="mixed", proposal="closed_form") as s:
        s.set_history(n, T, W, V, u)
        s.set_tuning(targets_per_block=128, sources_per_sum=32, history_window=1)
        s.set_wait_limit(0)
        s.step(1)
        with pytest.raises(emppp.EmpppError) as e:
            s.get_state()
        assert e.value.status == emppp.ERR_TIMEOUT
        s.set_history(n, T, W, V, u)
        s.set_wait_limit(1 << 16)
        s.step(1)
        s.get_state()
        E2, B2 = s.get_fields()
    assert np.array_equal(E0, E2) and np.array_equal(B0, B2)
    with emppp.Solver(N, D, DT, precision="mixed") as s:
        with pytest.raises(emppp.EmpppError):
            s.set_wait_limit(-1)


def test_window_requires_its_shape():
    with emppp.Solver(300, 16, DT, precision="mixed") as s:
        for tpb, sps in ((128, 8), (64, 8), (256, 8), (128, 16)):
            with pytest.raises(emppp.EmpppError):
                s.set_tuning(targets_per_block=tpb, sources_per_sum=sps, history_window=1)
        s.set_tuning(targets_per_block=128, sources_per_sum=32, history_window=1)


def test_window_full_size_identical():
    """N = 65536, depth 1024, 251-slot history (the benchmark's workload, where the autotuner times the window
    instance): fields and counts equal to (128, 32) without the window, bit for bit."""
    N, n, D = 65536, 250, 1024
    h = history_case(N, n, sigma=20e-6, seed=0)
    T, W, V, u = window(h, D)
    E0, B0, s0, st0 = _fields(T, W, V, u, n, D, "closed_form", False)
    E1, B1, s1, st1 = _fields(T, W, V, u, n, D, "closed_form", True)
    assert st0 == emppp.OK and st1 == emppp.OK
    assert np.array_equal(E0, E1) and np.array_equal(B0, B1) and s0 == s1
