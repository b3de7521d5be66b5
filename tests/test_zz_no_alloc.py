"""emppp_fields_noalloc: the self-field evaluation for callers that cannot let the library allocate
device memory (their framework's allocator owns the GPU, or they run under a fixed memory budget).

It must give the same fields as the allocating path (emppp_set_history + emppp_step +
emppp_get_fields) within the tolerance of the other GPU tests -- every component within 1e-12 of
sum_j |E_ij| (resp. |B_ij|) of its target -- and keep doing so when it is called again, because its
working memory is one fixed device array that every call reuses. The file is named so that pytest
collects it last; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import DT, field_errors, history_case, window

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2605_05543_gb300 import emppp  # noqa: E402

TOL = 1e-12


def _allocating_path(h, D):
    T, W, V, u = window(h, D)
    with emppp.Solver(W.shape[1], D, DT) as s:
        s.set_history(h.n, T, W, V, u)
        s.step(1)
        return s.get_fields()


def _no_alloc_path(h, D):
    T, W, V, _ = window(h, D)
    dev = torch.device("cuda:0")
    Td, Wd, Vd = (torch.from_numpy(a).to(dev) for a in (T, W, V))
    N = W.shape[1]
    E = torch.full((N, 3), float("nan"), dtype=torch.float64, device=dev)
    B = torch.full_like(E, float("nan"))
    stream = torch.cuda.current_stream()
    emppp.fields_noalloc(Td, Wd, Vd, E, B, stream=stream)
    stream.synchronize()
    return E.cpu().numpy(), B.cpu().numpy()


def test_no_alloc_matches_allocating_path_on_consecutive_calls():
    # two calls in a row with different sizes: the second reuses the scratch the first one left
    cases = [(300, 40, 32, 5e-6, 21), (1000, 200, 128, 10e-6, 22)]
    for N, n, D, sigma, seed in cases:
        h = history_case(N, n, sigma=sigma, seed=seed)
        E_ref, B_ref = _allocating_path(h, D)
        E, B = _no_alloc_path(h, D)
        k0 = max(0, n - D + 1)
        _, _, _, M = oracle.self_fields(h.T[k0:], h.W[k0:], h.V[k0:], n - k0, D, mags=True)
        eE, eB = field_errors(E, B, E_ref, B_ref, M)
        assert eE <= TOL and eB <= TOL, (N, eE, eB)


def test_no_alloc_repeat_is_identical():
    h = history_case(500, 60, seed=23)
    a = _no_alloc_path(h, 64)
    b = _no_alloc_path(h, 64)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    dev = torch.device("cuda:0")
    T = torch.zeros(4097, dtype=torch.float64, device=dev)
    W = torch.zeros(4097, 2, 3, dtype=torch.float64, device=dev)
    E = torch.zeros(2, 3, dtype=torch.float64, device=dev)
    with pytest.raises(emppp.EmpppError) as ei:
        emppp.fields_noalloc(T, W, W, E, E)
    assert ei.value.status == emppp.ERR_ARG
    N = 348161
    T1 = torch.zeros(1, dtype=torch.float64, device=dev)
    W1 = torch.zeros(1, N, 3, dtype=torch.float64, device=dev)
    E1 = torch.zeros(N, 3, dtype=torch.float64, device=dev)
    with pytest.raises(emppp.EmpppError) as ei:
        emppp.fields_noalloc(T1, W1, W1, E1, E1)
    assert ei.value.status == emppp.ERR_ARG
