"""emppp_fields_noalloc: the self-field evaluation for callers that cannot let the library allocate
device memory (their framework's allocator owns the GPU, or they run under a fixed memory budget).

It must give the fields of the FP64 oracle and of the allocating path (emppp_set_history + emppp_step +
emppp_get_fields) within the tolerance of the other GPU tests -- every component within 1e-12 of
sum_j |E_ij| (resp. |B_ij|) of its target -- and keep doing so when it is called again, because its
working memory is one fixed device array that every call reuses; a call must leave the device's free
memory unchanged. The file is named so that pytest collects it last; it also passes when run alone in
a fresh process.
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


def _allocating_path(h, D, w=None):
    T, W, V, u = window(h, D)
    with emppp.Solver(W.shape[1], D, DT) as s:
        s.set_history(h.n, T, W, V, u, w=None if w is None else w.copy())
        s.step(1)
        return s.get_fields()


def _device_inputs(h, D, w=None):
    T, W, V, _ = window(h, D)
    dev = torch.device("cuda:0")
    Td, Wd, Vd = (torch.from_numpy(a).to(dev) for a in (T, W, V))
    wd = None if w is None else torch.from_numpy(w).to(dev)
    N = W.shape[1]
    E = torch.full((N, 3), float("nan"), dtype=torch.float64, device=dev)
    B = torch.full_like(E, float("nan"))
    return Td, Wd, Vd, wd, E, B


def _no_alloc_path(h, D, w=None):
    Td, Wd, Vd, wd, E, B = _device_inputs(h, D, w)
    stream = torch.cuda.current_stream()
    emppp.fields_noalloc(Td, Wd, Vd, E, B, w=wd, stream=stream)
    stream.synchronize()
    return E.cpu().numpy(), B.cpu().numpy()


def _oracle(h, D, w=None):
    k0 = max(0, h.n - D + 1)
    return oracle.self_fields(h.T[k0:], h.W[k0:], h.V[k0:], h.n - k0, D, weights=w, mags=True)


def test_no_alloc_matches_oracle_and_allocating_path_on_consecutive_calls():
    # two calls in a row with different sizes: the second reuses the scratch the first one left
    cases = [(300, 40, 32, 5e-6, 21), (1000, 200, 128, 10e-6, 22)]
    for N, n, D, sigma, seed in cases:
        h = history_case(N, n, sigma=sigma, seed=seed)
        E_alloc, B_alloc = _allocating_path(h, D)
        E, B = _no_alloc_path(h, D)
        E_ref, B_ref, _, M = _oracle(h, D)
        eE, eB = field_errors(E, B, E_ref, B_ref, M)
        assert eE <= TOL and eB <= TOL, ("oracle", N, eE, eB)
        eE, eB = field_errors(E, B, E_alloc, B_alloc, M)
        assert eE <= TOL and eB <= TOL, ("allocating path", N, eE, eB)


def test_no_alloc_with_weights():
    N, n, D = 257, 50, 64
    h = history_case(N, n, sigma=5e-6, seed=24)
    w = np.random.default_rng(24).uniform(0.5, 3.0, N)
    E, B = _no_alloc_path(h, D, w)
    E_ref, B_ref, _, M = _oracle(h, D, w)
    assert max(field_errors(E, B, E_ref, B_ref, M)) <= TOL
    E_alloc, B_alloc = _allocating_path(h, D, w)
    assert max(field_errors(E, B, E_alloc, B_alloc, M)) <= TOL


def test_no_alloc_leaves_free_device_memory_unchanged():
    h = history_case(2000, 100, sigma=10e-6, seed=25)
    Td, Wd, Vd, wd, E, B = _device_inputs(h, 128)
    stream = torch.cuda.current_stream()
    emppp.fields_noalloc(Td, Wd, Vd, E, B, stream=stream)  # first call: module load and address look-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    E1 = E.clone()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        emppp.fields_noalloc(Td, Wd, Vd, E, B, stream=stream)
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 == free1, (free0, free1, free2)
    assert torch.equal(E, E1)


def test_no_alloc_repeat_is_identical():
    h = history_case(500, 60, seed=23)
    a = _no_alloc_path(h, 64)
    b = _no_alloc_path(h, 64)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("nslots", [1, 2])
def test_no_alloc_shortest_histories(nslots):
    N = 130
    h = history_case(N, nslots - 1, sigma=3e-6, seed=26)
    E, B = _no_alloc_path(h, nslots)
    E_ref, B_ref, _, M = _oracle(h, nslots)
    assert max(field_errors(E, B, E_ref, B_ref, M)) <= TOL


@pytest.mark.parametrize("nslots", [1, 2])
def test_no_alloc_non_finite_position_gives_nan_fields(nslots):
    """A NaN position (a fault of the caller's state) makes the fields of the targets that see it NaN; the
    call still returns OK, and the next call on valid input is correct."""
    N = 64
    h = history_case(N, nslots - 1, sigma=3e-6, seed=27)
    bad = history_case(N, nslots - 1, sigma=3e-6, seed=27)
    bad.W[:, 5, 1] = np.nan  # in every slot, so that no bracket of particle 5 is finite
    E, B = _no_alloc_path(bad, nslots)
    assert np.all(np.isnan(E)) and np.all(np.isnan(B))  # every target sees particle 5 (or is particle 5)
    E, B = _no_alloc_path(h, nslots)
    E_ref, B_ref, _, M = _oracle(h, nslots)
    assert max(field_errors(E, B, E_ref, B_ref, M)) <= TOL


def test_no_alloc_rejects_sizes_beyond_its_scratch_and_mixed_devices():
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
    with pytest.raises(ValueError):
        emppp.fields_noalloc(T.cpu(), W, W, E, E)
