"""Per-pair identity of the retarded-time brackets (Sec. 2.2) with the oracle's search (GB300).

emppp_bracket_dump writes, for every ordered pair of the present state, the bracket the pair kernel
found: 4 (k1 - k0) + branch. The oracle's bracket table runs the paper's search (out-of-history test,
near-field shortcut, bisection) in FP64 for the same pairs. Every proposal and both precisions must give
that table exactly -- zero mismatches -- which aggregate branch counts alone cannot show (two compensating
flips, or a flip to an adjacent slot, leave every count unchanged). Cases: several target tiles with
ragged tails, a ring window that has wrapped, a single-slot history, a learned proposal with an untrained
network (starting slots all over the history), targets on the light sphere of a stored slot (every such
test decided inside the FP32 guard band; also of the oldest slot, ahead of the source, where the mixed
path's oldest-slot bound is tried), and a bunch whose far cluster the FP32 split cannot hold.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import DT, history_case, light_sphere_case, window

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2605_05543_gb300 import emppp, inputs  # noqa: E402

PROPOSALS = ["bisect", "closed_form", "mlp"]


def _dump(T, W, V, u, n, D, precision, proposal, bunches=None):
    N = W.shape[1]
    with emppp.Solver(N if bunches is None else 0, D, DT, precision=precision, proposal=proposal,
                      bunches=bunches) as s:
        s.set_history(n, T, W, V, u)
        if proposal == "mlp":
            s.set_proposal(inputs.mlp_init_params(5))
        return s.bracket_dump()


def _mismatches(got, ref):
    bad = np.argwhere(got != ref)
    return len(bad), bad[:5].tolist()


# (N, n, D, sigma, seed): ragged target tiles; n >= D so the ring window has wrapped; one slot only
CASES = [(300, 60, 32, 5e-6, 51), (300, 60, 256, 5e-6, 52), (129, 0, 16, 3e-6, 53), (1000, 200, 128, 10e-6, 54)]


@pytest.mark.parametrize("proposal", PROPOSALS)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("N,n,D,sigma,seed", CASES)
def test_bracket_dump_equals_oracle(N, n, D, sigma, seed, precision, proposal):
    h = history_case(N, n, sigma=sigma, seed=seed)
    T, W, V, u = window(h, D)
    got, k0 = _dump(T, W, V, u, n, D, precision, proposal)
    assert k0 == max(0, n - D + 1)
    ref = oracle.bracket_table(h.T, h.W, n, D)
    nbad, where = _mismatches(got, ref)
    assert nbad == 0, (nbad, where)
    # every branch is exercised by the larger cases
    if n >= 60:
        assert set(np.unique(ref[ref >= 0] % 4)) >= {0, 2}


@pytest.mark.parametrize("oldest", [False, True])
@pytest.mark.parametrize("proposal", PROPOSALS)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bracket_dump_at_the_light_sphere(precision, proposal, oldest):
    n, D, nb = 40, 64, 64
    T, W, V, u = light_sphere_case(nb, n, oldest=oldest)
    got, _ = _dump(T, W, V, u, n, D, precision, proposal, bunches=[2] * nb)
    ref = np.full((2 * nb, 2 * nb), -1, dtype=np.int32)
    for b in range(nb):
        sl = slice(2 * b, 2 * b + 2)
        ref[sl, sl] = oracle.bracket_table(T, W[:, sl], n, D)
    nbad, where = _mismatches(got, ref)
    assert nbad == 0, (nbad, where)


@pytest.mark.parametrize("proposal", PROPOSALS)
def test_bracket_dump_far_from_the_split_origin(proposal):
    b = inputs.gaussian_bunch(64, 2e-6, 3.0, seed=37)
    x = b.x.copy()
    x[32:] += np.array([1.5, 0.0, 0.0])  # a second cluster 1.5 m away: its FP32 tests all fall back to FP64
    h = inputs.synthetic_history(x, b.u, 20, DT, seed=38)
    D = 32
    T, W, V, u = window(h, D)
    got, _ = _dump(T, W, V, u, 20, D, "mixed", proposal)
    nbad, where = _mismatches(got, oracle.bracket_table(h.T, h.W, 20, D))
    assert nbad == 0, (nbad, where)


def test_bracket_dump_leaves_the_state_and_refuses_bad_calls():
    h = history_case(200, 30, seed=55)
    T, W, V, u = window(h, 64)
    with emppp.Solver(200, 64, DT, precision="mixed", proposal="mlp") as s:
        s.set_history(30, T, W, V, u)
        with pytest.raises(emppp.EmpppError) as ei:
            s.bracket_dump()  # no network set
        assert ei.value.status == emppp.ERR_STATE
        s.set_options(proposal="closed_form")
        a, _ = s.bracket_dump()
        b, _ = s.bracket_dump()
        x, _, t, nn = s.get_state()
        assert nn == 30 and np.array_equal(a, b) and np.array_equal(x, W[-1])
