"""The oracle's bracket table (the per-pair reference of the GPU's bracket dump) pinned against a brute-force
scan of the node test P(k): c (t - t_k) <= |r - w_k| over every slot of the window (Sec. 2.2). P is
monotone in k for |v| < c, so the bracket is its unique change of sign: out of history when P(k0) holds,
else k1 = the newest k with P(k) false, the near-field shortcut when k1 = n - 1 and bisection otherwise."""
import numpy as np
import pytest

import oracle
from paper_2605_05543_gb300 import inputs


def _brute(T, W, n, D, i, j):
    k0 = max(0, n - D + 1)
    r = W[n, i]
    P = [oracle.node_test(T, W, j, r, T[n], k) for k in range(k0, n + 1)]
    assert P[-1]  # P(n) always holds
    # monotone: once true, true for every newer slot
    first_true = P.index(True)
    assert all(P[first_true:])
    if first_true == 0:
        return 0  # out of history, k1 = k0
    k1 = k0 + first_true - 1
    return 4 * (k1 - k0) + (1 if k1 == n - 1 else 2)


@pytest.mark.parametrize("N,n,D,sigma,seed", [(12, 30, 64, 1e-6, 1), (12, 30, 8, 1e-6, 2), (9, 0, 4, 1e-6, 3),
                                              (10, 50, 64, 10e-6, 4)])
def test_bracket_table_equals_brute_force_scan(N, n, D, sigma, seed):
    b = inputs.gaussian_bunch(N, sigma, 3.0, seed=seed)
    h = inputs.synthetic_history(b.x, b.u, n, 1e-15, seed=seed + 10)
    tab = oracle.bracket_table(h.T, h.W, n, D)
    for i in range(N):
        for j in range(N):
            if i == j:
                assert tab[i, j] == -1
            else:
                assert tab[i, j] == _brute(h.T, h.W, n, D, i, j), (i, j)
    codes = tab[tab >= 0] % 4
    if n >= 30 and sigma <= 1e-6:
        assert np.any(codes == 2)  # the bisection branch is exercised
