"""The seeded input generator: published SplitMix64 outputs, the paper's printed beam kinematics and
the statistics of the bunch recipe (no GPU)."""
import math
import os

import numpy as np

from paper_2605_05543_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_splitmix64_published_vector():
    ref = [int(r[0]) for r in _rows("splitmix64_seed1234567.txt")]
    assert [int(v) for v in inputs.splitmix64(1234567, 5)] == ref
    # the generator is counter based: any window of the stream is reproducible on its own
    assert [int(v) for v in inputs.splitmix64(1234567, 2, offset=3)] == ref[3:5]


def test_normals_window_and_moments():
    a = inputs.normals(5, 40)
    assert np.array_equal(inputs.normals(5, 13, offset=27), a[27:40])
    z = inputs.normals(9, 400000)
    assert abs(z.mean()) < 5e-3 and abs(z.std() - 1) < 5e-3


def test_beam_kinematics_printed_in_paper():
    """Sec. 2.5 Table 1: E0 = 1 MeV gives gamma0 = 2.96 and beta = 0.941."""
    vals = {r[0]: float(r[1]) for r in _rows("beam_params_1MeV.txt")}
    mc2_MeV = inputs.M_E * inputs.C_LIGHT ** 2 / inputs.Q_E / 1e6
    g0 = 1.0 + vals["E0_MeV"] / mc2_MeV
    assert round(g0, 2) == vals["gamma0"]
    assert round(math.sqrt(1 - 1 / g0 ** 2), 3) == vals["beta"]
    b = inputs.gaussian_bunch(20000, 2e-3, g0, dE_rel=0.01, seed=3)
    gam = np.sqrt(1 + np.sum(b.u ** 2, axis=1) / inputs.C_LIGHT ** 2)
    K = (gam - 1) * mc2_MeV
    assert abs(K.mean() - 1.0) < 1e-3 and abs(K.std() / 1.0 - 0.01) < 5e-4


def test_bunch_recipe_statistics():
    N, sigma, g0 = 65536, 20e-6, 3.0
    b = inputs.gaussian_bunch(N, sigma, g0, seed=0)
    assert b.x.shape == (N, 3) and b.u.shape == (N, 3)
    assert np.allclose(b.x.std(axis=0), sigma, rtol=2e-2)
    u0 = inputs.C_LIGHT * math.sqrt(g0 ** 2 - 1)
    assert np.allclose(b.u[:, :2].std(axis=0), 1e-4 * u0, rtol=2e-2)
    assert np.all(b.u[:, 2] > 0)
    # same seed, same bunch; another seed, another bunch
    assert np.array_equal(inputs.gaussian_bunch(N, sigma, g0, seed=0).x, b.x)
    assert not np.array_equal(inputs.gaussian_bunch(N, sigma, g0, seed=1).x, b.x)


def test_synthetic_history_ends_at_present_state():
    b = inputs.gaussian_bunch(64, 10e-6, 3.0, seed=4)
    h = inputs.synthetic_history(b.x, b.u, 30, 1e-15)
    assert h.W.shape == (31, 64, 3) and h.T.shape == (31,)
    assert np.array_equal(h.W[30], b.x)
    assert np.all(np.linalg.norm(h.V, axis=2) < inputs.C_LIGHT)
    assert np.all(np.diff(h.T) > 0)


def test_batch_bunches_ranges():
    bb = inputs.batch_bunches()
    assert len(bb) == 64
    for N, s, g, seed in bb:
        assert 512 <= N <= 16384 and 5e-6 <= s <= 50e-6 and 2 <= g <= 20
