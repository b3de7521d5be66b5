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


def test_paper_bunch_recipe():
    """Sec. 2.5: the paper's own sampler (Table 1 widths, v_z mean shift, beam-to-lab rotation)."""
    vals = {r[0]: float(r[1]) for r in _rows("beam_params_1MeV.txt")}
    g0, beta = inputs.beam_kinematics(vals["E0_MeV"] * 1e6 * inputs.Q_E)
    assert round(g0, 2) == vals["gamma0"] and round(beta, 3) == vals["beta"]
    v0 = beta * inputs.C_LIGHT
    b = inputs.paper_bunch(20000, 1.0, seed=2)
    v = inputs.velocity_of(b.u)
    # the shifted longitudinal mean is v0 (to rounding), the transverse spread eps_r v0 / r_perp
    assert abs(v[:, 2].mean() - v0) <= 1e-9 * v0
    assert np.allclose(v[:, :2].std(axis=0), 1e-6 * v0 / 2e-3, rtol=2e-2)
    assert np.allclose(b.x.std(axis=0), 2e-3, rtol=2e-2)
    assert np.all(np.linalg.norm(v, axis=1) < inputs.C_LIGHT)
    mc2 = inputs.M_E * inputs.C_LIGHT ** 2
    # energy spread from gamma(E): relative spread delta_E of E0, before the speed adjustment
    gz = 1.0 / np.sqrt(1.0 - (v[:, 2] / inputs.C_LIGHT) ** 2)
    K = (gz - 1) * mc2 / (1e6 * inputs.Q_E)
    assert abs(np.median(K) - 1.0) < 2e-3
    # rotation: theta = 90 deg turns the beam axis onto +x; phi = 90 deg then onto +y; norms are kept
    for theta, phi, axis in ((math.pi / 2, 0.0, 0), (math.pi / 2, math.pi / 2, 1), (0.0, 1.3, 2)):
        r = inputs.paper_bunch(500, 10.0, theta=theta, phi=phi, center=inputs.PAPER_R0, seed=4)
        r0 = inputs.paper_bunch(500, 10.0, seed=4)
        vr = inputs.velocity_of(r.u)
        assert np.all(vr[:, axis] > 0.99 * inputs.C_LIGHT)
        d = r.x - np.asarray(inputs.PAPER_R0)
        assert np.allclose(np.linalg.norm(d, axis=1), np.linalg.norm(r0.x, axis=1), rtol=1e-12)
        assert np.allclose(np.linalg.norm(r.u, axis=1), np.linalg.norm(r0.u, axis=1), rtol=1e-12)
    R = inputs.rotation(0.4, -1.1)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-15) and abs(np.linalg.det(R) - 1) < 1e-15
    w = inputs.paper_bunch(10, 1.0, weight=2.5e6).weights
    assert w.shape == (10,) and np.all(w == 2.5e6)


def test_printed_baseline_states_move_at_the_beam_speed():
    """The paper's printed states of the baseline run (tests/golden/paper_centroid_steps.txt) against
    the 1 MeV beam kinematics: zbar / t is the beam speed beta c to within the printed digits (t to 3
    significant figures, zbar to 4)."""
    gamma0, beta0 = inputs.beam_kinematics(1.0e6 * inputs.Q_E)
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_centroid_steps.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    assert len(rows) == 2
    for Np, step, t, z in rows:
        t, z = float(t), float(z)
        assert abs(z / (t * inputs.C_LIGHT) / beta0 - 1.0) <= 1e-3, (Np, z / (t * inputs.C_LIGHT), beta0)
