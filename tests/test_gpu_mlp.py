"""Learned retarded-time proposal on the GB300 (a starting point for the retarded-time search of Sec. 2.2;
the paper has no network): training data, tensor-core network passes, Adam, and the proposal inside both
pair kernels.

- The sampler's delays t - t_r equal the oracle's retarded times, and its features and targets (the log of
  the delay over the uniform-motion delay of the source's present record) equal their definitions
  evaluated on the host.
- The tensor-core forward pass and gradient equal the FP64 reference in oracle/mlp.py with the same BF16
  rounding points, far closer than to the unrounded network.
- Adam steps equal a plain FP64 Adam driven by the reference gradients, and training lowers the loss.
- With the network as the proposal, fields and branch counts are those of the paper's bisection, bit for
  bit, in the FP64 and the mixed path; the mean number of node tests per pair is reported beside
  bisection's and the closed-form guess's.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp
from gpu_helpers import DT, history_case, window

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2605_05543_gb300 import emppp, inputs  # noqa: E402

C = inputs.C_LIGHT


def _pairs(N, m, seed):
    rng = np.random.default_rng(seed)
    i = rng.integers(0, N, m)
    j = rng.integers(0, N - 1, m)
    j = np.where(j >= i, j + 1, j)
    return np.stack([i, j], axis=1).astype(np.int32)


def _samples(h, D, pairs):
    T, W, V, u = window(h, D)
    with emppp.Solver(W.shape[1], D, DT) as s:
        s.set_history(h.n, T, W, V, u)
        return s.sample_delays(pairs)


def _params(seed):
    rng = np.random.default_rng(100 + seed)
    p = inputs.mlp_init_params(seed)
    p[mlp.OFF_B1:mlp.OFF_W2] = rng.normal(0.0, 0.3, mlp.H)
    p[mlp.OFF_B2:mlp.OFF_W3] = rng.normal(0.0, 0.3, mlp.H)
    p[mlp.OFF_B3] = 0.4
    return p.astype(np.float32)


@pytest.mark.parametrize("D", [32, 4096])
def test_sampler_matches_oracle_and_definitions(D):
    h = history_case(300, 60, sigma=10e-6, seed=31)
    pairs = _pairs(300, 700, 1)
    feat, delay, z = _samples(h, D, pairs)
    n = h.n
    k0 = max(0, n - D + 1)
    for q in range(0, pairs.shape[0], 7):
        i, j = pairs[q]
        ref = oracle.retarded(h.T, h.W, h.V, n, D, j, h.W[n, i])
        tau = h.T[n] - ref["tr"]
        assert abs(delay[q] - tau) <= 1e-10 * tau, (q, delay[q], tau)
    i, j = pairs[:, 0], pairs[:, 1]
    d = h.W[n, i] - h.W[n, j]
    L = C * DT * D
    vprev = h.V[n - 1, j] if n > k0 else h.V[n, j]
    dn = np.linalg.norm(d, axis=1)[:, None]
    ref = np.concatenate([d / dn, dn / L, h.V[n, j] / C,
                          (h.V[n, j] - vprev) / C * D], axis=1)
    assert np.all(np.abs(feat - ref) <= 1e-6 * np.abs(ref) + 1e-30)
    # uniform motion from the present record: c tau_u = [d.b + sqrt((d.b)^2 + (1 - b^2) |d|^2)] / (1 - b^2)
    b = h.V[n, j] / C
    db = np.sum(d * b, axis=1)
    dd = np.sum(d * d, axis=1)
    ig2 = 1.0 - np.sum(b * b, axis=1)
    sq = np.sqrt(db * db + ig2 * dd)
    ctau_u = np.where(db >= 0.0, (db + sq) / ig2, dd / (sq - db))  # the same root without cancellation
    zref = np.log(C * delay / ctau_u)
    assert np.max(np.abs(z - zref)) <= 1e-6 * max(1.0, np.max(np.abs(zref)))


def _dataset(m, seed=41, N=1024, n=200, D=256):
    h = history_case(N, n, sigma=10e-6, seed=seed)
    feat, delay, z = _samples(h, D, _pairs(N, m, seed))
    return feat, z


@pytest.mark.parametrize("m", [1, 16, 1000, 4103])
def test_forward_matches_reference(m):
    X, _ = _dataset(max(m, 64))
    X = X[:m]
    p = _params(1)
    zg = emppp.mlp_forward(p, X)
    zr, _ = mlp.forward(p, X, rounding=True)
    zu, _ = mlp.forward(p, X, rounding=False)
    err = np.max(np.abs(zg - zr))
    scale = max(1.0, np.max(np.abs(zr)))
    assert err <= 1e-4 * scale
    if m >= 1000:
        assert err < 0.25 * np.max(np.abs(zg - zu))  # the BF16 rounding points are the kernel's


@pytest.mark.parametrize("m", [1, 31, 33, 5000])
def test_inference_form_matches_reference(m):
    """The pair kernels' form (halved hidden layers, packed BF16 SiLU, tensor-core output) stays within
    BF16 activation rounding of the reference form."""
    X, Tz = _dataset(max(m, 64), seed=42)
    X = X[:m]
    p = _params(4)
    zi = emppp.mlp_forward(p, X, mode="inference")
    zr, _ = mlp.forward(p, X, rounding=True)
    scale = max(1.0, np.max(np.abs(zr)))
    assert np.all(np.isfinite(zi))
    assert np.max(np.abs(zi - zr)) <= 3e-2 * scale
    assert np.sqrt(np.mean((zi - zr) ** 2)) <= 5e-3 * scale


_BLOCKS = [(mlp.OFF_W1, mlp.OFF_B1), (mlp.OFF_B1, mlp.OFF_W2), (mlp.OFF_W2, mlp.OFF_B2), (mlp.OFF_B2, mlp.OFF_W3),
           (mlp.OFF_W3, mlp.OFF_B3), (mlp.OFF_B3, mlp.NUM_PARAMS)]


@pytest.mark.parametrize("m", [16, 1009, 20000])
def test_gradient_matches_reference(m):
    X, Tz = _dataset(m)
    p = _params(2)
    loss_g, g = emppp.mlp_gradient(p, X, Tz)
    loss_r, gr = mlp.loss_and_grad(p, X, Tz, rounding=True)
    assert abs(loss_g - loss_r) <= 1e-4 * loss_r
    for a, b in _BLOCKS:
        ref = gr[a:b]
        nrm = np.linalg.norm(ref)
        assert np.linalg.norm(g[a:b] - ref) <= 1e-3 * nrm, (a, b)
        assert np.max(np.abs(g[a:b] - ref)) <= 2e-3 * np.max(np.abs(ref)), (a, b)


def test_adam_steps_match_fp64_adam():
    m, batch = 868, 256
    X, Tz = _dataset(m, seed=43)
    p0 = _params(3)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    pg, losses = emppp.mlp_train(p0, X, Tz, epochs=1, batch=batch, lr=lr, beta1=b1, beta2=b2, eps=eps)
    p = p0.astype(np.float64)
    m1 = np.zeros_like(p)
    m2 = np.zeros_like(p)
    keep = np.ones(p.size, dtype=bool)
    for s, r0 in enumerate(range(0, m, batch), start=1):
        rows = slice(r0, min(m, r0 + batch))
        _, g = mlp.loss_and_grad(p.astype(np.float32), X[rows], Tz[rows], rounding=True)
        # elements whose sign is well above the FP32 accumulation error of their block
        for a, b in _BLOCKS:
            keep[a:b] &= np.abs(g[a:b]) > 1e-4 * np.max(np.abs(g[a:b]))
        m1 = b1 * m1 + (1 - b1) * g
        m2 = b2 * m2 + (1 - b2) * g * g
        p = p - lr * (m1 / (1 - b1 ** s)) / (np.sqrt(m2 / (1 - b2 ** s)) + eps)
    assert keep.mean() >= 0.9
    diff = np.abs(pg.astype(np.float64) - p)
    assert np.max(diff[keep]) <= 0.02 * lr
    assert np.max(diff) <= 2 * lr * 4
    assert losses.shape == (1,) and np.isfinite(losses[0])


def _train(X, Tz, epochs=40):
    p0 = inputs.mlp_init_params(0)
    l0, _ = emppp.mlp_gradient(p0, X, Tz)
    p, losses = emppp.mlp_train(p0, X, Tz, epochs=epochs, batch=512, lr=3e-3, lr_final=1e-5)
    l1, _ = emppp.mlp_gradient(p, X, Tz)
    return p, l0, l1, losses


def test_training_lowers_loss():
    X, Tz = _dataset(16384, seed=44)
    p, l0, l1, losses = _train(X, Tz)
    print(f"proposal net: loss {l0:.4f} -> {l1:.5f}; per epoch {np.array2string(losses[::5], precision=4)}")
    assert np.all(np.isfinite(losses))
    assert l1 <= 0.01 * l0
    assert losses[-1] < losses[0]


@pytest.fixture(scope="module")
def proposal_net():
    """A network trained on pairs of one stored state (N = 2048, sigma = 10 um, depth 256)."""
    N, n, D = 2048, 300, 256
    h = history_case(N, n, sigma=10e-6, seed=45)
    feat, delay, z = _samples(h, D, _pairs(N, 32768, 46))
    p, l0, l1, _ = _train(feat, z, epochs=60)
    return p, l1


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("N,seed", [(2048, 45), (1000, 48)])  # the training state; a ragged bunch
def test_mlp_proposal_gives_bisection_results(precision, N, seed, proposal_net):
    p, loss = proposal_net
    D = 256
    h = history_case(N, 300, sigma=10e-6, seed=seed)
    T, W, V, u = window(h, D)
    N = W.shape[1]
    out = {}
    for prop in ("bisect", "closed_form", "mlp"):
        with emppp.Solver(N, D, DT, precision=precision, proposal=prop) as s:
            s.set_history(h.n, T, W, V, u)
            if prop == "mlp":
                s.set_proposal(p)
            s.step(1)
            E, B = s.get_fields()
            st = s.stats()
        out[prop] = (E, B, st)
    Eb, Bb, sb = out["bisect"]
    for prop in ("closed_form", "mlp"):
        E, B, st = out[prop]
        assert np.array_equal(E, Eb) and np.array_equal(B, Bb), prop
        for k in ("pairs", "out_of_history", "shortcut", "bisection"):
            assert st[k] == sb[k], (prop, k)
    tpp = {k: out[k][2]["node_tests"] / out[k][2]["pairs"] for k in out}
    print(f"{precision} N={N}: node tests per pair bisect {tpp['bisect']:.3f} closed_form {tpp['closed_form']:.3f} "
          f"mlp {tpp['mlp']:.3f} (net loss {loss:.4f}); branches ooh {sb['out_of_history']} "
          f"shortcut {sb['shortcut']} bisection {sb['bisection']}")
    assert tpp["mlp"] < tpp["bisect"]


def test_mlp_proposal_needs_a_network():
    h = history_case(64, 20, seed=47)
    T, W, V, u = window(h, 16)
    with emppp.Solver(64, 16, DT, proposal="mlp") as s:
        s.set_history(h.n, T, W, V, u)
        with pytest.raises(emppp.EmpppError):
            s.step(1)
        with pytest.raises((emppp.EmpppError, ValueError)):
            s.set_proposal(np.zeros(10, dtype=np.float32))
        with pytest.raises(emppp.EmpppError):
            s.sample_delays(np.array([[3, 3]], dtype=np.int32))


def test_network_trained_out_of_sample_gains_over_bisection():
    """What the trained network gains over the method without it, out of sample: trained on (feature, delay)
    samples of the N = 4096 uniform-field run (sigma = 10 um, B = 5e-5 T along x, depth 512, from t = 0), then
    used on another bunch (N = 8192, sigma = 20 um, seeded step-200 history, depth 1024). Over the same step
    from the same state: fields identical to the paper's bisection (the brackets are the bisection's), node
    tests per pair far below bisection's and within 1 % of the closed-form guess (which sits at the floor of
    one test beyond the history and two for a bracket)."""
    rng = np.random.default_rng(60)
    N2, D2 = 4096, 512
    b = inputs.gaussian_bunch(N2, 10e-6, 3.0, seed=0)
    feats, zs = [], []
    with emppp.Solver(N2, D2, DT, precision="mixed", proposal="closed_form") as s:
        s.set_particles(b.x.copy(), b.u.copy())
        n = 0
        for k in (64, 256, 511):
            s.step(k - n, emppp.bext_uniform((5e-5, 0.0, 0.0)))
            n = k
            f, _, z = s.sample_delays(_pairs(N2, 1 << 17, int(rng.integers(1 << 30))))
            feats.append(f)
            zs.append(z)
    X, Z = np.concatenate(feats), np.concatenate(zs)
    p, losses = emppp.mlp_train(inputs.mlp_init_params(1), X, Z, epochs=3, batch=4096, lr=2e-3, lr_final=1e-5)
    assert np.all(np.isfinite(losses)) and losses[-1] < losses[0]
    N, n0, D = 8192, 200, 1024
    h = history_case(N, n0, sigma=20e-6, seed=61)
    T, W, V, u = window(h, D)
    out = {}
    for prop in ("bisect", "closed_form", "mlp"):
        with emppp.Solver(N, D, DT, precision="mixed", proposal=prop) as s:
            s.set_history(h.n, T, W, V, u)
            if prop == "mlp":
                s.set_proposal(p)
            s.step(1)
            E, B = s.get_fields()
            st = s.stats()
        out[prop] = (E, B, st["node_tests"] / st["pairs"])
    for prop in ("closed_form", "mlp"):
        assert np.array_equal(out[prop][0], out["bisect"][0]) and np.array_equal(out[prop][1], out["bisect"][1])
    tb, tc, tm = out["bisect"][2], out["closed_form"][2], out["mlp"][2]
    print(f"out of sample: node tests per pair bisection {tb:.4f}, closed form {tc:.4f}, network {tm:.4f}")
    assert tm < 0.5 * tb
    assert tm <= 1.01 * tc


def test_factor_table_beyond_int32_is_refused():
    """The mixed path's table of delay factors holds sum_b ceil(n_b / 512) n_b entries, addressed with 32-bit
    offsets: a bunch of 2^20 + 1 particles needs more than 2^31 - 1 of them, and emppp_set_proposal refuses it
    (a short history keeps the handle's own memory small); 2^20 - 512 particles fit."""
    params = inputs.mlp_init_params(3)
    with emppp.Solver((1 << 20) + 1, 2, DT, precision="mixed") as s:
        with pytest.raises(emppp.EmpppError) as e:
            s.set_proposal(params)
        assert e.value.status == emppp.ERR_ARG
    with emppp.Solver((1 << 20) - 512, 2, DT, precision="mixed") as s:
        s.set_proposal(params)
