"""Pins of the proposal-network reference in oracle/mlp.py (CPU only).

- The gradient of the plain network (rounding off) equals central finite differences of its loss.
- The forward pass of the plain network equals the same network built from torch's float64 Linear and
  SiLU modules, and its gradient equals torch autograd's.
- bf16() equals torch's float32 -> bfloat16 conversion (round to nearest, ties to even), including
  ties, subnormals, infinities and values that round up into the next binade.
- With rounding on, the result moves away from the plain network by no more than BF16 rounding allows.
"""
import numpy as np
import pytest

from oracle import mlp
from paper_2605_05543_gb300 import inputs


def _case(m=37, seed=3):
    rng = np.random.default_rng(seed)
    p = inputs.mlp_init_params(seed).astype(np.float64)
    # non-zero biases so that a dropped bias term shows
    p[mlp.OFF_B1:mlp.OFF_W2] = rng.normal(0.0, 0.3, mlp.H)
    p[mlp.OFF_B2:mlp.OFF_W3] = rng.normal(0.0, 0.3, mlp.H)
    p[mlp.OFF_B3] = 0.7
    X = rng.normal(0.0, 1.0, (m, mlp.N_IN))
    T = rng.normal(0.5, 1.0, m)
    return p, X, T


def test_layout():
    assert mlp.NUM_PARAMS == 4929 == inputs.MLP_NUM_PARAMS
    p = np.arange(mlp.NUM_PARAMS, dtype=np.float64)
    assert np.array_equal(mlp.pack(*mlp.unpack(p)), p)


def test_gradient_equals_finite_differences():
    p, X, T = _case()
    X = X.astype(np.float32).astype(np.float64)
    _, g = mlp.loss_and_grad(p, X, T, rounding=False)
    rng = np.random.default_rng(0)
    # every bias and output weight, plus a sample of W1 and W2 entries
    idx = np.concatenate([np.arange(mlp.OFF_B1, mlp.OFF_W2), np.arange(mlp.OFF_B2, mlp.NUM_PARAMS),
                          rng.choice(np.arange(mlp.OFF_W1, mlp.OFF_B1), 60, replace=False),
                          rng.choice(np.arange(mlp.OFF_W2, mlp.OFF_B2), 120, replace=False)])
    h = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        lp, _ = mlp.loss_and_grad(pp, X, T, rounding=False)
        lm, _ = mlp.loss_and_grad(pm, X, T, rounding=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_plain_network_equals_torch_modules():
    torch = pytest.importorskip("torch")
    p, X, T = _case(m=50, seed=5)
    X = X.astype(np.float32).astype(np.float64)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p)
    l1 = torch.nn.Linear(mlp.N_IN, mlp.H, dtype=torch.float64)
    l2 = torch.nn.Linear(mlp.H, mlp.H, dtype=torch.float64)
    l3 = torch.nn.Linear(mlp.H, 1, dtype=torch.float64)
    with torch.no_grad():
        l1.weight.copy_(torch.from_numpy(W1.T.copy()))
        l1.bias.copy_(torch.from_numpy(b1.copy()))
        l2.weight.copy_(torch.from_numpy(W2.T.copy()))
        l2.bias.copy_(torch.from_numpy(b2.copy()))
        l3.weight.copy_(torch.from_numpy(w3[None, :].copy()))
        l3.bias.fill_(float(b3))
    net = torch.nn.Sequential(l1, torch.nn.SiLU(), l2, torch.nn.SiLU(), l3)
    z_t = net(torch.from_numpy(X))[:, 0]
    loss_t = torch.mean((z_t - torch.from_numpy(T)) ** 2)
    loss_t.backward()
    z, _ = mlp.forward(p, X, rounding=False)
    loss, g = mlp.loss_and_grad(p, X, T, rounding=False)
    assert np.allclose(z, z_t.detach().numpy(), rtol=1e-13, atol=1e-13)
    assert abs(loss - loss_t.item()) <= 1e-13 * loss
    gt = mlp.pack(l1.weight.grad.numpy().T, l1.bias.grad.numpy(), l2.weight.grad.numpy().T, l2.bias.grad.numpy(),
                  l3.weight.grad.numpy()[0], l3.bias.grad.numpy()[0])
    assert np.allclose(g, gt, rtol=1e-11, atol=1e-14)


def test_bf16_equals_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    u = rng.integers(0, 2 ** 32, 200000, dtype=np.uint64).astype(np.uint32)
    x = u.view(np.float32)
    x = x[np.isfinite(x)]
    special = np.array([0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -1.0 - 2 ** -8,
                        3.3895314e38, 1e-40, -1e-40, np.inf, -np.inf, 65504.0, 2 ** -126], dtype=np.float32)
    # exact ties between neighbouring bf16 values: bf16 mantissa odd/even and a 0x8000 remainder
    ties = (np.arange(0x3F800000, 0x3F800000 + 64 * 0x10000, 0x10000, dtype=np.uint32) + 0x8000).view(np.float32)
    x = np.concatenate([x, special, ties])
    ref = torch.from_numpy(x.copy()).to(torch.bfloat16).to(torch.float64).numpy()
    got = mlp.bf16(x)
    same = (got == ref) | (np.isnan(got) & np.isnan(ref))
    assert np.all(same)


def test_rounding_stays_within_bf16_error():
    p, X, T = _case(m=200, seed=9)
    z0, _ = mlp.forward(p, X, rounding=False)
    z1, _ = mlp.forward(p, X, rounding=True)
    # relative BF16 rounding 2^-9 on each GEMM operand, summed over the layers' magnitudes
    assert np.max(np.abs(z1 - z0)) <= 0.05 * np.max(np.abs(z0))
    assert np.max(np.abs(z1 - z0)) > 0.0
    l0, g0 = mlp.loss_and_grad(p, X, T, rounding=False)
    l1, g1 = mlp.loss_and_grad(p, X, T, rounding=True)
    assert abs(l1 - l0) <= 0.05 * l0
    assert np.linalg.norm(g1 - g0) <= 0.05 * np.linalg.norm(g0)
