"""Reference of the learned-proposal network -- test infrastructure only.

A 10-64-64-1 perceptron with SiLU activations, z = w3 . silu(silu(X W1 + b1) W2 + b2) + b3, its mean
squared error against targets T, and the gradient of that loss, in FP64 with numpy. With
``rounding=True`` the GEMM operands are rounded to BF16 at the points the tensor-core kernels round
them (X, W1, silu(H1) and W2 in the forward pass; dH2 and W2 in the input gradient of layer 2); every
other quantity stays FP64. With ``rounding=False`` it is the plain network, which
tests/test_oracle_mlp.py pins by finite differences.

Parameter vector (float32 values, 4929): W1[10][64] (feature, unit), b1[64], W2[64][64] (in, out),
b2[64], w3[64], b3.

Only tests/, the smoke check and the benchmark's CPU-baseline leg use this module; it shares no code
with the CUDA library.
"""
from __future__ import annotations

import numpy as np

N_IN = 10
H = 64
OFF_W1 = 0
OFF_B1 = OFF_W1 + N_IN * H
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
NUM_PARAMS = OFF_B3 + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[OFF_W1:OFF_B1].reshape(N_IN, H), p[OFF_B1:OFF_W2], p[OFF_W2:OFF_B2].reshape(H, H), p[OFF_B2:OFF_W3],
            p[OFF_W3:OFF_B3], p[OFF_B3])


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def silu(x):
    return x * sigmoid(x)


def dsilu(x):
    s = sigmoid(x)
    return s * (1.0 + x * (1.0 - s))


def _r(x, rounding):
    return bf16(x) if rounding else np.asarray(x, dtype=np.float64)


def forward(p, X, rounding=True):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    Xr = _r(np.asarray(X, dtype=np.float32), rounding)
    H1 = Xr @ _r(W1, rounding) + b1
    A1 = silu(H1)
    H2 = _r(A1, rounding) @ _r(W2, rounding) + b2
    A2 = silu(H2)
    z = A2 @ w3 + b3
    return z, dict(Xr=Xr, H1=H1, A1=A1, H2=H2, A2=A2)


def loss_and_grad(p, X, T, rounding=True):
    """(mean squared error, gradient vector) of one batch."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    z, c = forward(p, X, rounding)
    m = z.shape[0]
    e = z - np.asarray(T, dtype=np.float64)
    loss = float(np.sum(e * e) / m)
    dz = 2.0 * e / m
    dH2 = dz[:, None] * w3[None, :] * dsilu(c["H2"])
    dA1 = _r(dH2, rounding) @ _r(W2, rounding).T
    dH1 = dA1 * dsilu(c["H1"])
    g = pack(c["Xr"].T @ dH1, dH1.sum(axis=0), c["A1"].T @ dH2, dH2.sum(axis=0), c["A2"].T @ dz, dz.sum())
    return loss, g
