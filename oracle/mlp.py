"""FP64 reference of the learned-guess MLP (TEST INFRASTRUCTURE ONLY).

Plain numpy forward pass and backpropagation of the network the library
trains: 16 -> 256 (SiLU) -> 256 (SiLU) -> 325, loss (1/n) sum mask (Y - T)^2.
Weight vector layout: W1[256][16], b1[256], W2[256][256], b2[256],
W3[325][256], b3[325].  Pinned by central finite differences in
tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import numpy as np

SHAPES = [(256, 16), (256,), (256, 256), (256,), (325, 256), (325,)]


def n_params() -> int:
    return int(sum(np.prod(s) for s in SHAPES))


def unpack(w: np.ndarray) -> list[np.ndarray]:
    out, o = [], 0
    w = np.asarray(w, dtype=np.float64)
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(w[o:o + k].reshape(s))
        o += k
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(w: np.ndarray, X: np.ndarray):
    W1, b1, W2, b2, W3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ W1.T + b1
    H1 = silu(Z1)
    Z2 = H1 @ W2.T + b2
    H2 = silu(Z2)
    Y = H2 @ W3.T + b3
    return Y, (X, Z1, H1, Z2, H2)


def loss(w, X, T, M) -> float:
    Y, _ = forward(w, X)
    return float(np.sum(M * (Y - T) ** 2) / X.shape[0])


def loss_and_grad(w, X, T, M):
    W1, b1, W2, b2, W3, b3 = unpack(w)
    Y, (X, Z1, H1, Z2, H2) = forward(w, X)
    n = X.shape[0]
    D = M * (Y - T)
    L = float(np.sum(D * D) / n)
    dY = 2.0 * D / n
    gW3 = dY.T @ H2
    gb3 = dY.sum(0)
    dZ2 = (dY @ W3) * dsilu(Z2)
    gW2 = dZ2.T @ H1
    gb2 = dZ2.sum(0)
    dZ1 = (dZ2 @ W2) * dsilu(Z1)
    gW1 = dZ1.T @ X
    gb1 = dZ1.sum(0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return L, g


def to_bf16(w: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even) and back to float64."""
    a = np.ascontiguousarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)
