"""FP64 CPU reference of the per-atom control-variate MLP (test infrastructure).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``. Plain PyTorch CPU
ops in float64 with autograd: the GPU forward and backward kernels are
checked against it.

Network (per atom): x in R^33 (16-nearest-neighbour (d / 4 A, R / 1.7 A)
pairs and the atom's own R / 1.7 A) -> z1 = W1 x + b1 (64) -> h1 = GELU(z1)
-> z2 = W2 h1 + b2 (64) -> h2 = GELU(z2) -> y = w3 . h2 + b3, GELU the exact
erf form. Parameters are one flat FP32 vector in the order W1 (64 x 33,
row-major), b1, W2 (64 x 64), b2, w3, b3 (6401 values); forward and
backward use the parameters rounded to BF16 (round to nearest even), with
the loss L = mean over atoms of (y - target)^2.
"""
from __future__ import annotations

import numpy as np
import torch

N_IN, N_HID = 33, 64
N_PARAMS = N_HID * N_IN + N_HID + N_HID * N_HID + N_HID + N_HID + 1


def unpack(p: torch.Tensor):
    o = 0
    W1 = p[o:o + N_HID * N_IN].reshape(N_HID, N_IN); o += N_HID * N_IN
    b1 = p[o:o + N_HID]; o += N_HID
    W2 = p[o:o + N_HID * N_HID].reshape(N_HID, N_HID); o += N_HID * N_HID
    b2 = p[o:o + N_HID]; o += N_HID
    w3 = p[o:o + N_HID]; o += N_HID
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def bf16_round(params) -> torch.Tensor:
    """FP32 master parameters rounded to BF16, as float64."""
    t = torch.as_tensor(np.asarray(params, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float64)


def forward(params, x) -> np.ndarray:
    p = bf16_round(params)
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = torch.as_tensor(np.asarray(x, dtype=np.float64))
    h1 = torch.nn.functional.gelu(X @ W1.T + b1)
    h2 = torch.nn.functional.gelu(h1 @ W2.T + b2)
    return (h2 @ w3 + b3).numpy()


def loss_and_grad(params, x, target):
    """(L, dL/dparams) with the BF16-rounded parameters, in float64."""
    p = bf16_round(params).clone().requires_grad_(True)
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = torch.as_tensor(np.asarray(x, dtype=np.float64))
    T = torch.as_tensor(np.asarray(target, dtype=np.float64))
    h1 = torch.nn.functional.gelu(X @ W1.T + b1)
    h2 = torch.nn.functional.gelu(h1 @ W2.T + b2)
    y = h2 @ w3 + b3
    L = ((y - T) ** 2).mean()
    L.backward()
    return float(L.detach()), p.grad.numpy().copy()


def init_params(seed: int = 0) -> np.ndarray:
    """Seeded FP32 initialisation (uniform +-1/sqrt(fan_in), output bias 0.5)."""
    rng = np.random.default_rng(seed)
    parts = [rng.uniform(-1, 1, N_HID * N_IN) / np.sqrt(N_IN), np.zeros(N_HID),
             rng.uniform(-1, 1, N_HID * N_HID) / np.sqrt(N_HID), np.zeros(N_HID),
             rng.uniform(-1, 1, N_HID) / np.sqrt(N_HID), np.array([0.5])]
    return np.concatenate(parts).astype(np.float32)
