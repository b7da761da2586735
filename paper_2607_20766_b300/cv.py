"""Learned control variate for union volumes (not in the paper).

A per-atom network (33 -> 64 -> 64 -> 1, GELU, BF16 weights, FP32
accumulation) maps each atom's 16-nearest-neighbour geometry to a crowding
weight om_i. The weighted Gaussians u~ = sum_i om_i g_i have a closed-form
volume, so the sampler estimates only the residual (u - u~)/m; the estimate
stays unbiased whatever the network predicts, and the plain estimator is the
om = 0 special case. Training targets are union attributions
om*_i = E_{N(c_i, 1/(2 alpha_i))}[u/m] drawn by the library's own sampler
(their v-weighted sum is the exact union volume). Every step -- features,
targets, forward, backward, Adam -- runs in the library's CUDA kernels; this
module only orders the calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as B


def init_params(seed: int = 0, device=None) -> torch.Tensor:
    """Seeded FP32 parameters (uniform +-1/sqrt(fan_in) weights, output bias 0.5)."""
    g = torch.Generator().manual_seed(seed)
    n_in, h = B.MLP_IN, B.MLP_HIDDEN
    parts = [(torch.rand(h * n_in, generator=g) * 2 - 1) / np.sqrt(n_in), torch.zeros(h),
             (torch.rand(h * h, generator=g) * 2 - 1) / np.sqrt(h), torch.zeros(h),
             (torch.rand(h, generator=g) * 2 - 1) / np.sqrt(h), torch.tensor([0.5])]
    p = torch.cat(parts).to(torch.float32)
    return p.to(device or "cuda")


class CrowdingNet:
    """FP32 master parameters and Adam moments on the device."""

    def __init__(self, seed: int = 0, device=None, params: torch.Tensor | None = None):
        self.params = init_params(seed, device) if params is None else params.to(torch.float32).contiguous()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0

    def predict(self, feats: torch.Tensor) -> torch.Tensor:
        return B.mlp_forward(self.params, feats.contiguous())

    def fit(self, feats: torch.Tensor, targets: torch.Tensor, epochs: int = 10, batch: int = 16384,
            lr: float = 2e-3, seed: int = 0) -> list[float]:
        """Minibatch Adam on the mean squared error; returns the mean loss of
        each epoch (read back once per epoch)."""
        feats = feats.contiguous()
        targets = targets.to(torch.float32).contiguous()
        n = feats.shape[0]
        g = torch.Generator(device=feats.device).manual_seed(seed)
        history = []
        for _ in range(epochs):
            perm = torch.randperm(n, generator=g, device=feats.device).to(torch.int32)
            # the epoch's minibatch loop (loss/gradient, Adam) runs inside the library
            losses = B.mlp_train_epoch(self.params, self.m, self.v, feats, targets, perm, batch, self.step, lr)
            self.step += losses.numel()
            history.append(float(losses.mean().item()))
        return history


def attributions_and_features(S, seed: int, M: int = 512):
    """(features [n_atoms, 33], targets om* [n_atoms]) of every atom of S."""
    return B.cv_features(S), B.union_attributions(S, seed, M)
