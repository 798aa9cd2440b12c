"""Learned initial guess for the pressure-correction solve: training driver.

Argument marshalling around the network entry points of the C ABI; the
forward pass, the gradients and the Adam update all run in CUDA kernels
(float32 master weights, bfloat16 copies used by the kernels).

Network (per dof i, neighbours N(i) of the P1 sparsity pattern without i):
inputs x_i = (b_i / s_b, phi1_i / s_phi, phi2_i / s_phi); two message-passing
layers of width 32 with ReLU, h = relu(W_a h_i + W_b mean_{N(i)} h + c); readout
y_i = w3 . h2_i + c3 + a0 x_i,2 + a1 x_i,3; guess phi0 = s_phi y.  The training
target of a recorded step is phi / s_phi, the loss the mean squared error.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi

H = 32
N_PARAMS = capi.OASIS_NET_PARAMS


def initial_params(seed: int = 0) -> np.ndarray:
    """He-scaled random hidden weights, zero biases, a zero readout and a skip
    term that starts as the previous correction (a0 = 1, a1 = 0): the untrained
    network returns the fallback phi^{n-1} exactly, so training starts from it
    (a random readout would start it ~10 % away, far beyond the step-to-step
    change of phi on smooth flows)."""
    g = np.random.default_rng(seed)
    w1 = g.standard_normal((2, H * 3)) * np.sqrt(2.0 / 6.0)
    w2 = g.standard_normal((2, H * H)) * np.sqrt(2.0 / (2 * H))
    w3 = np.zeros(H)
    p = np.concatenate([w1[0], w1[1], np.zeros(H), w2[0], w2[1], np.zeros(H), w3, [0.0], [1.0, 0.0]])
    assert p.size == N_PARAMS
    return p.astype(np.float32)


class GuessNet:
    """One network (parameters, Adam moments, work buffers) on a mesh."""

    def __init__(self, mesh, n_dofs: int, params=None, seed: int = 0, device="cuda"):
        self.n = int(n_dofs)
        self.device = torch.device(device)
        self.handle = capi.oasis_net_create(mesh)
        self.grad = torch.zeros(N_PARAMS, dtype=torch.float32, device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.adam_steps = 0
        self.set_params(initial_params(seed) if params is None else params)

    def set_params(self, params):
        capi.oasis_net_set_params(self.handle, np.asarray(params, dtype=np.float32))
        self.adam_steps = 0

    def get_params(self) -> np.ndarray:
        return capi.oasis_net_get_params(self.handle)

    def _stream(self):
        return torch.cuda.current_stream(self.device)

    def forward(self, feat: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        assert feat.dtype == torch.float32 and feat.is_contiguous() and feat.shape == (self.n, 3)
        y = out if out is not None else torch.empty(self.n, dtype=torch.float32, device=self.device)
        capi.oasis_net_forward(self.handle, feat, y, self._stream())
        return y

    def loss_and_grad(self, feat: torch.Tensor, target: torch.Tensor):
        """Loss (device [1]) and gradient (device [N_PARAMS]) of one sample."""
        assert target.dtype == torch.float32 and target.is_contiguous() and target.shape == (self.n,)
        capi.oasis_net_backward(self.handle, feat, target, self.grad, self.loss, self._stream())
        return self.loss, self.grad

    def adam_step(self, lr: float, grad: torch.Tensor | None = None, beta1=0.9, beta2=0.999, eps=1e-8):
        self.adam_steps += 1
        capi.oasis_net_adam(self.handle, self.grad if grad is None else grad, lr, beta1, beta2, eps,
                            self.adam_steps, self._stream())

    def fit(self, samples, epochs: int, lr: float = 2e-3, lr_final: float | None = None):
        """Adam over the recorded samples, one update per sample, cosine-decayed
        learning rate; returns the mean loss of each epoch (read once at the end)."""
        lr_final = lr * 0.05 if lr_final is None else lr_final
        per_epoch = torch.zeros(epochs, dtype=torch.float32, device=self.device)
        total = max(1, epochs * len(samples))
        k = 0
        for e in range(epochs):
            for feat, target in samples:
                c = 0.5 * (1.0 + np.cos(np.pi * k / total))
                self.loss_and_grad(feat, target)
                per_epoch[e] += self.loss[0]
                self.adam_step(lr_final + (lr - lr_final) * c)
                k += 1
        return (per_epoch / len(samples)).cpu().numpy()

    def close(self):
        if self.handle is not None:
            capi.oasis_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
