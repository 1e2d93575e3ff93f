"""Learned Givens surrogate of a dense GFT for nearly symmetric graphs.

When edge weights break a graph's symmetry (w = 1 + eps * g), no exact Haar
stage exists and the exact GFT is a dense n x n product.  A stack of Givens
rotation layers (Eq. 1, Fig. 1) with fixed butterfly pairings and trainable
angles can stand in for it at O(n log n) cost.  The angles are fitted on the
GPU, through this library's forward and backward kernels, to the exact basis
U that a plan computes (``Plan.basis()``): with the identity as input batch,
the surrogate's outputs are G^T and the loss ||G^T - U||_F^2 equals
||G - U^T||_F^2.  The exact plan stays the fallback and the reference: callers
compare the surrogate's error (``delta``) against their tolerance.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

from . import Givens, givens_apply


def xor_pairs(n: int, n_stages: int) -> np.ndarray:
    """Butterfly wiring: stage t pairs i with i XOR 2^(t mod log2 n)."""
    lg = int(round(math.log2(n)))
    if 1 << lg != n:
        raise ValueError("n must be a power of two")
    out = np.zeros((n_stages, n // 2, 2), dtype=np.int32)
    for t in range(n_stages):
        bit = 1 << (t % lg)
        lo = [i for i in range(n) if not i & bit]
        out[t, :, 0] = lo
        out[t, :, 1] = [i | bit for i in lo]
    return out


def signed_target(U: np.ndarray) -> np.ndarray:
    """A product of rotations has determinant +1: flip the last basis
    vector if the exact basis has determinant -1 (any sign is a valid GFT)."""
    U = np.array(U, dtype=np.float64, copy=True)
    if np.linalg.det(U) < 0:
        U[:, -1] *= -1
    return U


def delta(U_hat: np.ndarray, U: np.ndarray) -> float:
    """Sign-normalised relative error of Sec. VI-B."""
    n = U.shape[0]
    return float(np.linalg.norm(np.abs(U_hat.T @ U) - np.eye(n)) / math.sqrt(n))


class LearnedGFT:
    """Givens surrogate: train(), transform matrix, forward on batches."""

    def __init__(self, n: int, n_stages: Optional[int] = None, device="cuda"):
        import torch
        self.n = n
        self.n_stages = n_stages or 2 * int(round(math.log2(n)))
        self.pairs = xor_pairs(n, self.n_stages)
        self.net = Givens(n, self.pairs)
        self.theta = torch.zeros(self.n_stages, n // 2, device=device, dtype=torch.float32, requires_grad=True)
        self.device = device

    def train(self, U: np.ndarray, steps: int = 1500, lr: float = 0.05):
        """Fit the angles to the exact basis U on the GPU (Adam)."""
        import torch
        Ut = torch.from_numpy(signed_target(U)).float().to(self.device)
        X = torch.eye(self.n, device=self.device)
        opt = torch.optim.Adam([self.theta], lr=lr)
        hist = []
        for it in range(steps):
            Y = givens_apply(X, self.theta, self.net)
            loss = ((Y - Ut) ** 2).sum()
            opt.zero_grad()
            loss.backward()
            opt.step()
            if it % 100 == 0 or it == steps - 1:
                hist.append(float(loss.item()))
        return hist

    def matrix(self) -> np.ndarray:
        """U_hat with the surrogate's coefficients = U_hat^T x."""
        import torch
        with torch.no_grad():
            G_T = self.net.forward(self.theta.detach(), torch.eye(self.n, device=self.device))
        return G_T.double().cpu().numpy()

    def forward(self, x, out=None):
        return self.net.forward(self.theta.detach(), x, out=out)
