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

``CorrectedButterfly`` is the form that gains over the method without the
learned part.  The method without it is the exact butterfly of the graph
with its weights averaged over the involutions (the closest symmetric
graph): Haar stages plus leaf GFTs, U_s.  The learned part is a stack of
Givens layers on that butterfly's coefficients, wired between neighbours in
ascending-eigenvalue order (a perturbation of the weights mixes mostly
eigenvectors of close eigenvalues), trained so that U_s R matches the exact
basis.  With all angles zero it IS the symmetrised butterfly, so training
can only improve on it; the best angles seen are kept.
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


def brick_pairs(n: int, n_stages: int) -> np.ndarray:
    """Neighbour wiring: even stages pair (2i, 2i+1), odd stages pair
    (2i+1, 2i+2) and close the ring with (n-1, 0) (n even)."""
    if n % 2:
        raise ValueError("n must be even")
    out = np.zeros((n_stages, n // 2, 2), dtype=np.int32)
    for t in range(n_stages):
        if t % 2 == 0:
            out[t, :, 0] = np.arange(0, n, 2)
            out[t, :, 1] = np.arange(1, n, 2)
        else:
            out[t, :, 0] = np.append(np.arange(1, n - 1, 2), n - 1)
            out[t, :, 1] = np.append(np.arange(2, n, 2), 0)
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


def epsilon(U_hat: np.ndarray, U: np.ndarray, X: np.ndarray) -> float:
    """Coefficient-magnitude error of Sec. VI-B on signals (rows of X): the
    mean over signals of sum_j (|u_j^T x| - |u_hat_j^T x|)^2."""
    X = np.asarray(X, dtype=np.float64)
    return float(np.mean(np.sum((np.abs(X @ U) - np.abs(X @ U_hat)) ** 2, axis=1)))


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


def symmetrise_weights(Wm: np.ndarray, phis) -> np.ndarray:
    """The closest graph with the given symmetries: edge weights averaged
    over the group generated by the (commuting) involutions, i.e. w_ij
    replaced by the mean over {id, phi_1, phi_2, phi_1 phi_2, ...} of
    w_phi(i)phi(j).  Averaging once per involution in turn gives that mean
    when the involutions commute (reflections of paths, cycles, grids)."""
    Ws = np.array(Wm, dtype=np.float64, copy=True)
    for ph in phis:
        ph = np.asarray(ph)
        Ws = 0.5 * (Ws + Ws[np.ix_(ph, ph)])
    return Ws


def correction_target(U_s: np.ndarray, U: np.ndarray) -> np.ndarray:
    """T = U_s^T U' with U' = U up to column signs (each a valid GFT): signs
    that make T's diagonal non-negative, then, if det T = -1 (a product of
    rotations has determinant +1), the column of smallest |T_jj| flipped."""
    T = U_s.T @ U
    sg = np.where(np.diag(T) < 0, -1.0, 1.0)
    T = T * sg
    if np.linalg.det(T) < 0:
        j = int(np.argmin(np.abs(np.diag(T))))
        T[:, j] *= -1
    return T


class CorrectedButterfly:
    """Symmetrised butterfly (a plan of the averaged graph) followed by
    learned Givens layers on its coefficients: y = G (U_s^T x), with the
    surrogate basis U_hat = U_s G^T."""

    def __init__(self, plan_sym, n_stages: Optional[int] = None, device="cuda"):
        import torch
        self.plan = plan_sym
        self.n = n = plan_sym.n
        self.n_stages = n_stages or 2 * int(math.ceil(math.log2(n)))
        self.pairs = brick_pairs(n, self.n_stages)
        self.net = Givens(n, self.pairs)
        self.theta = torch.zeros(self.n_stages, n // 2, device=device, dtype=torch.float32, requires_grad=True)
        self.device = device
        self.U_s = plan_sym.basis()

    def _G_T(self, theta):
        import torch
        with torch.no_grad():
            return self.net.forward(theta.detach(), torch.eye(self.n, device=self.device)).double().cpu().numpy()

    def train(self, U: np.ndarray, steps: int = 1500, lr: float = 0.01):
        """Fit the angles on the GPU (Adam, identity inputs, loss
        ||G^T - T||_F^2 with T = correction_target(U_s, U)); keeps the
        angles of the smallest delta seen, starting from zero (delta of the
        symmetrised butterfly itself)."""
        import torch
        T = torch.from_numpy(correction_target(self.U_s, U)).float().to(self.device)
        X = torch.eye(self.n, device=self.device)
        opt = torch.optim.Adam([self.theta], lr=lr)
        best_d = delta(self.U_s, U)
        best = self.theta.detach().clone()
        hist = []
        for it in range(steps):
            Y = givens_apply(X, self.theta, self.net)
            loss = ((Y - T) ** 2).sum()
            opt.zero_grad()
            loss.backward()
            opt.step()
            if it % 50 == 0 or it == steps - 1:
                d = delta(self.U_s @ self._G_T(self.theta), U)
                hist.append((float(loss.item()), d))
                if d < best_d:
                    best_d, best = d, self.theta.detach().clone()
        with torch.no_grad():
            self.theta.copy_(best)
        return hist

    def matrix(self) -> np.ndarray:
        """U_hat: the surrogate's coefficients are U_hat^T x."""
        return self.U_s @ self._G_T(self.theta)

    def forward(self, x, out=None, tmp=None):
        """Butterfly of the averaged graph, then the learned layers."""
        import torch
        c = self.plan.forward(x, out=tmp)
        if out is None:
            out = torch.empty_like(x)
        return self.net.forward(self.theta.detach(), c, out=out)
