"""Layered Givens rotations in float64 (test infrastructure only).

Eq. 1 defines the Givens rotation Theta(p, q, theta): Theta_pp = Theta_qq =
cos(theta), Theta_qp = -Theta_pq = sin(theta), identity elsewhere.  Fig. 1
stacks layers of parallel rotations on disjoint pairs into a fast
transform; the learned surrogate is such a stack, y = G_S ... G_1 x, whose
angles are fitted to an exact GFT basis.

Signals are rows: Y = X (G_S ... G_1)^T.

Pins (tests/test_oracle_givens.py): the Haar unit as a signed pi/4 rotation,
rotation algebra (orthogonality, determinant 1, composition of angles, pi/2
maps e_p to e_q), the layered forward against a rotation-by-rotation loop,
central differences against the analytic derivative of a single rotation,
the butterfly pairings as perfect matchings.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np


def givens_matrix(n: int, p: int, q: int, theta: float) -> np.ndarray:
    """Eq. 1, entry by entry."""
    G = np.eye(n)
    c, s = math.cos(theta), math.sin(theta)
    G[p, p] = c
    G[q, q] = c
    G[q, p] = s
    G[p, q] = -s
    return G


def stage_matrix(n: int, pairs: Sequence[Sequence[int]], thetas: Sequence[float]) -> np.ndarray:
    """One layer of parallel rotations on disjoint pairs."""
    G = np.eye(n)
    for (p, q), t in zip(pairs, thetas):
        G = givens_matrix(n, int(p), int(q), float(t)) @ G
    return G


def transform_matrix(n: int, pairs: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """G = G_S ... G_1 for pairs (S, n/2, 2) and theta (S, n/2)."""
    G = np.eye(n)
    for s in range(pairs.shape[0]):
        G = stage_matrix(n, pairs[s], theta[s]) @ G
    return G


def forward(X: np.ndarray, pairs: np.ndarray, theta: np.ndarray) -> np.ndarray:
    n = X.shape[1]
    return np.asarray(X, dtype=np.float64) @ transform_matrix(n, pairs, theta).T


def loss(X, T, pairs, theta) -> float:
    """Squared Frobenius distance between the surrogate's outputs and T."""
    D = forward(X, pairs, theta) - np.asarray(T, dtype=np.float64)
    return float(np.sum(D * D))


def loss_grad_fd(X, T, pairs, theta, h: float = 1e-6) -> np.ndarray:
    """Central finite differences of ``loss`` with respect to every angle."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.zeros_like(theta)
    for idx in np.ndindex(theta.shape):
        tp = theta.copy()
        tm = theta.copy()
        tp[idx] += h
        tm[idx] -= h
        g[idx] = (loss(X, T, pairs, tp) - loss(X, T, pairs, tm)) / (2 * h)
    return g


def xor_pairs(n: int, n_stages: int) -> np.ndarray:
    """Pairings i <-> i XOR 2^(t mod log2 n) for stage t (butterfly wiring);
    each pair listed once with its smaller index first."""
    lg = int(round(math.log2(n)))
    if 1 << lg != n:
        raise ValueError("xor pairing needs n a power of two")
    out = np.zeros((n_stages, n // 2, 2), dtype=np.int32)
    for t in range(n_stages):
        bit = 1 << (t % lg)
        k = 0
        for i in range(n):
            if i & bit == 0:
                out[t, k] = (i, i | bit)
                k += 1
    return out
