"""Approximate GFT by layers of Givens rotations, alone and after the Haar
stages ("Haar + approximate GFT", Sec. VI-B), in float64 (test
infrastructure only).

Approximate GFT (the comparison method of Sec. VI-B; its code is not in the
paper, which cites the parallel truncated Jacobi algorithm of Le Magoarou
et al.): starting from A = L, layer t picks disjoint node pairs greedily by
the magnitude of the current off-diagonal entries (largest |a_pq| first,
ties by (p, q) order, until no entry with two free nodes is left; entries
of at most 1e-14 max(1, max|L|) count as zero, and a layer with nothing to
pair ends the run) and for
each pair the rotation J(p, q, theta) that zeroes a_pq (the symmetric 2x2
Schur decomposition); the layer's rotations commute and are applied at
once, A <- J_t^T A J_t.  After J layers U_hat = J_1 ... J_J, the
coefficients are U_hat^T x, and the final permutation (Fig. 1's Pi_{J+1})
orders them by the diagonal of A (the approximate eigenvalues), ascending.

Haar + approximate GFT: the Haar stages of the symmetric decomposition
(Sec. IV, Eq. 20 per stage: (a+b)/sqrt2 at X, (a-b)/sqrt2 at the partner)
followed by the approximate GFT of every leaf Laplacian (J layers each, the
leaves side by side), outputs ordered by approximate eigenvalue with ties by
(leaf, index) as in ``gft.output_order``.

The transform is kept as layers of 2x2 units (p, q, m) acting as
(x_p, x_q) <- (m00 x_p + m01 x_q, m10 x_p + m11 x_q): a Haar unit is
m = [[1, 1], [1, -1]] / sqrt2, a rotation J^T is m = [[c, -s], [s, c]].

Pins (tests/test_oracle_approx.py): choose_pairs / truncated_jacobi -- the
2x2 closed form, Jacobi's off-norm identity per layer, greedy order and
maximality; haar_approx_gft -- convergence to the exact GFT, the Haar-only
case against Eq. 20's stage matrices and Thm. 3's blocks, Rayleigh-quotient
eigenvalues, the Sec. VI-B observation on both 8x8 grids; forward /
apply_units -- equal to the dense product.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Sequence, Tuple

import numpy as np

from .gft import decompose, output_order
from .jacobi import sym_schur2

SQRT2 = math.sqrt(2.0)

Unit = Tuple[int, int, Tuple[float, float, float, float]]


ZERO_TOL = 1e-14      # off-diagonal entries at most this x max(1, max|L|) count as zero


def choose_pairs(A: np.ndarray, tol: float = 0.0) -> List[Tuple[int, int]]:
    """One layer's greedy pairing over the upper triangle: entries with
    |a_pq| > tol by decreasing magnitude (ties by (p, q)), taken while both
    nodes are still free."""
    m = A.shape[0]
    cand = [(-abs(A[p, q]), p, q) for p in range(m) for q in range(p + 1, m) if abs(A[p, q]) > tol]
    cand.sort()
    used = [False] * m
    out = []
    for _, p, q in cand:
        if not used[p] and not used[q]:
            used[p] = used[q] = True
            out.append((p, q))
    return out


def truncated_jacobi(L: np.ndarray, n_layers: int):
    """(layers, A): layers[t] = [(p, q, c, s)], A = J^T L J after them."""
    A = np.array(L, dtype=np.float64, copy=True)
    tol = ZERO_TOL * max(1.0, float(np.max(np.abs(A)))) if A.size else 0.0
    layers = []
    for _ in range(n_layers):
        pairs = choose_pairs(A, tol)
        if not pairs:
            break
        rots = [(p, q) + sym_schur2(A[p, p], A[q, q], A[p, q]) for p, q in pairs]
        for p, q, c, s in rots:                    # columns: A <- A J
            ap, aq = A[:, p].copy(), A[:, q].copy()
            A[:, p] = c * ap - s * aq
            A[:, q] = s * ap + c * aq
        for p, q, c, s in rots:                    # rows: A <- J^T A
            ap, aq = A[p, :].copy(), A[q, :].copy()
            A[p, :] = c * ap - s * aq
            A[q, :] = s * ap + c * aq
        for p, q, _, _ in rots:
            A[p, q] = A[q, p] = 0.0
        layers.append(rots)
    return layers, A


@dataclass
class ApproxGFT:
    n: int
    layers: List[List[Unit]]    # Haar stages first, then the Givens layers
    perm: np.ndarray            # coefficient j is read from node perm[j]
    lam: np.ndarray             # approximate eigenvalues, output order
    U: np.ndarray               # U_hat, columns in output order
    n_haar: int                 # leading Haar layers


def apply_units(layers, X: np.ndarray) -> np.ndarray:
    """Every unit in order on every row of X (one signal per row)."""
    W = np.array(X, dtype=np.float64, copy=True)
    for layer in layers:
        for p, q, (m00, m01, m10, m11) in layer:
            a, b = W[:, p].copy(), W[:, q].copy()
            W[:, p] = m00 * a + m01 * b
            W[:, q] = m10 * a + m11 * b
    return W


def haar_approx_gft(L: np.ndarray, phis: Sequence[Sequence[int]], n_layers: int,
                    split_components: bool = False) -> ApproxGFT:
    """phis = [] gives the plain approximate GFT (one leaf: the graph)."""
    fact = decompose(L, phis, split_components)
    n = fact.n
    r = 1.0 / SQRT2
    layers: List[List[Unit]] = [[(x, y, (r, r, r, -r)) for x, y in st] for st in fact.stages]
    n_haar = len(layers)
    leaf_layers, entries, slots = [], [], []
    for k, leaf in enumerate(fact.leaves):
        rots, A = truncated_jacobi(leaf.L, n_layers)
        leaf_layers.append([[(leaf.labels[p], leaf.labels[q], (c, -s, s, c)) for p, q, c, s in lay]
                            for lay in rots])
        for i, lab in enumerate(leaf.labels):
            entries.append((float(A[i, i]), k, i))
            slots.append(lab)
    depth = max((len(v) for v in leaf_layers), default=0)
    for t in range(depth):
        layers.append([u for v in leaf_layers if t < len(v) for u in v[t]])
    pos = output_order(entries)
    perm = np.zeros(n, dtype=np.int64)
    lam = np.zeros(n)
    for i, (l, _, _) in enumerate(entries):
        perm[pos[i]] = slots[i]
        lam[pos[i]] = l
    U = apply_units(layers, np.eye(n))[:, perm]
    return ApproxGFT(n, layers, perm, lam, U, n_haar)


def forward(f: ApproxGFT, X: np.ndarray) -> np.ndarray:
    """Coefficients U_hat^T x of every row of X, in output order."""
    return apply_units(f.layers, X)[:, f.perm]
