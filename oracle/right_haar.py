"""Right Haar stage for bipartite graphs, in float64 (test infrastructure only).

Sec. III-A ("Conditions for Right Haar Units"): a GFT with a right butterfly
stage of p Haar units computes U^T x = B_{n,p} diag(E^T, F^T) x (Eq. 8, with
B_{n,p} of Eq. 7), i.e. two independent sub-transforms E (on one part of the
nodes) and F (on the other) followed by p Haar units on the outputs; the
columns of U then come in pairs (e; f) / sqrt2 and (e; -f) / sqrt2 (Eq. 9).
Lemma 1 and Thm. 1: the Laplacian of a k-regular bipartite graph has such a
GFT with p = n/2; Thm. 2: so does the normalised Laplacian of any bipartite
graph, with p = the size of the smaller part.

Both cases share one structure, which is what this module checks and uses:
with the parts S1, S2 (every edge joins them), L[S1, S1] = alpha I and
L[S2, S2] = alpha I (alpha = k, resp. 1), so with C = -L[S1, S2]
    L (a; b) = (alpha a - C b; alpha b - C^T a).
For a singular triple C q = sigma a, C^T a = sigma q this gives
L (a; q) = (alpha - sigma)(a; q) and L (a; -q) = (alpha + sigma)(a; -q)
(Lemma 1's pairing u <-> (u1; -u2), eigenvalues mirrored about alpha), and
the left singular vectors of C beyond its smaller dimension are
eigenvectors (a; 0) with eigenvalue alpha.  So E = the left singular
vectors of C on the larger part, F = the right singular vectors on the
smaller part, p = |smaller part|; Thm. 1's constructive proof pairs the
eigenvectors in the same way.  The SVD is numpy's (a library routine).

Readings (listed in the design notes): the larger part is E's (the first
n - p entries in Eq. 8), the smaller part F's; ties go to the part of
colour 0.  Within a part, nodes are in ascending label order.  Pair c puts
the sum (the (e; f) vector, eigenvalue alpha - sigma_c) in E's column c and
the difference in F's column c.  Output order: ascending eigenvalue with
clusters ordered by (E before F, column index); signs: the canonical sign
rule of ``gft`` is applied to each sum vector (and to each unpaired
vector), the difference vector of a pair follows it.

Pins (tests/test_oracle_right_haar.py): closed-form spectra (even cycles,
hypercubes, complete bipartite normalised), the mirrored spectrum against
LAPACK's eigvalsh, Eq. 9's pair structure and E^T C F = diag(sigma), staged
against dense transforms, op_counts, the structural rejections.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional, Tuple

import numpy as np

from .gft import canonical_sign, output_order
from .graph import bipartition

SQRT2 = math.sqrt(2.0)
STRUCT_TOL = 1e-12      # alpha I blocks and zero within-part entries, x max(1, max|L|)


@dataclass
class RightHaarGFT:
    n: int
    alpha: float
    big: List[int]          # labels of E's part (ascending)
    small: List[int]        # labels of F's part (ascending)
    E: np.ndarray           # |big| x |big|, columns orthonormal
    F: np.ndarray           # |small| x |small|
    sigma: np.ndarray       # |small| singular values of C, column c of E / F
    pos: np.ndarray         # output index of entry i (E columns, then F columns)
    lam: np.ndarray         # eigenvalues in output order
    U: np.ndarray           # n x n basis, columns in output order

    @property
    def p(self) -> int:
        return len(self.small)


def right_structure(L: np.ndarray, side: Optional[np.ndarray] = None) -> Tuple[float, List[int], List[int]]:
    """(alpha, big part, small part) if L has the structure above for the
    two-colouring `side` (found from L's off-diagonal pattern if None);
    raises ValueError otherwise."""
    L = np.asarray(L, dtype=np.float64)
    n = L.shape[0]
    tol = STRUCT_TOL * max(1.0, float(np.max(np.abs(L))))
    if side is None:
        side = bipartition(L, tol)
        if side is None:
            raise ValueError("graph is not bipartite")
    side = np.asarray(side)
    S = [[i for i in range(n) if side[i] == c] for c in (0, 1)]
    alpha = float(L[0, 0])
    for i in range(n):
        if abs(L[i, i] - alpha) > tol:
            raise ValueError(f"diagonal entry {i} differs from alpha = {alpha}")
    for part in S:
        for i in part:
            for j in part:
                if i != j and abs(L[i, j]) > tol:
                    raise ValueError(f"entry ({i}, {j}) joins two nodes of one part")
    big, small = (S[0], S[1]) if len(S[0]) >= len(S[1]) else (S[1], S[0])
    return alpha, big, small


def right_haar_gft(L: np.ndarray, side: Optional[np.ndarray] = None) -> RightHaarGFT:
    L = np.asarray(L, dtype=np.float64)
    n = L.shape[0]
    alpha, big, small = right_structure(L, side)
    m1, p = len(big), len(small)
    C = -L[np.ix_(big, small)]
    if p > 0:
        P, sig, QT = np.linalg.svd(C, full_matrices=True)
        E, F = P.copy(), QT.T.copy()
    else:
        E, F, sig = np.eye(m1), np.zeros((0, 0)), np.zeros(0)
    sig = np.asarray(sig[:p], dtype=np.float64)
    cols, entries = [], []
    # paired columns: sum vector (E_c; F_c)/sqrt2 and difference (E_c; -F_c)/sqrt2
    for c in range(p):
        v = np.zeros(n)
        v[big] = E[:, c] / SQRT2
        v[small] = F[:, c] / SQRT2
        sg = canonical_sign(v)
        E[:, c] *= sg
        F[:, c] *= sg
    for c in range(m1):
        v = np.zeros(n)
        if c < p:
            v[big] = E[:, c] / SQRT2
            v[small] = F[:, c] / SQRT2
            entries.append((alpha - float(sig[c]), 0, c))
        else:
            v[big] = E[:, c]
            sg = canonical_sign(v)
            E[:, c] *= sg
            v *= sg
            entries.append((alpha, 0, c))
        cols.append(v)
    for c in range(p):
        v = np.zeros(n)
        v[big] = E[:, c] / SQRT2
        v[small] = -F[:, c] / SQRT2
        cols.append(v)
        entries.append((alpha + float(sig[c]), 1, c))
    pos = output_order(entries)
    U = np.zeros((n, n))
    lam = np.zeros(n)
    for i, (l, _, _) in enumerate(entries):
        U[:, pos[i]] = cols[i]
        lam[pos[i]] = l
    return RightHaarGFT(n, alpha, big, small, E, F, sig, pos, lam, U)


def forward_staged(f: RightHaarGFT, X: np.ndarray) -> np.ndarray:
    """Eq. 8 on every row: a = E^T x[big], b = F^T x[small], then the right
    Haar units (a_c + b_c)/sqrt2 and (a_c - b_c)/sqrt2 for c < p, a_c
    unchanged for c >= p; coefficients placed in output order."""
    X = np.asarray(X, dtype=np.float64)
    m1, p = len(f.big), f.p
    a = X[:, f.big] @ f.E
    b = X[:, f.small] @ f.F
    Y = np.zeros_like(X)
    Y[:, f.pos[:p]] = (a[:, :p] + b) / SQRT2
    Y[:, f.pos[p:m1]] = a[:, p:]
    Y[:, f.pos[m1:]] = (a[:, :p] - b) / SQRT2
    return Y


def inverse_staged(f: RightHaarGFT, Y: np.ndarray) -> np.ndarray:
    """x = diag(E, F) B_{n,p}^T y: the Haar units on the coefficient pairs
    first, then the two sub-transforms."""
    Y = np.asarray(Y, dtype=np.float64)
    m1, p = len(f.big), f.p
    ys, yd = Y[:, f.pos[:p]], Y[:, f.pos[m1:]]
    a = np.zeros((Y.shape[0], m1))
    a[:, :p] = (ys + yd) / SQRT2
    a[:, p:] = Y[:, f.pos[p:m1]]
    b = (ys - yd) / SQRT2
    X = np.zeros_like(Y)
    X[:, f.big] = a @ f.E.T
    X[:, f.small] = b @ f.F.T
    return X


def op_counts(f: RightHaarGFT) -> Tuple[int, int]:
    """(additions, multiplications) per signal with the 1/sqrt2 factors
    folded into E and F: |big|^2 + |small|^2 multiplies (the count
    p^2 + (n-p)^2 of Sec. V-G for one stage), m(m-1) adds per
    sub-transform and 2 per right Haar unit."""
    m1, p = len(f.big), f.p
    return m1 * (m1 - 1) + p * (p - 1) + 2 * p, m1 * m1 + p * p
