"""Graph algebra of the paper, written out in float64 (test infrastructure only).

Sec. II-B: Laplacian L = D - W + S (Eq. 3) and the weight/Laplacian
conversions (Eqs. 4 and 5).  Sec. IV-A: involutions and phi-symmetric graphs
(Definitions 1 and 2, p_phi of Eq. 19).  Sec. IV-B: node partition X/Y/Z and
the permuted butterfly matrix B_phi (Eq. 20), block diagonalisation
L_phi = B_phi^T L B_phi (Thm. 3).  Sec. IV-C: the weights and self-loops of
G+ and G- in closed form (Thm. 4, proof in the Appendix), and the even/odd
components of a signal (Eq. 21).

Pins (tests/test_oracle_graph.py, tests/test_oracle_right_haar.py):
laplacian -- the quadratic form sum w_ij (x_i - x_j)^2 + sum s_i x_i^2 and the
Eq. 4 / 5 round trip; is_involution / partition / b_phi -- Definition 1,
orthogonality, the Haar action; block_diagonalize / thm4_subgraphs -- Thm. 3's
zero off-blocks and Thm. 4's weights against the congruence, the edge
removal cases; even_odd -- Eq. 21; connected_components; normalized_laplacian
-- a hand-computed case and the complete bipartite spectrum {0, 1, 2};
bipartition -- a hand-checked two-colouring and an odd cycle.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np

SQRT2 = math.sqrt(2.0)


def laplacian(W: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Eq. 5: l_ii = s_i + sum_{j != i} w_ij, l_ij = -w_ij (i != j)."""
    W = np.asarray(W, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    n = W.shape[0]
    L = np.zeros((n, n))
    for i in range(n):
        acc = s[i]
        for j in range(n):
            if j != i:
                acc += W[i, j]
                L[i, j] = -W[i, j]
        L[i, i] = acc
    return L


def weights_from_laplacian(L: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Eq. 4: s_i = sum_j l_ij, w_ij = -l_ij (i != j)."""
    L = np.asarray(L, dtype=np.float64)
    n = L.shape[0]
    s = np.array([sum(L[i, j] for j in range(n)) for i in range(n)])
    W = -L.copy()
    np.fill_diagonal(W, 0.0)
    return W, s


def is_involution(phi) -> bool:
    """Definition 1: phi is a permutation with phi(phi(i)) = i."""
    phi = np.asarray(phi)
    n = len(phi)
    if phi.min(initial=0) < 0 or phi.max(initial=0) >= n:
        return False
    return all(int(phi[int(phi[i])]) == i for i in range(n))


def is_phi_symmetric(W, s, phi, tol: float = 0.0) -> bool:
    """Definition 2: w_ij = w_{phi(i) phi(j)} for all i, j, including the
    self-loops s_i = s_{phi(i)}."""
    n = len(phi)
    for i in range(n):
        if abs(s[i] - s[phi[i]]) > tol:
            return False
        for j in range(n):
            if abs(W[i, j] - W[phi[i], phi[j]]) > tol:
                return False
    return True


def laplacian_is_phi_symmetric(L, phi, tol: float) -> bool:
    """Definition 2 read on the Laplacian: by Eqs. 4-5 the graph is
    phi-symmetric iff l_ij = l_{phi(i) phi(j)} for all i, j."""
    n = len(phi)
    for i in range(n):
        for j in range(n):
            if abs(L[i, j] - L[phi[i], phi[j]]) > tol:
                return False
    return True


def p_phi(phi) -> int:
    """Eq. 19: number of Haar units = half the number of non-fixed nodes."""
    return sum(1 for i in range(len(phi)) if phi[i] != i) // 2


def partition(phi) -> Tuple[List[int], List[int], List[int]]:
    """Sec. IV-B: Z = fixed points of phi; each pair {i, phi(i)} puts its
    smaller index in X and its partner in Y.  Y is returned in partner order
    (Y[k] = phi(X[k])), X and Z ascending."""
    n = len(phi)
    X = [i for i in range(n) if phi[i] > i]
    Z = [i for i in range(n) if phi[i] == i]
    Y = [int(phi[i]) for i in X]
    return X, Y, Z


def b_phi(phi) -> np.ndarray:
    """Eq. 20: the permuted butterfly matrix B_phi."""
    n = len(phi)
    X, Y, Z = partition(phi)
    B = np.zeros((n, n))
    r = 1.0 / SQRT2
    for i in X:
        B[i, i] = r
        B[i, phi[i]] = r
    for i in Y:
        B[i, i] = -r
        B[i, phi[i]] = r
    for i in Z:
        B[i, i] = 1.0
    return B


def block_diagonalize(L, phi):
    """Thm. 3: L_phi = B_phi^T L B_phi by dense products.  Returns
    (L_plus, L_minus, offblock) where L_plus is L_phi on X then Z (rows and
    columns), L_minus is L_phi on Y in partner order, and offblock is the
    largest |entry| of L_phi coupling X u Z with Y (zero in exact arithmetic
    for a phi-symmetric graph)."""
    L = np.asarray(L, dtype=np.float64)
    B = b_phi(phi)
    Lphi = B.T @ L @ B
    X, Y, Z = partition(phi)
    P = X + Z
    Lp = Lphi[np.ix_(P, P)]
    Lm = Lphi[np.ix_(Y, Y)]
    off = float(np.max(np.abs(Lphi[np.ix_(P, Y)]))) if (P and Y) else 0.0
    return Lp, Lm, off


def thm4_subgraphs(W, s, phi):
    """Thm. 4: weights and self-loops of G+ (nodes X then Z) and G- (nodes Y
    in partner order) in closed form.  Returns (W+, s+, W-, s-)."""
    X, Y, Z = partition(phi)
    P = X + Z
    Xs, Zs = set(X), set(Z)
    npl, nm = len(P), len(Y)
    Wp, sp = np.zeros((npl, npl)), np.zeros(npl)
    Wm, sm = np.zeros((nm, nm)), np.zeros(nm)
    for a, i in enumerate(P):
        for b, j in enumerate(P):
            if a == b:
                continue
            if i in Xs and j in Xs:
                Wp[a, b] = W[i, j] + W[i, phi[j]]
            elif i in Zs and j in Zs:
                Wp[a, b] = W[i, j]
            else:  # one in X, the other in Z
                Wp[a, b] = SQRT2 * W[i, j]
        if i in Xs:
            sp[a] = s[i] - (SQRT2 - 1.0) * sum(W[i, j] for j in Z)
        else:
            sp[a] = s[i] + (2.0 - SQRT2) * sum(W[i, j] for j in X)
    for a, i in enumerate(Y):
        for b, j in enumerate(Y):
            if a != b:
                Wm[a, b] = W[i, j] - W[i, phi[j]]
        sm[a] = s[i] + 2.0 * sum(W[i, j] for j in X) + sum(W[i, j] for j in Z)
    return Wp, sp, Wm, sm


def even_odd(x_plus, x_minus, phi):
    """Eq. 21: even/odd node-domain components from the Haar outputs.
    x_plus is indexed like G+ (X then Z), x_minus like G- (Y)."""
    X, Y, Z = partition(phi)
    n = len(phi)
    xe, xo = np.zeros(n), np.zeros(n)
    pos_plus = {v: k for k, v in enumerate(X + Z)}
    pos_minus = {v: k for k, v in enumerate(Y)}
    r = 1.0 / SQRT2
    for i in X:
        xe[i] = x_plus[pos_plus[i]] * r
        xo[i] = x_minus[pos_minus[phi[i]]] * r
    for i in Y:
        xe[i] = x_plus[pos_plus[phi[i]]] * r
        xo[i] = -x_minus[pos_minus[i]] * r
    for i in Z:
        xe[i] = x_plus[pos_plus[i]]
        xo[i] = 0.0
    return xe, xo


def connected_components(L, tol: float = 0.0) -> List[List[int]]:
    """Components of the graph whose edges are the nonzero off-diagonal
    entries of L; each component ascending, components ordered by their
    smallest index."""
    n = L.shape[0]
    seen = [False] * n
    comps = []
    for r in range(n):
        if seen[r]:
            continue
        stack, comp = [r], []
        seen[r] = True
        while stack:
            v = stack.pop()
            comp.append(v)
            for u in range(n):
                if u != v and not seen[u] and abs(L[v, u]) > tol:
                    seen[u] = True
                    stack.append(u)
        comps.append(sorted(comp))
    return comps


def normalized_laplacian(W: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Symmetric normalised Laplacian D^-1/2 L D^-1/2 (Sec. II-B), with
    L = D - W + S (Eq. 3) and degrees d_i = sum_j w_ij, the self-loop w_ii = s_i
    included.  Every degree must be positive."""
    W = np.asarray(W, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    n = W.shape[0]
    d = np.zeros(n)
    for i in range(n):
        d[i] = s[i] + sum(W[i, j] for j in range(n) if j != i)
        if d[i] <= 0:
            raise ValueError(f"node {i} has degree {d[i]}")
    L = laplacian(W, s)
    N = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            N[i, j] = L[i, j] / math.sqrt(d[i] * d[j])
    return N


def bipartition(L, tol: float = 0.0):
    """Two-colouring of the graph whose edges are the nonzero off-diagonal
    entries of L (Sec. II-B: every edge joins the two parts).  Each
    connected component gives colour 0 to its smallest node.  Returns an
    int array of 0 / 1 per node, or None if some component has an odd cycle."""
    n = L.shape[0]
    side = [-1] * n
    for r in range(n):
        if side[r] >= 0:
            continue
        side[r] = 0
        queue = [r]
        while queue:
            v = queue.pop(0)
            for u in range(n):
                if u == v or abs(L[v, u]) <= tol:
                    continue
                if side[u] < 0:
                    side[u] = 1 - side[v]
                    queue.append(u)
                elif side[u] == side[v]:
                    return None
    return np.array(side, dtype=np.int32)
