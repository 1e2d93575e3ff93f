"""Cyclic-by-row Jacobi eigensolver in float64 (test infrastructure only).

The paper builds every GFT from the eigenvectors of a Laplacian (Sec. II-B)
and cites Jacobi's method for its Givens rotations (Sec. I-A).  This is the
textbook cyclic Jacobi method: sweep over all pairs p < q in row order; for
each nonzero a_pq pick the rotation J(p, q, theta) that zeroes it (the
symmetric 2x2 Schur decomposition), update A <- J^T A J and V <- V J; stop
when off(A) <= tol * ||A||_F.

Pins (tests/test_oracle_jacobi.py): LAPACK's eigvalsh on random matrices,
the 2x2 closed form, degenerate spectra, the sweep limit.
"""
from __future__ import annotations

import math

import numpy as np


class NoConvergence(RuntimeError):
    pass


def sym_schur2(app: float, aqq: float, apq: float):
    """(c, s) such that [[c, s], [-s, c]]^T [[app, apq], [apq, aqq]]
    [[c, s], [-s, c]] is diagonal."""
    if apq == 0.0:
        return 1.0, 0.0
    tau = (aqq - app) / (2.0 * apq)
    # smaller root of t^2 + 2 tau t - 1 = 0; hypot avoids overflow of tau^2
    if tau >= 0.0:
        t = 1.0 / (tau + math.hypot(1.0, tau))
    else:
        t = -1.0 / (-tau + math.hypot(1.0, tau))
    c = 1.0 / math.sqrt(1.0 + t * t)
    return c, t * c


def off_norm(A: np.ndarray) -> float:
    """Frobenius norm of the off-diagonal part (summed directly, not as a
    difference of two large sums)."""
    O = A.copy()
    np.fill_diagonal(O, 0.0)
    return math.sqrt(float(np.sum(O * O)))


def jacobi_eigh(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 100):
    """Eigen-decomposition of a real symmetric matrix.  Returns (lam, V) with
    A = V diag(lam) V^T; eigenvalues in the order Jacobi leaves them on the
    diagonal (not sorted).  Raises NoConvergence after max_sweeps."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    fro = math.sqrt(float(np.sum(A * A)))
    sweeps = 0
    while off_norm(A) > tol * fro:
        if sweeps == max_sweeps:
            raise NoConvergence(f"Jacobi: {max_sweeps} sweeps, off={off_norm(A):.3e}")
        sweeps += 1
        for p in range(n - 1):
            for q in range(p + 1, n):
                if A[p, q] == 0.0:
                    continue
                c, s = sym_schur2(A[p, p], A[q, q], A[p, q])
                # columns: A <- A J
                ap, aq = A[:, p].copy(), A[:, q].copy()
                A[:, p] = c * ap - s * aq
                A[:, q] = s * ap + c * aq
                # rows: A <- J^T A
                ap, aq = A[p, :].copy(), A[q, :].copy()
                A[p, :] = c * ap - s * aq
                A[q, :] = s * ap + c * aq
                A[p, q] = A[q, p] = 0.0
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
    return np.diag(A).copy(), V
