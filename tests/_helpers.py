"""Comparison helpers for bases defined only up to sign and rotation inside
repeated eigenvalues (Sec. III: the GFT is not unique when an eigenvalue is
repeated).  Pure numpy; no transform arithmetic."""
from __future__ import annotations

import numpy as np


def clusters(lam, tol: float = 1e-9):
    """Index groups of consecutive (ascending) eigenvalues closer than
    tol * max(1, max|lam|)."""
    lam = np.asarray(lam, dtype=np.float64)
    if lam.size == 0:
        return []
    t = tol * max(1.0, float(np.max(np.abs(lam))))
    out, cur = [], [0]
    for j in range(1, lam.size):
        if lam[j] - lam[j - 1] > t:
            out.append(cur)
            cur = []
        cur.append(j)
    out.append(cur)
    return out


def projector_distance(Ua, Ub, lam, tol: float = 1e-9) -> float:
    """Largest Frobenius distance between the eigenspace projectors."""
    worst = 0.0
    for S in clusters(lam, tol):
        Pa = Ua[:, S] @ Ua[:, S].T
        Pb = Ub[:, S] @ Ub[:, S].T
        worst = max(worst, float(np.linalg.norm(Pa - Pb)))
    return worst


def align(Y_ref, U_test, U_ref, lam, tol: float = 1e-9):
    """Express reference coefficients in the test basis, eigenspace by
    eigenspace: y_test,S = (U_test,S^T U_ref,S) y_ref,S."""
    Y_ref = np.asarray(Y_ref, dtype=np.float64)
    out = np.empty_like(Y_ref)
    for S in clusters(lam, tol):
        Q = U_test[:, S].T @ U_ref[:, S]
        out[:, S] = Y_ref[:, S] @ Q.T
    return out


def simple_column_sign_error(U_test, U_ref, lam, tol: float = 1e-9) -> float:
    """Largest entrywise difference over the columns of simple eigenvalues
    (clusters of one).  Their vectors are unique up to sign, and the sign
    rule fixes the sign, so these columns must agree entry by entry: a sign
    flip shows up as an O(1) difference."""
    worst = 0.0
    for S in clusters(lam, tol):
        if len(S) == 1:
            j = S[0]
            worst = max(worst, float(np.max(np.abs(np.asarray(U_test)[:, j] - np.asarray(U_ref)[:, j]))))
    return worst


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / (nb if nb > 0 else 1.0)


def sign_normalize(U):
    """Flip each column so that its largest-magnitude entry (first on ties)
    is positive; used to compare against closed forms."""
    U = np.array(U, dtype=np.float64, copy=True)
    for c in range(U.shape[1]):
        a = np.abs(U[:, c])
        i = int(np.nonzero(a >= (1 - 1e-9) * a.max())[0][0])
        if U[i, c] < 0:
            U[:, c] *= -1
    return U


def read_golden_matrix(path):
    """Parse a tests/golden/*.txt matrix fixture: '#' comments, optional
    'key: values' lines, then rows of numbers."""
    meta, rows = {}, []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if ":" in line:
                k, v = line.split(":", 1)
                meta[k.strip()] = [float(t) for t in v.split()]
                continue
            rows.append([float(t) for t in line.split()])
    return meta, np.array(rows)
