"""Error measures of Sec. VI-B (test infrastructure only).

RE (Eq. 23): ||U - U_hat||_F / ||U||_F.  delta: the sign-normalised version,
||(|U_hat^T U|) - I||_F / sqrt(n).  epsilon: mean over signals of the summed
squared differences of coefficient magnitudes, |u_j^T x| - |u_hat_j^T x|.

Pins (tests/test_oracle_givens.py::test_metrics_identities): Eq. 23's
identity ||U - U_hat||_F / ||U||_F = ||U_hat^T U - I||_F / sqrt(n) for
orthogonal matrices, RE(-U, U) = 2 while delta ignores column signs, epsilon
vanishes for a sign-flipped basis.
"""
from __future__ import annotations

import numpy as np


def relative_error(U_hat: np.ndarray, U: np.ndarray) -> float:
    return float(np.linalg.norm(U - U_hat) / np.linalg.norm(U))


def delta(U_hat: np.ndarray, U: np.ndarray) -> float:
    n = U.shape[0]
    return float(np.linalg.norm(np.abs(U_hat.T @ U) - np.eye(n)) / np.sqrt(n))


def epsilon(U_hat: np.ndarray, U: np.ndarray, X: np.ndarray) -> float:
    """X holds one signal per row."""
    X = np.asarray(X, dtype=np.float64)
    A = np.abs(X @ U)
    B = np.abs(X @ U_hat)
    return float(np.mean(np.sum((A - B) ** 2, axis=1)))
