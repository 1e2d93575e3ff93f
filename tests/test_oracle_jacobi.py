"""Pins for oracle.jacobi: agreement with LAPACK (numpy.linalg.eigh) on
random and degenerate symmetric matrices, 2x2 closed form, residual and
orthogonality, and the sweep limit."""
import math

import numpy as np
import pytest

from oracle import jacobi
from _helpers import projector_distance


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (7, 3), (16, 4), (33, 5)])
def test_matches_lapack(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    A = A + A.T
    lam, V = jacobi.jacobi_eigh(A)
    order = np.argsort(lam)
    lam, V = lam[order], V[:, order]
    ref_lam, ref_V = np.linalg.eigh(A)
    scale = np.linalg.norm(A)
    assert np.max(np.abs(lam - ref_lam)) <= 1e-13 * scale
    assert np.max(np.abs(V.T @ V - np.eye(n))) <= 1e-13
    assert np.max(np.abs(A @ V - V * lam)) <= 1e-12 * scale
    assert projector_distance(V, ref_V, ref_lam, tol=1e-9) <= 1e-10


def test_two_by_two_closed_form():
    a, b, d = 2.0, 0.5, -1.0
    lam, V = jacobi.jacobi_eigh(np.array([[a, b], [b, d]]))
    mid, rad = (a + d) / 2, math.hypot((a - d) / 2, b)
    assert np.allclose(np.sort(lam), [mid - rad, mid + rad], atol=1e-15)
    c, s = jacobi.sym_schur2(a, d, b)
    J = np.array([[c, s], [-s, c]])
    B = J.T @ np.array([[a, b], [b, d]]) @ J
    assert abs(B[0, 1]) < 1e-15 and math.isclose(c * c + s * s, 1.0)


def test_degenerate_spectra():
    # repeated eigenvalues: an orthogonal similarity of diag(1,1,1,3,3)
    rng = np.random.default_rng(9)
    Q, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    A = Q @ np.diag([1.0, 1.0, 1.0, 3.0, 3.0]) @ Q.T
    lam, V = jacobi.jacobi_eigh(A)
    assert np.allclose(np.sort(lam), [1, 1, 1, 3, 3], atol=1e-13)
    assert np.max(np.abs(A @ V - V * lam)) < 1e-12
    # already diagonal / zero: no rotation needed
    lam, V = jacobi.jacobi_eigh(np.diag([3.0, -1.0, 2.0]))
    assert np.array_equal(lam, [3.0, -1.0, 2.0]) and np.array_equal(V, np.eye(3))
    lam, V = jacobi.jacobi_eigh(np.zeros((4, 4)))
    assert np.array_equal(lam, np.zeros(4))


def test_sweep_limit_raises():
    A = np.random.default_rng(1).standard_normal((12, 12))
    with pytest.raises(jacobi.NoConvergence):
        jacobi.jacobi_eigh(A + A.T, max_sweeps=1)
