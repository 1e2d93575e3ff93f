"""Pins for oracle.givens and oracle.metrics: the Haar unit as a signed
pi/4 rotation (Sec. III), rotation algebra, an analytic derivative for the
finite-difference gradient, and the identities of Sec. VI-B."""
import math

import numpy as np
import pytest

from oracle import givens, metrics


def test_haar_unit_is_signed_pi4_rotation():
    """Sec. III: Haar unit = diag(1, -1) Theta^T(1, 2, pi/4): outputs
    (x1 + x2)/sqrt2 and (x1 - x2)/sqrt2."""
    a, b = 0.3, -1.7
    H = np.diag([1.0, -1.0]) @ givens.givens_matrix(2, 0, 1, math.pi / 4).T
    y = H @ np.array([a, b])
    assert np.allclose(y, [(a + b) / math.sqrt(2), (a - b) / math.sqrt(2)], atol=1e-16)


def test_rotation_algebra():
    G1 = givens.givens_matrix(5, 1, 3, 0.4)
    G2 = givens.givens_matrix(5, 1, 3, -1.1)
    assert np.allclose(G1 @ G1.T, np.eye(5), atol=1e-15)
    assert math.isclose(np.linalg.det(G1), 1.0)
    assert np.allclose(G1 @ G2, givens.givens_matrix(5, 1, 3, -0.7), atol=1e-15)
    # theta = pi/2 sends e_p to e_q
    e = np.zeros(5)
    e[1] = 1
    assert np.allclose(givens.givens_matrix(5, 1, 3, math.pi / 2) @ e, np.eye(5)[3], atol=1e-15)


def test_forward_matches_rotation_by_rotation_loop():
    n, S = 8, 4
    pairs = givens.xor_pairs(n, S)
    theta = np.random.default_rng(0).uniform(-3, 3, (S, n // 2))
    X = np.random.default_rng(1).standard_normal((3, n))
    Y = givens.forward(X, pairs, theta)
    for r in range(3):
        v = X[r].copy()
        for s in range(S):
            for (p, q), t in zip(pairs[s], theta[s]):
                vp, vq = v[p], v[q]
                v[p] = math.cos(t) * vp - math.sin(t) * vq
                v[q] = math.sin(t) * vp + math.cos(t) * vq
        assert np.allclose(Y[r], v, atol=1e-14)


def test_fd_gradient_matches_analytic_single_rotation():
    """L(theta) = ||Theta x - t||^2 has dL/dtheta = 2 (Theta x - t) . (dTheta x)
    with dTheta = [[-sin, -cos], [cos, -sin]] on (p, q)."""
    x = np.array([[0.7, -0.2]])
    t = np.array([[0.1, 0.5]])
    pairs = np.array([[[0, 1]]])
    th = np.array([[0.37]])
    c, s = math.cos(0.37), math.sin(0.37)
    r = np.array([[c, -s], [s, c]]) @ x[0] - t[0]
    d = np.array([[-s, -c], [c, -s]]) @ x[0]
    g = givens.loss_grad_fd(x, t, pairs, th)
    assert math.isclose(g[0, 0], 2 * r @ d, rel_tol=1e-8)


def test_xor_pairs_are_perfect_matchings():
    P = givens.xor_pairs(16, 8)
    for s in range(8):
        flat = P[s].ravel()
        assert sorted(flat) == list(range(16))
        assert all(q - p == 1 << (s % 4) for p, q in P[s])


def test_metrics_identities():
    """Eq. 23: RE = ||U - U_hat||_F/||U||_F = ||U_hat^T U - I||_F / sqrt(n) for
    orthogonal matrices; delta is blind to column signs while RE is not;
    epsilon is zero for a sign flip."""
    rng = np.random.default_rng(4)
    U, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    V, _ = np.linalg.qr(U + 0.1 * rng.standard_normal((6, 6)))
    assert math.isclose(metrics.relative_error(V, U),
                        np.linalg.norm(V.T @ U - np.eye(6)) / math.sqrt(6), rel_tol=1e-12)
    assert math.isclose(metrics.relative_error(-U, U), 2.0, rel_tol=1e-12)
    assert metrics.delta(-U, U) < 1e-14
    X = rng.standard_normal((10, 6))
    assert metrics.epsilon(-U, U, X) < 1e-25
    assert metrics.epsilon(V, U, X) > 0
