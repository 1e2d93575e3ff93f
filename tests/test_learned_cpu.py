"""Host helpers of the learned surrogate (no GPU): the two wirings, the
symmetrisation of the weights over the involutions, the training target of
the learned correction, and the error measures of Sec. VI-B."""
import itertools

import numpy as np
import pytest

import gft_workloads as W
from paper_1907_07875_gb300.learned import (brick_pairs, correction_target, delta, epsilon, signed_target,
                                             symmetrise_weights, xor_pairs)


def _matchings_ok(P, n):
    for stage in P:
        nodes = stage.reshape(-1)
        assert sorted(nodes.tolist()) == list(range(n))      # a perfect matching of the n nodes


@pytest.mark.parametrize("n", [4, 8, 16, 64])
def test_xor_wiring(n):
    P = xor_pairs(n, 2 * int(np.log2(n)))
    _matchings_ok(P, n)
    for t, stage in enumerate(P):
        assert all((a ^ b) == 1 << (t % int(np.log2(n))) for a, b in stage)


@pytest.mark.parametrize("n", [4, 6, 10, 16])
def test_brick_wiring_pairs_neighbours_on_a_ring(n):
    P = brick_pairs(n, 5)
    _matchings_ok(P, n)
    for stage in P:
        assert all((b - a) % n == 1 for a, b in stage)        # ring neighbours only
    with pytest.raises(ValueError):
        brick_pairs(7, 2)


def test_symmetrise_weights_is_the_group_average():
    rng = np.random.default_rng(3)
    N = 4
    g = W.grid(N)
    phis = [np.asarray(W.grid_lr(N)), np.asarray(W.grid_ud(N))]
    Wn = g.W * (1 + 0.3 * rng.standard_normal(g.W.shape))
    Wn = np.triu(Wn, 1)
    Wn = Wn + Wn.T
    Ws = symmetrise_weights(Wn, phis)
    group = [np.arange(g.n), phis[0], phis[1], phis[0][phis[1]]]
    mean = sum(Wn[np.ix_(p, p)] for p in group) / len(group)
    assert np.allclose(Ws, mean)
    for p in phis:
        assert np.allclose(Ws[np.ix_(p, p)], Ws)
    assert np.allclose(symmetrise_weights(Ws, phis), Ws)        # idempotent on symmetric graphs


def _random_orthogonal(n, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    return q


def test_correction_target_is_a_rotation_to_a_signed_basis():
    Us, U = _random_orthogonal(8, 1), _random_orthogonal(8, 2)
    T = correction_target(Us, U)
    assert np.allclose(T.T @ T, np.eye(8)) and np.linalg.det(T) > 0
    # Us T equals U up to the sign of each column
    assert np.allclose(np.abs(Us @ T), np.abs(U))
    for s in itertools.product([1.0, -1.0], repeat=3):
        Uf = U.copy()
        Uf[:, :3] *= np.array(s)
        assert np.allclose(np.abs(Us @ correction_target(Us, Uf)), np.abs(U))


def test_signed_target_has_determinant_one():
    U = _random_orthogonal(6, 4)
    for V in (U, U * np.array([-1, 1, 1, 1, 1, 1.0])):
        S = signed_target(V)
        assert np.linalg.det(S) > 0 and np.allclose(np.abs(S), np.abs(V))


def test_delta_and_epsilon_sign_invariance():
    U = _random_orthogonal(5, 5)
    flipped = U * np.array([1, -1, 1, -1, -1.0])
    assert delta(U, U) < 1e-12 and delta(flipped, U) < 1e-12
    X = np.random.default_rng(6).standard_normal((50, 5))
    assert epsilon(flipped, U, X) < 1e-20
    V = _random_orthogonal(5, 7)
    d = delta(V, U)
    assert d == pytest.approx(np.linalg.norm(np.abs(V.T @ U) - np.eye(5)) / np.sqrt(5))
    assert d > 0.1
