"""Pins for oracle.approx (approximate GFT by greedy layers of Givens
rotations, alone and after the Haar stages, Sec. VI-B):

* a 2x2 matrix is diagonalised by one rotation, eigenvalues = eigvalsh's;
* Jacobi's identity per layer: off(A)^2 drops by exactly 2 * sum a_pq^2 of
  the zeroed entries (disjoint rotations), and the zeroed entries are 0;
* the greedy pairing is disjoint, starts with the largest |a_pq| and is
  maximal (no nonzero entry joins two free nodes);
* with enough layers U_hat converges to the exact GFT (delta -> 0, the
  approximate eigenvalues to eigvalsh's), alone and after the Haar stages;
* with no layers, Haar + approximate is the Haar stages alone: U_hat^T L U_hat
  is block diagonal with the leaf Laplacians of Thm. 3 as blocks;
* the staged forward equals x U_hat; U_hat is orthogonal;
* the paper's observation for its two grids (Sec. VI-B): at equal layer
  counts the Haar + approximate GFT is closer to the exact GFT than the
  approximate GFT alone.
A transposed rotation, a wrong Haar sign or a dropped layer fails them.
"""
import math

import numpy as np
import pytest

import gft_workloads as W
from oracle import approx as A
from oracle import gft, graph, metrics


def _L(g):
    return graph.laplacian(g.W, g.s)


def _off2(M):
    O = M.copy()
    np.fill_diagonal(O, 0.0)
    return float(np.sum(O * O))


def test_single_rotation_diagonalises_2x2():
    rng = np.random.default_rng(5)
    for _ in range(20):
        a, b, c = rng.standard_normal(3)
        M = np.array([[a, c], [c, b]])
        layers, Af = A.truncated_jacobi(M, 1)
        assert len(layers) == 1 and len(layers[0]) == 1
        assert abs(Af[0, 1]) == 0.0
        _, _, cc, ss = layers[0][0]
        J = np.array([[cc, ss], [-ss, cc]])
        D = J.T @ M @ J
        assert abs(D[0, 1]) <= 1e-15 * max(1, abs(M).max())
        assert np.allclose(np.sort(np.diag(Af)), np.linalg.eigvalsh(M), atol=1e-14)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_jacobi_identity_and_greedy_pairing(seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((9, 9))
    M = B + B.T
    prev = M.copy()
    for t in range(1, 6):
        layers, At = A.truncated_jacobi(M, t)
        rots = layers[-1]
        nodes = [v for p, q, _, _ in rots for v in (p, q)]
        assert len(nodes) == len(set(nodes))
        pairs = A.choose_pairs(prev)
        assert [(p, q) for p, q, _, _ in rots] == pairs
        upper = np.triu(prev, 1)                      # the pairing reads the upper triangle
        assert abs(prev[pairs[0]]) == np.abs(upper).max()
        free = set(range(9)) - set(nodes)
        assert all(prev[p, q] == 0 for p in free for q in free if p < q)
        drop = 2 * sum(prev[p, q] ** 2 for p, q in pairs)
        assert abs((_off2(prev) - _off2(At)) - drop) <= 1e-12 * _off2(M)
        for p, q in pairs:
            assert At[p, q] == 0.0
        prev = At


@pytest.mark.parametrize("g", [W.path(8), W.near_symmetric_path(16, 0.05, seed=1),
                               W.grid(4, weights="sym_uniform", seed=2)], ids=lambda g: g.name)
def test_converges_to_exact_gft(g):
    L = _L(g)
    f = A.haar_approx_gft(L, [], 80)
    lam, U = gft.dense_gft(L)
    assert np.max(np.abs(f.lam - lam)) <= 1e-10
    assert metrics.delta(f.U, U) <= 1e-9
    assert np.max(np.abs(f.U.T @ f.U - np.eye(g.n))) <= 1e-13


def test_haar_plus_approx_converges_and_zero_layers_is_haar_only():
    g = W.grid6_bidiag(8)
    L = _L(g)
    f0 = A.haar_approx_gft(L, g.phis, 0)
    fact = gft.decompose(L, g.phis)
    B = np.eye(g.n)
    for st in fact.stages:                            # B_1 ... B_S of Eq. 20
        B = B @ gft.stage_matrix(g.n, st)
    assert np.max(np.abs(A.apply_units(f0.layers, np.eye(g.n)) - B)) <= 1e-15
    H = f0.U
    assert np.max(np.abs(H.T @ H - np.eye(g.n))) <= 1e-14
    Bt = H.T @ L @ H                                  # = the leaf Laplacians (Thm. 3), in output order
    for leaf in fact.leaves:
        idx = [int(np.nonzero(f0.perm == lab)[0][0]) for lab in leaf.labels]
        assert np.max(np.abs(Bt[np.ix_(idx, idx)] - leaf.L)) <= 1e-13
        rest = [j for j in range(g.n) if j not in idx]
        assert np.max(np.abs(Bt[np.ix_(idx, rest)])) <= 1e-13
    f = A.haar_approx_gft(L, g.phis, 80)
    lam, U = gft.dense_gft(L)
    assert metrics.delta(f.U, U) <= 1e-9
    assert np.max(np.abs(f.lam - lam)) <= 1e-10


@pytest.mark.parametrize("g", [W.grid6_bidiag(8), W.zgrid(8), W.skeleton25()], ids=lambda g: g.name)
def test_forward_matches_matrix(g):
    L = _L(g)
    f = A.haar_approx_gft(L, g.phis, 7)
    X = W.signals(5, g.n, 3).astype(np.float64)
    assert np.max(np.abs(A.forward(f, X) - X @ f.U)) <= 1e-13 * g.n
    assert np.max(np.abs(f.U.T @ f.U - np.eye(g.n))) <= 1e-13
    assert f.n_haar == len(g.phis)
    # the approximate eigenvalues are the Rayleigh quotients of U_hat's columns
    R = f.U.T @ L @ f.U
    assert np.max(np.abs(np.diag(R) - f.lam)) <= 1e-12 * np.abs(L).max()
    # one leaf: U_hat^T L U_hat is the matrix the Jacobi layers leave
    fp = A.haar_approx_gft(L, [], 7)
    _, Aj = A.truncated_jacobi(L, 7)
    Rp = fp.U.T @ L @ fp.U
    assert abs(_off2(Rp) - _off2(Aj)) <= 1e-12 * _off2(L)


@pytest.mark.parametrize("g", [W.grid6_bidiag(8), W.zgrid(8)], ids=lambda g: g.name)
def test_symmetry_speeds_up_the_approximation(g):
    """Sec. VI-B: for both 8x8 grids, Haar + approximate GFT has a smaller
    sign-normalised error than the approximate GFT at the same layer count
    (from 10 layers on; below that both are near the error of a random
    ordering)."""
    L = _L(g)
    _, U = gft.dense_gft(L)
    for J in (10, 20, 30):
        d_plain = metrics.delta(A.haar_approx_gft(L, [], J).U, U)
        d_haar = metrics.delta(A.haar_approx_gft(L, g.phis, J).U, U)
        assert d_haar < d_plain, (J, d_haar, d_plain)
