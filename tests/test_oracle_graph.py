"""Pins for oracle.graph: Eqs. 3-6, Definition 2, Eq. 20, Thm. 3, Thm. 4,
Eq. 21 and Lemma 4, checked against facts other than the code itself."""
import math

import numpy as np
import pytest

import gft_workloads as W
from oracle import graph


def _random_graph(n, seed, loops=True):
    rng = np.random.default_rng(seed)
    A = np.triu(rng.uniform(0.1, 1.0, (n, n)) * (rng.random((n, n)) < 0.6), 1)
    Wm = A + A.T
    s = rng.uniform(0, 1, n) * (rng.random(n) < 0.5) if loops else np.zeros(n)
    return Wm, s


@pytest.mark.parametrize("seed", range(5))
def test_laplacian_quadratic_form(seed):
    """Eq. 6: f^T L f = sum_{edges} w_ij (f_i - f_j)^2 + sum_k s_k f_k^2."""
    Wm, s = _random_graph(9, seed)
    L = graph.laplacian(Wm, s)
    f = np.random.default_rng(100 + seed).standard_normal(9)
    rhs = sum(Wm[i, j] * (f[i] - f[j]) ** 2 for i in range(9) for j in range(i + 1, 9))
    rhs += float(np.sum(s * f * f))
    assert abs(f @ L @ f - rhs) <= 1e-12 * max(1.0, abs(rhs))


def test_laplacian_round_trip_and_psd():
    """Eqs. 4-5 are inverse to each other; L is symmetric PSD (Sec. II-B)."""
    Wm, s = _random_graph(11, 7)
    L = graph.laplacian(Wm, s)
    W2, s2 = graph.weights_from_laplacian(L)
    assert np.allclose(W2, Wm, atol=1e-15) and np.allclose(s2, s, atol=1e-14)
    assert np.array_equal(L, L.T)
    assert np.linalg.eigvalsh(L).min() > -1e-12
    # no self-loops: the constant vector is in the null space
    L0 = graph.laplacian(Wm, np.zeros(11))
    assert np.max(np.abs(L0 @ np.ones(11))) < 1e-14


def test_involution_definition():
    assert graph.is_involution([3, 2, 1, 0])          # phi_a of Sec. IV-A (0-based)
    assert graph.is_involution([3, 1, 2, 0])          # phi_b of Sec. IV-A
    assert not graph.is_involution([1, 2, 0])         # 3-cycle
    assert not graph.is_involution([0, 0, 2])
    assert graph.p_phi([3, 1, 2, 0]) == 1
    assert graph.p_phi([3, 2, 1, 0]) == 2


def test_partition_and_b_phi_orthogonal_symmetric():
    """Eq. 20: B_phi is symmetric and orthogonal (like B_{n,p}, Eq. 7) and for
    phi = reversal with n = 2p it equals B_{n,p} up to the order of Y."""
    phi = np.array([5, 1, 3, 2, 4, 0])
    X, Y, Z = graph.partition(phi)
    assert X == [0, 2] and Y == [5, 3] and Z == [1, 4]
    B = graph.b_phi(phi)
    assert np.array_equal(B, B.T)
    assert np.allclose(B @ B.T, np.eye(6), atol=1e-15)
    # B_{8,4} of Eq. 7 written out from its printed block form
    p = 4
    J = np.fliplr(np.eye(p))
    B84 = np.block([[np.eye(p), J], [J, -np.eye(p)]]) / math.sqrt(2)
    assert np.allclose(graph.b_phi(W.reversal(8)), B84, atol=1e-15)


def test_b_phi_action_is_haar_units():
    """B_phi^T x gives (x_i + x_phi(i))/sqrt2 on X and (x_phi(i) - x_i)/sqrt2
    on Y (Sec. IV-B), i.e. one Haar unit per pair."""
    phi = W.reversal(8)
    x = np.arange(1.0, 9.0)
    y = graph.b_phi(phi).T @ x
    for i in range(4):
        assert math.isclose(y[i], (x[i] + x[7 - i]) / math.sqrt(2), rel_tol=1e-15)
        assert math.isclose(y[7 - i], (x[i] - x[7 - i]) / math.sqrt(2), rel_tol=1e-15)


@pytest.mark.parametrize("phi", [
    [7, 6, 5, 4, 3, 2, 1, 0],
    [7, 1, 5, 3, 4, 2, 6, 0],
    [0, 2, 1, 3, 5, 4, 6, 7],
    [1, 0, 3, 2, 5, 4, 7, 6],
])
def test_thm3_block_diagonal_and_thm4_weights(phi):
    """Thm. 3: L_phi = B_phi^T L B_phi has no X u Z / Y coupling for a
    phi-symmetric graph; Thm. 4's closed-form weights give the same blocks
    as the congruence (a second, independent route)."""
    phi = np.array(phi)
    g = W.planted_symmetric(8, phi, density=0.7, seed=int(phi.sum()) + 11)
    assert graph.is_phi_symmetric(g.W, g.s, phi)
    L = graph.laplacian(g.W, g.s)
    Lp, Lm, off = graph.block_diagonalize(L, phi)
    assert off <= 1e-14 * np.abs(L).max()
    Wp, sp, Wm_, sm = graph.thm4_subgraphs(g.W, g.s, phi)
    assert np.allclose(graph.laplacian(Wp, sp), Lp, atol=1e-13)
    assert np.allclose(graph.laplacian(Wm_, sm), Lm, atol=1e-13)
    # spectra: G+ and G- together carry the spectrum of G
    ev = np.sort(np.concatenate([np.linalg.eigvalsh(Lp), np.linalg.eigvalsh(Lm)]))
    assert np.allclose(ev, np.linalg.eigvalsh(L), atol=1e-12)


def test_edge_removal_cases():
    """Sec. IV-C cases: (1) an edge b between i and phi(i) becomes a self-loop
    2b in G-; (3) two symmetric edges d to a common Z node become one edge
    sqrt2 d in G+, self-loops -(sqrt2-1)d on the X node and (2-sqrt2)d on the
    Z node in G+, and a self-loop d on the Y node in G-."""
    b, d = 0.7, 0.3
    # nodes: 0 (X), 1 (Z), 2 (Y); phi = (2, 1, 0)
    Wm = np.zeros((3, 3))
    Wm[0, 2] = Wm[2, 0] = b
    Wm[0, 1] = Wm[1, 0] = d
    Wm[2, 1] = Wm[1, 2] = d
    phi = np.array([2, 1, 0])
    Wp, sp, Wmm, sm = graph.thm4_subgraphs(Wm, np.zeros(3), phi)
    assert math.isclose(Wp[0, 1], math.sqrt(2) * d)
    assert math.isclose(sp[0], -(math.sqrt(2) - 1) * d)
    assert math.isclose(sp[1], (2 - math.sqrt(2)) * d)
    assert math.isclose(sm[0], 2 * b + d)


def test_even_odd_components():
    """Eq. 21: x = x_even + x_odd with x_even(phi(i)) = x_even(i) and
    x_odd(phi(i)) = -x_odd(i)."""
    phi = np.array([6, 1, 5, 3, 4, 2, 0])
    X, Y, Z = graph.partition(phi)
    x = np.random.default_rng(3).standard_normal(7)
    u = graph.b_phi(phi).T @ x
    xe, xo = graph.even_odd(u[X + Z], u[Y], phi)
    assert np.allclose(xe + xo, x, atol=1e-15)
    assert np.allclose(xe, xe[phi], atol=1e-15)
    assert np.allclose(xo, -xo[phi], atol=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_lemma4_two_sparse_condition_is_single_pair_symmetry(seed):
    """Lemma 4: an eigenvector (e_i - e_j)/sqrt2 exists iff w_vi = w_vj for all
    other v (Eq. 22); the paper notes this is phi-symmetry for the single
    transposition (i j).  Checked on graphs with and without that property."""
    rng = np.random.default_rng(seed)
    n = 6
    Wm, s = _random_graph(n, seed, loops=False)
    i, j = 1, 4
    if seed % 2 == 0:  # plant Eq. 22
        for v in range(n):
            if v not in (i, j):
                Wm[v, j] = Wm[j, v] = Wm[v, i]
    phi = np.arange(n)
    phi[i], phi[j] = j, i
    eq22 = all(Wm[v, i] == Wm[v, j] for v in range(n) if v not in (i, j))
    assert eq22 == graph.is_phi_symmetric(Wm, s, phi)
    L = graph.laplacian(Wm, s)
    u = np.zeros(n)
    u[i], u[j] = 1 / math.sqrt(2), -1 / math.sqrt(2)
    Lu = L @ u
    is_eig = np.allclose(Lu, (u @ Lu) * u, atol=1e-12)
    assert is_eig == eq22
    del rng


def test_connected_components():
    L = np.zeros((6, 6))
    for a, b in ((0, 3), (3, 5), (1, 2)):
        L[a, b] = L[b, a] = -1
    assert graph.connected_components(L) == [[0, 3, 5], [1, 2], [4]]
