"""Pins for oracle.right_haar (Sec. III-A: right Haar units of bipartite
graphs, Lemma 1, Thms. 1-2) against closed-form spectra, the structure the
paper derives, independent library eigensolvers and hand-checked tiny cases:

* even cycles (2-regular bipartite): eigenvalues 2 - 2cos(2 pi k / n);
* hypercubes Q_d (d-regular bipartite): eigenvalues 2j with multiplicity
  binomial(d, j);
* complete bipartite K_{a,b}, normalised Laplacian: {0, 1 (n-2 times), 2};
* Lemma 1 / Thm. 2: spectrum mirrored about alpha (k, resp. 1), checked on
  numpy's eigvalsh, and the oracle's eigenvalues equal to eigvalsh's;
* Eq. 9: every pair of columns shares its first-part entries and has
  opposite second-part entries; unpaired columns vanish on the smaller part;
* U orthogonal and L U = U diag(lam); staged forward / inverse (Eq. 8)
  equal to the dense product.
A wrong eigenvalue assignment of the pair, a transposed coupling block, a
dropped 1/sqrt2 or missing null-space vectors each fail one of them.
"""
import math

import numpy as np
import pytest

import gft_workloads as W
from oracle import graph, right_haar as R


def _L(g, normalised):
    return graph.normalized_laplacian(g.W, g.s) if normalised else graph.laplacian(g.W, g.s)


def _check_basis(L, f, atol=1e-12):
    n = L.shape[0]
    U, lam = f.U, f.lam
    assert np.max(np.abs(U.T @ U - np.eye(n))) <= 1e-13
    assert np.max(np.abs(L @ U - U * lam)) <= atol * max(1.0, np.abs(L).max())
    assert np.all(np.diff(lam) >= -1e-12)


@pytest.mark.parametrize("n", [4, 6, 12, 20])
def test_even_cycle_closed_form(n):
    g = W.cycle(n)
    L = _L(g, False)
    f = R.right_haar_gft(L)                       # parts found by two-colouring
    assert f.alpha == 2.0 and f.p == n // 2
    lam = np.sort(2 - 2 * np.cos(2 * math.pi * np.arange(n) / n))
    assert np.max(np.abs(f.lam - lam)) <= 1e-13
    _check_basis(L, f)


def test_printed_c4_columns_by_right_haar():
    """Sec. III: the 4-cycle is bipartite (parts {1, 3} and {2, 4} of the
    printed labels); the right Haar unit of its first column pair gives the
    printed lam = 0 column (1, 1, 1, 1)/2 as the sum vector and the printed
    lam = 4 column (1, -1, 1, -1)/2 as the difference vector, signs included
    (the sign rule fixes the sum vector, the difference follows it)."""
    import os
    from _helpers import read_golden_matrix
    meta, M = read_golden_matrix(os.path.join(os.path.dirname(__file__), "golden", "u_c4.txt"))
    Uc4 = M * meta["scale"][0]
    g = W.cycle(4)
    f = R.right_haar_gft(_L(g, False))
    assert np.allclose(f.lam, meta["eigenvalues"], atol=1e-13)
    for c in (0, 3):
        assert np.allclose(f.U[:, c], Uc4[:, c], atol=1e-13)


@pytest.mark.parametrize("n", [6, 12, 20])
def test_even_cycle_extreme_columns_signed(n):
    """Even cycle: the simple eigenvalues 0 and 4 have the closed-form
    vectors 1/sqrt(n) and (-1)^i / sqrt(n); both start positive, and the
    second is Lemma 1's image (u1, -u2) of the first."""
    g = W.cycle(n)
    f = R.right_haar_gft(_L(g, False))
    i = np.arange(n)
    assert np.allclose(f.U[:, 0], np.full(n, 1 / math.sqrt(n)), atol=1e-13)
    assert np.allclose(f.U[:, n - 1], (-1.0) ** i / math.sqrt(n), atol=1e-13)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_hypercube_closed_form(d):
    g = W.hypercube(d)
    L = _L(g, False)
    f = R.right_haar_gft(L, g.meta["side"])
    lam = np.concatenate([np.full(math.comb(d, j), 2.0 * j) for j in range(d + 1)])
    assert np.max(np.abs(f.lam - lam)) <= 1e-12
    _check_basis(L, f)


@pytest.mark.parametrize("a,b", [(3, 3), (5, 2), (1, 4)])
def test_complete_bipartite_normalised(a, b):
    n = a + b
    Wm = np.zeros((n, n))
    Wm[:a, a:] = 1.0
    Wm[a:, :a] = 1.0
    L = graph.normalized_laplacian(Wm, np.zeros(n))
    f = R.right_haar_gft(L)
    lam = np.array([0.0] + [1.0] * (n - 2) + [2.0])
    assert np.max(np.abs(f.lam - lam)) <= 1e-13
    assert len(f.big) == max(a, b) and f.p == min(a, b)
    _check_basis(L, f)


def test_normalised_laplacian_by_hand():
    """Path 0 - 1 - 2 with weights 1 and 3: degrees 1, 4, 3;
    entries -w_ij / sqrt(d_i d_j) off the diagonal, 1 on it."""
    Wm = np.array([[0, 1, 0], [1, 0, 3], [0, 3, 0]], dtype=float)
    N = graph.normalized_laplacian(Wm, np.zeros(3))
    ref = np.array([[1, -1 / 2, 0], [-1 / 2, 1, -3 / math.sqrt(12)], [0, -3 / math.sqrt(12), 1]])
    assert np.max(np.abs(N - ref)) <= 1e-15
    lam = np.linalg.eigvalsh(N)
    assert np.max(np.abs(lam - [0, 1, 2])) <= 1e-14     # bipartite: mirrored about 1


@pytest.mark.parametrize("case", range(len(W.right_haar_graphs())))
def test_mirror_and_library_spectrum(case):
    """Lemma 1 (alpha = k) and Thm. 2 (alpha = 1): lam_i + lam_{n-1-i} = 2 alpha;
    the oracle's eigenvalues equal numpy's eigvalsh of L."""
    g, normalised = W.right_haar_graphs()[case]
    L = _L(g, normalised)
    f = R.right_haar_gft(L, g.meta.get("side"))
    ev = np.linalg.eigvalsh(L)
    assert np.max(np.abs(ev + ev[::-1] - 2 * f.alpha)) <= 1e-12 * max(1.0, f.alpha)
    assert np.max(np.abs(f.lam - ev)) <= 1e-12 * max(1.0, f.alpha)
    if not normalised and "degree" in g.meta:
        assert abs(f.alpha - g.meta["degree"]) <= 1e-12
    if normalised:
        assert f.alpha == pytest.approx(1.0, abs=1e-15)
    _check_basis(L, f)


@pytest.mark.parametrize("case", range(len(W.right_haar_graphs())))
def test_pair_structure_eq9(case):
    g, normalised = W.right_haar_graphs()[case]
    L = _L(g, normalised)
    f = R.right_haar_gft(L, g.meta.get("side"))
    m1, p = len(f.big), f.p
    big, small = np.array(f.big), np.array(f.small)
    for c in range(p):
        us, ud = f.U[:, f.pos[c]], f.U[:, f.pos[m1 + c]]
        assert np.max(np.abs(us[big] - ud[big])) <= 1e-15
        assert np.max(np.abs(us[small] + ud[small])) <= 1e-15
        assert np.linalg.norm(us[big]) == pytest.approx(1 / math.sqrt(2), abs=1e-13)
        assert f.lam[f.pos[c]] == pytest.approx(f.alpha - f.sigma[c], abs=1e-13)
        assert f.lam[f.pos[m1 + c]] == pytest.approx(f.alpha + f.sigma[c], abs=1e-13)
    for c in range(p, m1):
        u = f.U[:, f.pos[c]]
        assert np.max(np.abs(u[small])) == 0.0
        assert f.lam[f.pos[c]] == f.alpha
    # the coupling block really is what the sub-transforms diagonalise
    C = -L[np.ix_(big, small)]
    S = f.E.T @ C @ f.F
    D = np.zeros_like(S)
    D[np.arange(p), np.arange(p)] = f.sigma
    assert np.max(np.abs(S - D)) <= 1e-12 * max(1.0, f.alpha)


@pytest.mark.parametrize("case", range(len(W.right_haar_graphs())))
def test_staged_transform_matches_dense(case):
    g, normalised = W.right_haar_graphs()[case]
    L = _L(g, normalised)
    f = R.right_haar_gft(L, g.meta.get("side"))
    X = W.signals(7, g.n, 400 + case).astype(np.float64)
    Y = R.forward_staged(f, X)
    assert np.max(np.abs(Y - X @ f.U)) <= 1e-13 * np.abs(X).max() * g.n
    assert np.max(np.abs(R.inverse_staged(f, Y) - X)) <= 1e-13 * np.abs(X).max() * g.n


def test_op_counts():
    f = R.right_haar_gft(_L(W.random_bipartite(7, 4, 0.4, seed=2103), True))
    assert R.op_counts(f) == (7 * 6 + 4 * 3 + 8, 49 + 16)


def test_structure_rejections():
    with pytest.raises(ValueError, match="not bipartite"):
        R.right_haar_gft(_L(W.cycle(7), False))
    with pytest.raises(ValueError, match="diagonal"):            # path: end degrees 1, inner 2
        R.right_haar_gft(_L(W.path(6), False))
    g = W.krbg(4, 2, seed=1, shuffle=False)
    bad = g.meta["side"].copy()
    bad[0], bad[4] = bad[4], bad[0]                              # a wrong colouring
    with pytest.raises(ValueError, match="one part"):
        R.right_haar_gft(_L(g, False), bad)


def test_bipartition_by_hand():
    """Two components: 0-2-4 chain and 1-3 edge; colours start at each
    component's smallest node."""
    L = np.zeros((5, 5))
    for i, j in [(0, 2), (2, 4), (1, 3)]:
        L[i, j] = L[j, i] = -1.0
    assert graph.bipartition(L).tolist() == [0, 0, 1, 1, 0]
    L[0, 4] = L[4, 0] = -1.0                                     # odd cycle 0-2-4
    assert graph.bipartition(L) is None
