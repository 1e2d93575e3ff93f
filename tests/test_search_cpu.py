"""Involution search (Sec. V-F) through the C ABI, on the host.

Pins: brute force over all T(n) involutions (n <= 8) with the oracle's
Definition-2 test gives the largest number of pairs any valid involution
has; the library's search must find that many, and its involution must pass
the oracle's test.  Trees (identical branches): the skeleton's left/right
limbs, path reversal, random trees with planted identical branches.  Stages
found by search must give a valid plan (analysis only here; the transform is
checked on the GPU)."""
import numpy as np
import pytest

import gft_workloads as W
from oracle import gft as ogft
from oracle import graph as ograph


@pytest.fixture(scope="module")
def gft():
    from paper_1907_07875_gb300.build import build
    build()
    import paper_1907_07875_gb300 as g
    return g


def _tol(L):
    return 1e-12 * max(1.0, float(np.abs(L).max()))


def _max_pairs_brute_tree_bound(L):
    # no valid involution of this tree moves node 1 (the hub) or the third
    # branch, so at most (12 - 4) / 2 = 4 pairs
    return (L.shape[0] - 4) // 2


def _max_pairs_brute(L):
    n = L.shape[0]
    best = 0
    for phi in W.all_involutions(n):
        if ograph.laplacian_is_phi_symmetric(L, phi, _tol(L)):
            best = max(best, int(np.sum(phi > np.arange(n))))
    return best


@pytest.mark.parametrize("seed", range(12))
def test_search_matches_brute_force(gft, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 9))
    planted = rng.permutation(n)
    phi0 = np.arange(n)
    for k in range(int(rng.integers(1, n // 2 + 1))):   # planted involution: a few disjoint swaps
        a, b = planted[2 * k], planted[2 * k + 1]
        phi0[a], phi0[b] = b, a
    g = W.planted_symmetric(n, phi0, density=float(rng.uniform(0.3, 0.9)), seed=seed)
    L = ograph.laplacian(g.W, g.s)
    phi, pairs = gft.find_involution(L)
    assert ograph.is_involution(phi)
    assert ograph.laplacian_is_phi_symmetric(L, phi, _tol(L))
    assert pairs == int(np.sum(phi > np.arange(n)))
    assert pairs == _max_pairs_brute(L)


def test_no_symmetry_gives_identity(gft):
    rng = np.random.default_rng(3)
    n = 7
    Wm = np.triu(rng.uniform(0.1, 1.0, (n, n)), 1)
    Wm = Wm + Wm.T                                  # all weights distinct: no nontrivial automorphism
    L = ograph.laplacian(Wm, np.zeros(n))
    phi, pairs = gft.find_involution(L)
    assert pairs == 0 and phi.tolist() == list(range(n))
    assert _max_pairs_brute(L) == 0


def test_trees_identical_branches(gft):
    g = W.skeleton25()
    L = ograph.laplacian(g.W, g.s)
    phi, pairs = gft.find_involution(L)
    assert pairs == 10 and phi.tolist() == g.phis[0].tolist()
    for n in (2, 7, 8, 33):
        g = W.path(n)
        phi, pairs = gft.find_involution(ograph.laplacian(g.W, g.s))
        assert pairs == n // 2 and phi.tolist() == W.reversal(n).tolist()
    # hub 1 with two identical leaves (0, 2), two identical weighted branches
    # (3-4-5, 6-7-8) and a third branch that differs inside (9-10-11): the
    # leaves and the identical branches are swapped, the third stays
    n = 12
    Wm = np.zeros((n, n))
    def edge(i, j, w):
        Wm[i, j] = Wm[j, i] = w
    edge(0, 1, 1.0); edge(1, 2, 1.0)
    for base in (3, 6):                                  # identical branches 3-4-5 and 6-7-8 on node 1
        edge(1, base, 0.5); edge(base, base + 1, 0.7); edge(base + 1, base + 2, 0.2)
    edge(1, 9, 0.5); edge(9, 10, 0.9); edge(10, 11, 0.2)  # same root weight, different inside
    L = ograph.laplacian(Wm, np.zeros(n))
    phi, pairs = gft.find_involution(L)
    assert ograph.laplacian_is_phi_symmetric(L, phi, _tol(L))
    assert pairs == 4 and int(phi[0]) == 2 and [int(phi[i]) for i in (3, 4, 5)] == [6, 7, 8]
    assert [int(phi[i]) for i in (9, 10, 11)] == [9, 10, 11]
    assert _max_pairs_brute_tree_bound(L) <= 4


@pytest.mark.parametrize("g,pairs_min", [(W.grid(4), 8), (W.cycle(12), 6), (W.grid(5, 4), 10),
                                         (W.bipartite(16, 0.3, seed=2), 8), (W.star(7), 3), (W.complete(6), 3)])
def test_general_graphs(gft, g, pairs_min):
    L = ograph.laplacian(g.W, g.s)
    phi, pairs = gft.find_involution(L)
    assert ograph.laplacian_is_phi_symmetric(L, phi, _tol(L))
    assert pairs >= pairs_min


def test_classes_restrict_pairs(gft):
    g = W.path(6)
    L = ograph.laplacian(g.W, g.s)
    phi, pairs = gft.find_involution(L, classes=[0, 1, 2, 3, 4, 5])   # every node its own class
    assert pairs == 0


@pytest.mark.parametrize("g", [W.skeleton25(), W.grid(8), W.cycle(16), W.path(12), W.grid(6, weights="sym_uniform",
                                                                                              seed=4)],
                         ids=lambda g: g.name)
def test_searched_stages_make_valid_plans(gft, g):
    L = ograph.laplacian(g.W, g.s)
    phis = gft.search_stages(L, max_stages=6)
    assert len(phis) >= 1
    plan = gft.Plan(L, phis, analyze_only=True)          # the library's own validation accepts them
    ref = ogft.decompose(L, phis)                        # and so does the oracle's step-by-step decomposition
    assert plan.leaves() == [b.labels for b in ref.leaves]
    dense = gft.Plan(L, [], analyze_only=True)
    assert plan.info["fast_mults"] < dense.info["fast_mults"]
    for off in ref.offblock:
        assert off <= 1e-12 * max(1.0, np.abs(L).max())


def test_search_rejects_bad_input(gft):
    with pytest.raises(gft.GftError) as e:
        gft.find_involution(np.array([[1.0, 2.0], [0.0, 1.0]]))
    assert e.value.status == "GFT_ERR_NOT_LAPLACIAN"


@pytest.mark.parametrize("seed", range(12))
def test_planted_symmetries_of_larger_graphs(gft, seed):
    """Random graphs of 12-40 nodes with a planted involution (random pairs,
    weights copied to image pairs): the search returns a valid symmetry
    (an involution under which L is symmetric, Definition 2) with at least
    as many pairs as the planted one."""
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(12, 41))
    perm = rng.permutation(n)
    k = int(rng.integers(1, n // 2 + 1))
    phi = np.arange(n)
    for a in range(k):
        i, j = perm[2 * a], perm[2 * a + 1]
        phi[i], phi[j] = j, i
    g = W.planted_symmetric(n, phi, density=float(rng.uniform(0.2, 0.6)), seed=seed)
    L = ograph.laplacian(g.W, g.s)
    found, pairs = gft.find_involution(L)
    assert ograph.is_involution(found)
    assert ograph.laplacian_is_phi_symmetric(L, [int(v) for v in found], 1e-12 * max(1.0, np.abs(L).max()))
    assert pairs == sum(1 for i in range(n) if found[i] > i)
    assert pairs >= k
