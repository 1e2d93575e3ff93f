"""The seeded workload recipes the bench and the GPU tests share: the size
sweep's shape (graph count, size range, coefficients, families) and the
symmetry of every family's graphs under the involutions it hands to the
plans (Definition 2: W[phi, phi] = W, S[phi] = S), checked without a GPU."""
import numpy as np
import pytest

import gft_workloads as W


def test_size_sweep_recipe_shape():
    specs = W.config5_specs()
    assert len(specs) == 10000
    fams = {f for f, n, gs, b, ss in specs}
    assert fams == {"path", "cycle", "grid", "skeleton", "bipartite"}
    ns = np.array([n for f, n, gs, b, ss in specs])
    assert ns.min() >= 4 and ns.max() <= 1024
    total = sum(b * n for f, n, gs, b, ss in specs)
    assert total >= 1 << 28 and total < (1 << 28) * 1.01
    for f, n, gs, b, ss in specs:
        assert b == -(-(1 << 28) // (10000 * n))            # the same share of coefficients per graph
        assert (gs is None) == (f != "bipartite")           # only the random family has a graph seed
        if f == "cycle":
            assert n % 4 == 0
        if f == "skeleton":
            assert n == 25
    assert specs == W.config5_specs()                        # seeded: the same recipe every call


@pytest.mark.parametrize("fam,n,seed", [("path", 37, None), ("cycle", 40, None), ("grid", 49, None),
                                        ("skeleton", 25, None), ("bipartite", 30, 12345)])
def test_family_graphs_are_symmetric_under_their_involutions(fam, n, seed):
    g = W.make_graph(fam, n, seed)
    assert g.W.shape == (g.n, g.n) and np.allclose(g.W, g.W.T)
    for phi in g.phis:
        phi = np.asarray(phi)
        assert np.array_equal(phi[phi], np.arange(g.n))     # an involution
        assert np.allclose(g.W[np.ix_(phi, phi)], g.W)
        assert np.allclose(np.asarray(g.s)[phi], g.s)
