"""Oracle jobs run in a process pool (spawn) by the GPU batch tests: the FP64
oracle's fast GFT of one graph, rebuilt in the worker from its seeded recipe
so that only small tuples cross the process boundary.  Pure oracle calls; no
library code is imported here."""
from __future__ import annotations

import numpy as np

import gft_workloads as W
from oracle import gft as ogft
from oracle import graph as ograph


def config3_graph(k: int):
    return W.config3(coeffs_per_kind=1 << 10)[k][0]


def oracle_basis(recipe):
    """recipe = ("config3", k), ("grid", N), or ("config5" | "graph",
    family, n, graph_seed) with the size sweep's families.
    Returns (lam, U, pos) of the oracle's fast GFT (Sec. IV: U = B_1 ... B_S
    diag(U_k), ascending eigenvalues, the sign rule)."""
    if recipe[0] == "config3":
        g = config3_graph(recipe[1])
    elif recipe[0] == "grid":
        g = W.grid(recipe[1])
    else:
        _, fam, n, gs = recipe
        g = W.make_graph(fam, n, gs)
    f = ogft.fast_gft(ograph.laplacian(g.W, g.s), g.phis)
    return f.lam, f.U, np.asarray(f.pos)
