"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only *draws inputs*: edge weights, self-loop weights, node-pairing
involutions and graph signals.  It holds none of the transform's arithmetic
(no Laplacian, no decomposition, no eigenvectors), so that both sides of every
parity test start from the same numbers without sharing any computation.

Graph families follow the paper's examples (Sec. V): symmetric line graphs,
cycle graphs (steerable DFT), 4-connected grids with the involutions of
Table II, skeletal graphs (Sec. V-F), bipartite graphs (Sec. III-A), graphs
with 2-sparse eigenvectors (Sec. V-A), plus nearly symmetric graphs whose
weights break the symmetry.  Labels are 0-based; grid node (k, l) has label
k*N2 + l (row-major, image coordinates).

Signals: NumPy PCG64 ``default_rng(seed)``, FP64 N(0,1) (or U[0,1], the
paper's Sec. VI distribution) rounded to FP32.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Graph", "signals", "path", "path_recursive", "nested_reversals", "cycle", "cycle_recursive", "grid", "skeleton25", "bipartite",
    "star", "complete", "near_symmetric_path", "near_symmetric_grid",
    "planted_symmetric", "reversal", "cycle_second_reflection", "grid_lr",
    "grid_ud", "grid_diag", "grid_antidiag", "grid_centro", "involution_count",
    "all_involutions", "grid6_bidiag", "zgrid", "runtime_table_graphs", "config1", "config2", "config3", "config4", "config5", "config5_specs",
    "make_graph", "krbg", "random_bipartite", "hypercube", "right_haar_graphs",
]


@dataclass
class Graph:
    """A weighted undirected graph: symmetric weights W (zero diagonal),
    self-loop weights s, and the stage involutions to decompose it with."""
    name: str
    W: np.ndarray                      # (n, n) float64, symmetric, zero diagonal
    s: np.ndarray                      # (n,) float64 self-loop weights
    phis: List[np.ndarray] = field(default_factory=list)  # per stage, int32 (n,)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.W.shape[0])


# --------------------------------------------------------------------------
# signals
# --------------------------------------------------------------------------
def signals(batch: int, n: int, seed: int, dist: str = "normal") -> np.ndarray:
    """(batch, n) float32 signals, one per row; FP64 draws rounded to FP32."""
    rng = np.random.default_rng(seed)
    if dist == "normal":
        x = rng.standard_normal((batch, n))
    elif dist == "uniform":
        x = rng.random((batch, n))
    else:
        raise ValueError(f"unknown distribution {dist!r}")
    return x.astype(np.float32)


# --------------------------------------------------------------------------
# involutions (node pairings)
# --------------------------------------------------------------------------
def reversal(n: int) -> np.ndarray:
    """i <-> n-1-i: the symmetry of a symmetric line graph and of a cycle."""
    return (n - 1 - np.arange(n)).astype(np.int32)


def cycle_second_reflection(n: int) -> np.ndarray:
    """i <-> (n/2 - 1 - i) mod n: the cycle's second reflection axis, which
    maps each half produced by :func:`reversal` onto itself (n divisible by 4)."""
    if n % 4:
        raise ValueError("second cycle reflection needs n divisible by 4")
    i = np.arange(n)
    return ((n // 2 - 1 - i) % n).astype(np.int32)


def _grid_map(N1: int, N2: int, f) -> np.ndarray:
    phi = np.empty(N1 * N2, dtype=np.int32)
    for k in range(N1):
        for l in range(N2):
            kk, ll = f(k, l)
            phi[k * N2 + l] = kk * N2 + ll
    return phi


def grid_lr(N1: int, N2: Optional[int] = None) -> np.ndarray:
    N2 = N1 if N2 is None else N2
    return _grid_map(N1, N2, lambda k, l: (k, N2 - 1 - l))


def grid_ud(N1: int, N2: Optional[int] = None) -> np.ndarray:
    N2 = N1 if N2 is None else N2
    return _grid_map(N1, N2, lambda k, l: (N1 - 1 - k, l))


def grid_diag(N: int) -> np.ndarray:
    return _grid_map(N, N, lambda k, l: (l, k))


def grid_antidiag(N: int) -> np.ndarray:
    return _grid_map(N, N, lambda k, l: (N - 1 - l, N - 1 - k))


def grid_centro(N1: int, N2: Optional[int] = None) -> np.ndarray:
    """Point symmetry about the grid centre, (k, l) -> (N1-1-k, N2-1-l)."""
    N2 = N1 if N2 is None else N2
    return _grid_map(N1, N2, lambda k, l: (N1 - 1 - k, N2 - 1 - l))


def involution_count(n: int) -> int:
    """Number of involutions on n elements, by the recurrence
    T(n) = T(n-1) + (n-1) T(n-2) (a counting fact, used to size brute force)."""
    a, b = 1, 1  # T(0), T(1)
    if n == 0:
        return 1
    for m in range(2, n + 1):
        a, b = b, b + (m - 1) * a
    return b


def all_involutions(n: int):
    """Yield every involution of {0..n-1} as an int32 array."""
    phi = list(range(n))

    def rec(i):
        while i < n and phi[i] != i:
            i += 1
        if i >= n:
            yield np.array(phi, dtype=np.int32)
            return
        # i fixed
        yield from rec(i + 1)
        for j in range(i + 1, n):
            if phi[j] == j:
                phi[i], phi[j] = j, i
                yield from rec(i + 1)
                phi[i], phi[j] = i, j

    # recursion above only moves forward from i, so a fixed i is final
    yield from rec(0)


# --------------------------------------------------------------------------
# graph families
# --------------------------------------------------------------------------
def _empty(n):
    return np.zeros((n, n)), np.zeros(n)


def _add_edge(W, i, j, w):
    W[i, j] = w
    W[j, i] = w


def path(n: int, weights: Optional[Sequence[float]] = None, s=None) -> Graph:
    W, s0 = _empty(n)
    w = np.ones(n - 1) if weights is None else np.asarray(weights, dtype=np.float64)
    for i in range(n - 1):
        _add_edge(W, i, i + 1, w[i])
    s = s0 if s is None else np.asarray(s, dtype=np.float64)
    return Graph(f"path{n}", W, s, [reversal(n)])


def nested_reversals(n: int, first: int, min_len: int = 4) -> List[np.ndarray]:
    """Involutions (on labels 0..n-1) reversing the prefix 0..L-1 for
    L = first, first/2, first/4, ... while L is even and at least min_len,
    identity elsewhere.  After a reversal stage of a uniform path, the
    sum block G+ is again a uniform path on the prefix of the smaller labels
    (Sec. V-B, recursion at the end of Sec. IV-C), so every prefix reversal
    is a symmetry of the current G+ block and leaves the other blocks alone."""
    out, L = [], first
    while L >= min_len and L % 2 == 0:
        phi = np.arange(n, dtype=np.int32)
        phi[:L] = L - 1 - np.arange(L)
        out.append(phi)
        L //= 2
    return out


def path_recursive(n: int, min_len: int = 4) -> Graph:
    """Uniform path with the reversal applied recursively to every sum
    block: stage s reverses labels 0..n/2^(s-1)-1 (while that length is even
    and at least min_len).  Leaves: the difference blocks of n/2, n/4, ...
    nodes (DCT-IV type) and a final small uniform path."""
    g = path(n)
    g.name = f"path{n}_rec"
    g.phis = nested_reversals(n, n, min_len) if n % 2 == 0 else [reversal(n)]
    return g


def cycle_recursive(n: int, min_len: int = 4) -> Graph:
    """Cycle (n divisible by 4) with its two reflections and then the
    recursive reversals of the G++ block, a uniform path on labels
    0..n/4-1 (DCT-II, Sec. V-C)."""
    g = cycle(n)
    g.name = f"cycle{n}_rec"
    if n % 4 == 0:
        g.phis = list(g.phis) + nested_reversals(n, n // 4, min_len)
    return g


def cycle(n: int) -> Graph:
    W, s = _empty(n)
    for i in range(n):
        _add_edge(W, i, (i + 1) % n, 1.0)
    phis = [reversal(n)]
    if n % 4 == 0:
        phis.append(cycle_second_reflection(n))
    return Graph(f"cycle{n}", W, s, phis)


def _grid_edges(N1, N2):
    E = []
    for k in range(N1):
        for l in range(N2):
            i = k * N2 + l
            if l + 1 < N2:
                E.append((i, i + 1))
            if k + 1 < N1:
                E.append((i, i + N2))
    return E


def grid(N1: int, N2: Optional[int] = None, weights: str = "unit",
         seed: Optional[int] = None) -> Graph:
    """4-connected N1 x N2 grid.  weights='unit', or 'sym_uniform': one
    U[0.1, 1] weight drawn per edge orbit under {id, LR, UD, LR.UD} so the
    grid keeps both axis symmetries."""
    N2 = N1 if N2 is None else N2
    n = N1 * N2
    W, s = _empty(n)
    E = _grid_edges(N1, N2)
    if weights == "unit":
        for i, j in E:
            _add_edge(W, i, j, 1.0)
    elif weights == "sym_uniform":
        rng = np.random.default_rng(seed)
        lr, ud = grid_lr(N1, N2), grid_ud(N1, N2)
        group = [lambda v: v, lambda v: lr[v], lambda v: ud[v], lambda v: lr[ud[v]]]
        done = set()
        for i, j in E:
            key = (min(i, j), max(i, j))
            if key in done:
                continue
            w = rng.uniform(0.1, 1.0)
            for g in group:
                a, b = int(g(i)), int(g(j))
                _add_edge(W, a, b, w)
                done.add((min(a, b), max(a, b)))
    else:
        raise ValueError(weights)
    return Graph(f"grid{N1}x{N2}_{weights}", W, s, [grid_lr(N1, N2), grid_ud(N1, N2)],
                 {"N1": N1, "N2": N2})


def grid6_bidiag(N: int, a: float = 0.5) -> Graph:
    """Bi-diagonally symmetric 6-connected N x N grid (Sec. V-D, Fig. 7; the
    runtime experiment uses a = 0.5): the 4-connected grid with unit weights
    plus the (1, 1) diagonals (k, l) - (k+1, l+1) with weight a.  Symmetric
    under the diagonal and the anti-diagonal reflections."""
    n = N * N
    W, s = _empty(n)
    for i, j in _grid_edges(N, N):
        _add_edge(W, i, j, 1.0)
    for k in range(N - 1):
        for l in range(N - 1):
            _add_edge(W, k * N + l, (k + 1) * N + l + 1, a)
    return Graph(f"grid6bidiag{N}x{N}_a{a}", W, s, [grid_diag(N), grid_antidiag(N)], {"N1": N, "N2": N})


def zgrid(N: int, w: float = 2.0) -> Graph:
    """z-shaped N x N grid (Sec. V-D, Fig. 8; the runtime experiment uses
    w = 2): horizontal edges with weight 1 and anti-diagonal edges
    (k, l) - (k+1, l-1) with weight w.  Symmetric under the point reflection
    about the grid centre."""
    n = N * N
    W, s = _empty(n)
    for k in range(N):
        for l in range(N):
            if l + 1 < N:
                _add_edge(W, k * N + l, k * N + l + 1, 1.0)
            if k + 1 < N and l >= 1:
                _add_edge(W, k * N + l, (k + 1) * N + l - 1, w)
    return Graph(f"zgrid{N}x{N}_w{w}", W, s, [grid_centro(N)], {"N1": N, "N2": N})


def skeleton25() -> Graph:
    """25-joint skeleton: spine chain 0-4; left arm 5-9 and right arm 10-14
    attached at joint 3; left leg 15-19 and right leg 20-24 attached at
    joint 0; unit weights; the left/right involution swaps the limbs."""
    n = 25
    W, s = _empty(n)
    for i in range(4):
        _add_edge(W, i, i + 1, 1.0)
    for base, root in ((5, 3), (10, 3), (15, 0), (20, 0)):
        _add_edge(W, root, base, 1.0)
        for k in range(4):
            _add_edge(W, base + k, base + k + 1, 1.0)
    phi = np.arange(n, dtype=np.int32)
    for k in range(5):
        phi[5 + k], phi[10 + k] = 10 + k, 5 + k
        phi[15 + k], phi[20 + k] = 20 + k, 15 + k
    return Graph("skeleton25", W, s, [phi])


def bipartite(n: int, p: float = 0.1, seed: Optional[int] = None) -> Graph:
    """Random bipartite graph with halves {0..h-1}, {h..n-1} (h = n/2):
    cross edges drawn with probability p and weights U[0.1, 1], made
    symmetric (B = B^T) so that i <-> i + h is a symmetry."""
    if n % 2:
        raise ValueError("bipartite graph needs even n")
    h = n // 2
    rng = np.random.default_rng(seed)
    mask = rng.random((h, h)) < p
    val = rng.uniform(0.1, 1.0, size=(h, h))
    B = np.where(mask, val, 0.0)
    B = np.triu(B) + np.triu(B, 1).T
    W, s = _empty(n)
    W[:h, h:] = B
    W[h:, :h] = B.T
    phi = ((np.arange(n) + h) % n).astype(np.int32)
    return Graph(f"bipartite{n}", W, s, [phi], {"halves": h})


def _relabel(W: np.ndarray, side: np.ndarray, rng) -> tuple:
    perm = rng.permutation(W.shape[0])          # new label of old node i is perm[i]
    W2 = np.zeros_like(W)
    W2[np.ix_(perm, perm)] = W
    side2 = np.empty_like(side)
    side2[perm] = side
    return W2, side2


def krbg(m: int, k: int, seed: Optional[int] = None, weighted: bool = True,
         shuffle: bool = True) -> Graph:
    """k-regular bipartite graph on 2m nodes (Lemma 1, Thm. 1): the cross
    block is a sum of k random permutation matrices, each with one weight
    (U[0.5, 1.5] if weighted, else 1), so every node has the same weighted
    degree (the sum of the k weights).  shuffle: random node labels, so the
    two parts are not contiguous.  meta['side'] marks the parts (0 / 1),
    meta['degree'] the common weighted degree."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 1.5, size=k) if weighted else np.ones(k)
    B = np.zeros((m, m))
    for t in range(k):
        B[np.arange(m), rng.permutation(m)] += w[t]
    n = 2 * m
    W, s = _empty(n)
    W[:m, m:] = B
    W[m:, :m] = B.T
    side = np.repeat(np.array([0, 1], dtype=np.int32), m)
    if shuffle:
        W, side = _relabel(W, side, rng)
    return Graph(f"krbg{n}_k{k}" + ("w" if weighted else ""), W, s, [], {"side": side, "degree": float(w.sum())})


def random_bipartite(n1: int, n2: int, p: float = 0.2, seed: Optional[int] = None,
                     shuffle: bool = True) -> Graph:
    """Random bipartite graph with parts of n1 and n2 nodes (Thm. 2: any
    bipartite graph, used with its normalised Laplacian): cross edges with
    probability p and weights U[0.1, 1]; a node left without an edge gets
    one to a random node of the other part, so every degree is positive."""
    rng = np.random.default_rng(seed)
    mask = rng.random((n1, n2)) < p
    for i in range(n1):
        if not mask[i].any():
            mask[i, rng.integers(n2)] = True
    for j in range(n2):
        if not mask[:, j].any():
            mask[rng.integers(n1), j] = True
    B = np.where(mask, rng.uniform(0.1, 1.0, size=(n1, n2)), 0.0)
    n = n1 + n2
    W, s = _empty(n)
    W[:n1, n1:] = B
    W[n1:, :n1] = B.T
    side = np.concatenate([np.zeros(n1, np.int32), np.ones(n2, np.int32)])
    if shuffle:
        W, side = _relabel(W, side, rng)
    return Graph(f"rbip{n1}x{n2}", W, s, [], {"side": side})


def hypercube(d: int) -> Graph:
    """d-dimensional hypercube (2^d nodes, i ~ i xor 2^b): d-regular and
    bipartite by the parity of the number of set bits."""
    n = 1 << d
    W, s = _empty(n)
    for i in range(n):
        for b in range(d):
            j = i ^ (1 << b)
            if i < j:
                _add_edge(W, i, j, 1.0)
    side = np.array([bin(i).count("1") & 1 for i in range(n)], dtype=np.int32)
    return Graph(f"hypercube{d}", W, s, [], {"side": side, "degree": float(d)})


def right_haar_graphs():
    """Bipartite cases of the right Haar stage: (graph, normalised) pairs.
    normalised = False: the combinatorial Laplacian of a k-regular bipartite
    graph (Thm. 1); True: the normalised Laplacian D^-1/2 L D^-1/2 of any
    bipartite graph (Thm. 2)."""
    return [
        (cycle(12), False), (krbg(8, 3, seed=2101), False), (krbg(20, 4, seed=2102, weighted=False), False),
        (hypercube(4), False), (random_bipartite(7, 4, 0.4, seed=2103), True),
        (random_bipartite(30, 18, 0.15, seed=2104), True), (krbg(32, 5, seed=2105), False),
        (random_bipartite(40, 40, 0.1, seed=2106), True), (krbg(64, 6, seed=2302), False),
    ]


def star(n: int) -> Graph:
    """Star with centre 0 and n-1 unit-weight leaves."""
    W, s = _empty(n)
    for i in range(1, n):
        _add_edge(W, 0, i, 1.0)
    return Graph(f"star{n}", W, s, [])


def complete(n: int) -> Graph:
    W = np.ones((n, n)) - np.eye(n)
    return Graph(f"complete{n}", W, np.zeros(n), [])


def near_symmetric_path(n: int, eps: float, seed: Optional[int] = None) -> Graph:
    """Path with weights 1 + eps*g, g ~ N(0,1): no exact symmetry."""
    rng = np.random.default_rng(seed)
    w = 1.0 + eps * rng.standard_normal(n - 1)
    g = path(n, w)
    g.name = f"nspath{n}_eps{eps}"
    g.phis = []
    return g


def near_symmetric_grid(N: int, eps: float, seed: Optional[int] = None) -> Graph:
    rng = np.random.default_rng(seed)
    n = N * N
    W, s = _empty(n)
    for i, j in _grid_edges(N, N):
        _add_edge(W, i, j, 1.0 + eps * rng.standard_normal())
    return Graph(f"nsgrid{N}x{N}_eps{eps}", W, s, [], {"N1": N, "N2": N})


def planted_symmetric(n: int, phi: np.ndarray, density: float = 0.5,
                      seed: Optional[int] = None, self_loops: bool = True) -> Graph:
    """Random graph made phi-symmetric by copying each weight to its image
    pair (and each self-loop to its image node); weights U[0.1, 1]."""
    rng = np.random.default_rng(seed)
    W, s = _empty(n)
    for i in range(n):
        for j in range(i + 1, n):
            a, b = sorted((int(phi[i]), int(phi[j])))
            if (a, b) < (i, j):
                continue  # already assigned from its image
            if rng.random() < density:
                w = rng.uniform(0.1, 1.0)
                _add_edge(W, i, j, w)
                _add_edge(W, a, b, w)
    if self_loops:
        for i in range(n):
            j = int(phi[i])
            if j < i:
                continue
            if rng.random() < 0.3:
                v = rng.uniform(0.1, 1.0)
                s[i] = v
                s[j] = v
    return Graph(f"planted{n}", W, s, [np.asarray(phi, dtype=np.int32)])


# --------------------------------------------------------------------------
# workload recipes (graph seeds 2000 + config index, signal seeds 1000 + index)
# --------------------------------------------------------------------------
def runtime_table_graphs():
    """The graphs of the paper's runtime table (Sec. VI-A) that the text fixes:
    cycles 12 and 80, bi-diagonally symmetric 6-connected grids 4x4 and 8x8
    (a = 0.5), z-shaped grids 4x4 and 8x8 (w = 2), the 25-joint skeleton.
    (The 15-joint skeleton is drawn only in a figure.)  Each item is
    (graph, split_components, (matrix adds, matrix mults, fast adds, fast
    mults, runtime reduction) as printed in the table)."""
    return [
        (cycle(12), False, (132, 144, 44, 30, 0.527)),
        (cycle(80), False, (6320, 6400, 1224, 1078, 0.797)),
        (grid6_bidiag(4), False, (240, 256, 80, 80, 0.537)),
        (grid6_bidiag(8), False, (4032, 4096, 1104, 1072, 0.685)),
        (zgrid(4), False, (240, 256, 128, 112, 0.415)),
        (zgrid(8), False, (4032, 4096, 2048, 2048, 0.450)),
        (skeleton25(), True, (600, 625, 272, 282, 0.475)),
    ]


def config1(batch: int = 4096):
    """Uniform path graph N=8 with the reflection involution; N(0,1) signals."""
    g = path(8)
    return [(g, batch, 1001)]


def config2(batch: int = 1 << 20):
    """25-node skeleton, left/right involution; 2^20 signals."""
    return [(skeleton25(), batch, 1002)]


def config3(coeffs_per_kind: int = 1 << 23):
    """Grids 8x8, 16x16, 32x32 (unit and axis-symmetrised U[0.1,1] weights)
    and cycles 64, 256; an equal number of coefficients per graph kind."""
    kinds = []
    for idx, N in enumerate((8, 16, 32)):
        kinds.append(grid(N))
        kinds.append(grid(N, weights="sym_uniform", seed=2003 * 100 + idx))
    kinds.append(cycle(64))
    kinds.append(cycle(256))
    out = []
    for k, g in enumerate(kinds):
        out.append((g, coeffs_per_kind // g.n, 1003 * 100 + k))
    return out


def config4():
    """Nearly symmetric paths N=16/32 and 8x8 grids, eps in {0.01,0.05,0.1}."""
    out = []
    k = 0
    for eps in (0.01, 0.05, 0.1):
        for maker, arg in ((near_symmetric_path, 16), (near_symmetric_path, 32),
                           (near_symmetric_grid, 8)):
            out.append(maker(arg, eps, seed=2004 * 100 + k))
            k += 1
    return out


def config5_specs(n_graphs: int = 10000, total_coeffs: int = 1 << 28, seed: int = 2005):
    """Size sweep recipe without building the graphs: graphs of sizes 8..1024
    (log-uniform per family) from the path, cycle, grid, skeleton and
    bipartite families.  Returns (family, n, graph_seed, batch, signal_seed)
    tuples with ceil(total / (n_graphs * n)) signals each; graph_seed is
    None for the deterministic families.  ``make_graph`` builds one."""
    rng = np.random.default_rng(seed)
    fams = ("path", "cycle", "grid", "skeleton", "bipartite")
    out = []
    for gi in range(n_graphs):
        fam = fams[gi % len(fams)]
        n = int(round(np.exp(rng.uniform(np.log(8), np.log(1024)))))
        gseed = None
        if fam == "path":
            n = max(n, 2)
        elif fam == "cycle":
            n = max(4, n - n % 4)
        elif fam == "grid":
            N = max(2, int(round(np.sqrt(n))))
            n = N * N
        elif fam == "skeleton":
            n = 25
        else:
            n = max(8, n - n % 2)
            gseed = int(rng.integers(1 << 31))
        b = -(-total_coeffs // (n_graphs * n))
        out.append((fam, n, gseed, b, 1005 * 100000 + gi))
    return out


def make_graph(family: str, n: int, graph_seed: Optional[int] = None) -> Graph:
    if family == "path":
        return path(n)
    if family == "cycle":
        return cycle(n)
    if family == "grid":
        N = int(round(np.sqrt(n)))
        return grid(N)
    if family == "skeleton":
        return skeleton25()
    if family == "bipartite":
        return bipartite(n, seed=graph_seed)
    raise ValueError(family)


def config5(n_graphs: int = 10000, total_coeffs: int = 1 << 28, seed: int = 2005):
    """The size sweep as (graph, batch, signal_seed) triples (builds every
    graph: use ``config5_specs`` for the full 10^4-graph recipe)."""
    return [(make_graph(f, n, gs), b, ss) for f, n, gs, b, ss in config5_specs(n_graphs, total_coeffs, seed)]
