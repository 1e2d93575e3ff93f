"""Dense GFT and the paper's symmetry-based fast GFT, in float64 (test
infrastructure only).

Definition of the result (Sec. II-B): the GFT of a signal x on a graph with
Laplacian L = U diag(lam) U^T is U^T x, columns of U ordered by ascending
eigenvalue (graph frequency).  The fast GFT of Sec. IV reaches that result
exactly; this module computes it both ways:

* ``dense_gft``      -- Jacobi on L, sort, canonical signs.
* ``decompose``      -- the paper's stages, in the paper's order: check the
                        involution (Def. 1) and phi-symmetry (Def. 2), form
                        X/Y/Z (Sec. IV-B), L_phi = B_phi^T L B_phi (Thm. 3),
                        split into G+ / G- (Eq. 17 in permuted form), and
                        recurse on every block with the next involution
                        (end of Sec. IV-C).  Optionally split a leaf into its
                        connected components (Sec. V-E, Fig. 9 caption).
* ``fast_gft``       -- Jacobi on every leaf, U = B_1 ... B_S diag(U_k)
                        (Eq. 13 applied stage by stage), output order and signs.
* ``forward_dense`` / ``forward_staged`` / ``inverse_staged`` -- apply to a
                        batch of signals (rows), densely or stage by stage.

Readings where the paper is silent (each listed in the design notes):
X holds the member of each pair that comes first in the block's node order;
G+ lists X then Z, G- lists the partners of X in the same order; leaves are
in depth-first order with + before -; output coefficients are in ascending
eigenvalue order, eigenvalues within 1e-9 * max(1, |lam|_max) of their
neighbour form a cluster ordered by (leaf, index within leaf); the sign of
each basis vector makes its first significant entry (magnitude above 1e-8
of the vector's largest) positive -- the convention of the closed forms the
paper quotes (DCT-II, Sec. II-B and V-B; the printed 4-cycle basis, Sec. III),
whose first entries are all positive.

Pins (tests/test_oracle_gft.py): dense_gft -- DCT-II closed form for
uniform paths, real-DFT eigenspaces for cycles, separable 2-D DCT for grids,
the printed 4-cycle basis; decompose / fast_gft -- DCT-II and DCT-IV / DST-II
sub-blocks, DST-VII components of the skeleton, fast = dense eigenspaces on
every family, brute force over all involutions for n <= 8, rejections;
output_order -- the cluster rule; canonical_sign -- the closed forms with
their own signs, no normalisation (DCT-II bases of paths, the DCT-II /
DCT-IV leaves of the 8-node path, the DST-VII limbs of the skeleton, the
printed 4-cycle columns of simple eigenvalues); forward_staged / inverse_staged -- equal to the
dense product; op_counts -- the runtime table's printed counts where the
text fixes them (the 25-joint skeleton's printed counts: parity unpinned).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

from .graph import (block_diagonalize, connected_components, is_involution,
                    laplacian_is_phi_symmetric, partition)
from .jacobi import jacobi_eigh

SQRT2 = math.sqrt(2.0)
CLUSTER_TOL = 1e-9
SIGN_TOL = 1e-8          # entries below this fraction of max|u| are zeros for the sign rule
SYM_TOL = 1e-12          # phi-symmetry check, relative to max(1, max |L|)
ZERO_TOL = 1e-12         # structural zero for component splitting, same scale


def canonical_sign(u: np.ndarray) -> float:
    """+1 or -1 such that the first entry with |u_i| > 1e-8 max|u| becomes
    positive.  Entries that vanish in exact arithmetic come out of the
    eigensolver near 1e-15 max|u| and are skipped; the closed forms quoted by
    the paper (DCT-II c_k cos(pi k (i + 1/2) / N), the 4-cycle basis of
    Sec. III) all start with a positive entry and keep their signs."""
    a = np.abs(u)
    i = int(np.nonzero(a > SIGN_TOL * a.max())[0][0])
    return 1.0 if u[i] > 0 else -1.0


def dense_gft(L: np.ndarray):
    """(lam ascending, U) with L = U diag(lam) U^T, canonical column signs."""
    lam, V = jacobi_eigh(L)
    order = np.argsort(lam, kind="stable")
    lam, V = lam[order], V[:, order]
    for c in range(V.shape[1]):
        V[:, c] *= canonical_sign(V[:, c])
    return lam, V


@dataclass
class Block:
    labels: List[int]            # original node labels, in block order
    L: np.ndarray                # block Laplacian in that order
    tag: str = ""                # "+"/"-" path from the root


@dataclass
class Factorization:
    n: int
    stages: List[List[Tuple[int, int]]]    # per stage: (X label, partner label)
    leaves: List[Block]
    offblock: List[float] = field(default_factory=list)  # Thm. 3 residual per stage


def decompose(L: np.ndarray, phis: Sequence[Sequence[int]],
              split_components: bool = False) -> Factorization:
    L = np.asarray(L, dtype=np.float64)
    n = L.shape[0]
    scale = max(1.0, float(np.max(np.abs(L))))
    blocks = [Block(list(range(n)), L.copy(), "")]
    stages, offs = [], []
    for s_idx, phi in enumerate(phis):
        phi = [int(v) for v in phi]
        if len(phi) != n or not is_involution(np.array(phi)):
            raise ValueError(f"stage {s_idx}: not an involution")
        new_blocks, pairs, offmax = [], [], 0.0
        for b in blocks:
            pos = {lab: k for k, lab in enumerate(b.labels)}
            loc = []
            for lab in b.labels:
                if phi[lab] not in pos:
                    raise ValueError(f"stage {s_idx}: involution leaves block {b.tag!r}")
                loc.append(pos[phi[lab]])
            if all(loc[k] == k for k in range(len(loc))):
                new_blocks.append(b)
                continue
            if not laplacian_is_phi_symmetric(b.L, loc, SYM_TOL * scale):
                raise ValueError(f"stage {s_idx}: block {b.tag!r} is not phi-symmetric")
            X, Y, Z = partition(loc)
            Lp, Lm, off = block_diagonalize(b.L, loc)
            offmax = max(offmax, off)
            new_blocks.append(Block([b.labels[k] for k in X + Z], Lp, b.tag + "+"))
            new_blocks.append(Block([b.labels[k] for k in Y], Lm, b.tag + "-"))
            pairs += [(b.labels[x], b.labels[y]) for x, y in zip(X, Y)]
        blocks = new_blocks
        stages.append(pairs)
        offs.append(offmax)
    if split_components:
        split = []
        for b in blocks:
            comps = connected_components(b.L, ZERO_TOL * scale)
            if len(comps) == 1:
                split.append(b)
                continue
            for ci, comp in enumerate(comps):
                split.append(Block([b.labels[k] for k in comp], b.L[np.ix_(comp, comp)],
                                   f"{b.tag}.{ci}"))
        blocks = split
    return Factorization(n, stages, blocks, offs)


def stage_matrix(n: int, pairs: Sequence[Tuple[int, int]]) -> np.ndarray:
    """Eq. 20 applied to every block of one stage, in label coordinates:
    1/sqrt2 on (x,x), (x,y), (y,x), -1/sqrt2 on (y,y), 1 on unpaired labels."""
    B = np.eye(n)
    r = 1.0 / SQRT2
    for x, y in pairs:
        B[x, x] = r
        B[x, y] = r
        B[y, x] = r
        B[y, y] = -r
    return B


def output_order(entries: Sequence[Tuple[float, int, int]]) -> np.ndarray:
    """entries[i] = (eigenvalue, leaf, index within leaf) in leaf order.
    Returns pos with pos[i] = output coefficient index."""
    lam = np.array([e[0] for e in entries])
    m = len(entries)
    if m == 0:
        return np.zeros(0, dtype=np.int64)
    tol = CLUSTER_TOL * max(1.0, float(np.max(np.abs(lam))))
    idx = sorted(range(m), key=lambda i: lam[i])
    final = []
    start = 0
    for j in range(1, m + 1):
        if j == m or lam[idx[j]] - lam[idx[j - 1]] > tol:
            cluster = idx[start:j]
            cluster.sort(key=lambda i: (entries[i][1], entries[i][2]))
            final += cluster
            start = j
    pos = np.empty(m, dtype=np.int64)
    for p, i in enumerate(final):
        pos[i] = p
    return pos


@dataclass
class FastGFT:
    fact: Factorization
    leaf_lams: List[np.ndarray]
    leaf_vecs: List[np.ndarray]      # columns = leaf eigenvectors, ascending
    pos: np.ndarray                  # output index of each (leaf, local) entry
    lam: np.ndarray                  # eigenvalues in output order
    U: np.ndarray                    # n x n basis, columns in output order

    @property
    def n(self):
        return self.fact.n


def fast_gft(L: np.ndarray, phis, split_components: bool = False) -> FastGFT:
    fact = decompose(L, phis, split_components)
    n = fact.n
    Bs = [stage_matrix(n, p) for p in fact.stages]
    leaf_lams, leaf_vecs, cols, entries = [], [], [], []
    for k, leaf in enumerate(fact.leaves):
        lam, V = jacobi_eigh(leaf.L)
        order = np.argsort(lam, kind="stable")
        lam, V = lam[order], V[:, order].copy()
        for c in range(V.shape[1]):
            v = np.zeros(n)
            v[leaf.labels] = V[:, c]
            for B in reversed(Bs):       # U = B_1 B_2 ... B_S [U_k embedded]
                v = B @ v
            sg = canonical_sign(v)
            V[:, c] *= sg
            cols.append(v * sg)
            entries.append((float(lam[c]), k, c))
        leaf_lams.append(lam)
        leaf_vecs.append(V)
    pos = output_order(entries)
    U = np.zeros((n, n))
    lam_out = np.zeros(n)
    for i, (l, _, _) in enumerate(entries):
        U[:, pos[i]] = cols[i]
        lam_out[pos[i]] = l
    return FastGFT(fact, leaf_lams, leaf_vecs, pos, lam_out, U)


def forward_dense(U: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Coefficients of every row of X: Y = X U (y^T = U^T x per signal)."""
    return np.asarray(X, dtype=np.float64) @ U


def _leaf_positions(f: FastGFT):
    out, i = [], 0
    for V in f.leaf_vecs:
        m = V.shape[1]
        out.append(f.pos[i:i + m])
        i += m
    return out


def forward_staged(f: FastGFT, X: np.ndarray) -> np.ndarray:
    """Haar stages (B_phi^T per stage: (a+b)/sqrt2 at X, (a-b)/sqrt2 at the
    partner) then the leaf products U_k^T, placed in output order."""
    w = np.array(X, dtype=np.float64, copy=True)
    for pairs in f.fact.stages:
        if not pairs:
            continue
        xs = [p[0] for p in pairs]
        ys = [p[1] for p in pairs]
        a, b = w[:, xs].copy(), w[:, ys].copy()
        w[:, xs] = (a + b) / SQRT2
        w[:, ys] = (a - b) / SQRT2
    Y = np.zeros_like(w)
    for leaf, V, pos in zip(f.fact.leaves, f.leaf_vecs, _leaf_positions(f)):
        Y[:, pos] = w[:, leaf.labels] @ V
    return Y


def inverse_staged(f: FastGFT, Y: np.ndarray) -> np.ndarray:
    """Leaf products U_k, then the stages in reverse (B_phi is its own inverse)."""
    Y = np.asarray(Y, dtype=np.float64)
    w = np.zeros_like(Y)
    for leaf, V, pos in zip(f.fact.leaves, f.leaf_vecs, _leaf_positions(f)):
        w[:, leaf.labels] = Y[:, pos] @ V.T
    for pairs in reversed(f.fact.stages):
        if not pairs:
            continue
        xs = [p[0] for p in pairs]
        ys = [p[1] for p in pairs]
        a, b = w[:, xs].copy(), w[:, ys].copy()
        w[:, xs] = (a + b) / SQRT2
        w[:, ys] = (a - b) / SQRT2
    return w


def op_counts(f: FastGFT) -> Tuple[int, int]:
    """(additions, multiplications) per signal of the staged form with the
    1/sqrt2 factors folded into the leaf matrices: one add and one subtract
    per Haar unit, m^2 multiplies and m(m-1) adds per leaf of size m."""
    adds = sum(2 * len(p) for p in f.fact.stages)
    muls = 0
    for V in f.leaf_vecs:
        m = V.shape[1]
        muls += m * m
        adds += m * (m - 1)
    return adds, muls
