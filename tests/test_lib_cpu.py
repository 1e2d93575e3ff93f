"""CPU tests of the C-ABI library: it loads, exports every symbol that
include/gft.h declares, and its host-side plan analysis (integer work:
partitions, pairs, leaves, leaf Laplacians) matches the oracle bit for bit.
No GPU calls: plans are built with GFT_ANALYZE_ONLY."""
import os
import re
import subprocess

import numpy as np
import pytest

import gft_workloads as W
from oracle import gft as ogft
from oracle import graph as ograph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def gft():
    from paper_1907_07875_gb300.build import build
    build()
    import paper_1907_07875_gb300 as m
    m.lib()
    return m


def header_functions():
    txt = open(os.path.join(ROOT, "include", "gft.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gft_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(gft):
    from paper_1907_07875_gb300 import _native
    names = header_functions()
    assert len(names) >= 25
    lib = gft.lib()
    for nm in names:
        assert hasattr(lib, nm), nm
        assert nm in _native.SIGNATURES, nm
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gft_[a-z0-9_]+)", out))
    assert set(names) <= exported


def test_status_strings(gft):
    lib = gft.lib()
    for code, name in gft.STATUS.items():
        assert lib.gft_status_string(code).decode() == name
    assert lib.gft_version() >= 10000


def test_laplacian_matches_oracle(gft):
    for g in (W.skeleton25(), W.grid(5, weights="sym_uniform", seed=1), W.bipartite(12, 0.5, seed=3),
              W.planted_symmetric(7, np.array([6, 5, 2, 3, 4, 1, 0]), seed=4)):
        L = gft.laplacian(g.W, g.s)
        assert np.allclose(L, ograph.laplacian(g.W, g.s), rtol=0, atol=1e-15)
    with pytest.raises(gft.GftError) as e:
        gft.laplacian(np.array([[0, 1.0], [2.0, 0]]))
    assert e.value.status == "GFT_ERR_NOT_LAPLACIAN"


def _families():
    return [W.path(8), W.path(9), W.cycle(12), W.cycle(64), W.grid(4), W.grid(5, 4), W.grid(8),
            W.grid(6, weights="sym_uniform", seed=9), W.skeleton25(), W.bipartite(32, 0.2, seed=5),
            W.planted_symmetric(11, np.array([10, 9, 2, 7, 4, 5, 6, 3, 8, 1, 0]), seed=2)]


@pytest.mark.parametrize("g", _families(), ids=lambda g: g.name)
@pytest.mark.parametrize("split", [False, True])
def test_plan_structure_bit_exact(gft, g, split):
    """Stage pairs, leaf node lists (DFS order, + before -), and leaf
    Laplacians from the library equal the oracle's decomposition."""
    L = ograph.laplacian(g.W, g.s)
    plan = gft.Plan(L, g.phis, split_components=split, analyze_only=True)
    ref = ogft.decompose(L, g.phis, split_components=split)
    for s, pairs in enumerate(ref.stages):
        assert plan.stage_pairs(s).tolist() == [list(p) for p in pairs]
    assert plan.leaves() == [b.labels for b in ref.leaves]
    for k, b in enumerate(ref.leaves):
        assert np.allclose(plan.leaf_laplacian(k), b.L, rtol=0, atol=1e-13 * max(1, np.abs(L).max()))
    inf = plan.info
    assert inf["n_leaves"] == len(ref.leaves) and inf["has_device"] == 0
    adds, muls = (sum(2 * len(p) for p in ref.stages) + sum(len(b.labels) * (len(b.labels) - 1) for b in ref.leaves),
                  sum(len(b.labels) ** 2 for b in ref.leaves))
    assert (inf["fast_adds"], inf["fast_mults"]) == (adds, muls)


def test_error_codes(gft):
    g = W.path(6)
    L = ograph.laplacian(g.W, g.s)
    cases = [
        (dict(L=L, phis=[[1, 2, 0, 3, 4, 5]]), "GFT_ERR_NOT_INVOLUTION"),
        (dict(L=L, phis=[[0, 1, 2, 3, 4, 7]]), "GFT_ERR_NOT_INVOLUTION"),
        (dict(L=L, phis=[[1, 0, 2, 3, 4, 5]]), "GFT_ERR_NOT_SYMMETRIC"),
        (dict(L=L, phis=[W.reversal(6), [5, 1, 2, 3, 4, 0]]), "GFT_ERR_BLOCK_LEAK"),
        (dict(L=L + np.triu(np.ones((6, 6)) * 1e-3, 1), phis=[]), "GFT_ERR_NOT_LAPLACIAN"),
        (dict(L=np.where(np.eye(6) > 0, np.nan, L), phis=[]), "GFT_ERR_NOT_LAPLACIAN"),
    ]
    for kw, status in cases:
        with pytest.raises(gft.GftError) as e:
            gft.Plan(kw["L"], kw["phis"], analyze_only=True)
        assert e.value.status == status, (kw, e.value)
    # a stage that pairs a node already paired once with a node never paired
    # (different numbers of earlier stages) is reported as unsupported
    g3 = W.planted_symmetric(4, np.array([3, 1, 2, 0]), density=1.0, seed=1)
    L3 = ograph.laplacian(g3.W, g3.s)
    try:
        gft.Plan(L3, [[3, 1, 2, 0], [1, 0, 2, 3]], analyze_only=True)
    except gft.GftError as e:
        assert e.status in ("GFT_ERR_UNSUPPORTED", "GFT_ERR_BLOCK_LEAK", "GFT_ERR_NOT_SYMMETRIC")
    lib = gft.lib()
    import ctypes as C
    assert lib.gft_plan_create(0, None, 0, None, 0, C.byref(C.c_void_p())) == 1
    assert lib.gft_plan_create(4, None, 0, None, 0, C.byref(C.c_void_p())) == 1
    assert lib.gft_plan_destroy(None) == 0


def test_analyze_only_plan_refuses_device_calls(gft):
    g = W.path(8)
    plan = gft.Plan(ograph.laplacian(g.W, g.s), g.phis, analyze_only=True)
    for call in (plan.eigenvalues, plan.basis, plan.output_map, plan.device_error):
        with pytest.raises(gft.GftError) as e:
            call()
        assert e.value.status == "GFT_ERR_NO_DEVICE"


def test_create_many_analysis_matches_single_and_is_all_or_nothing(gft):
    """gft_plan_create_many decomposes each graph exactly as gft_plan_create
    does (bit-exact stage pairs and leaves against the oracle); one bad graph
    fails the whole call with that graph's status."""
    graphs = [W.path(9), W.cycle(12), W.grid(5, 4), W.skeleton25(), W.bipartite(16, 0.3, seed=2)]
    Ls = [ograph.laplacian(g.W, g.s) for g in graphs]
    plans = gft.plans_from_laplacians(Ls, [g.phis for g in graphs], analyze_only=True)
    for g, L, plan in zip(graphs, Ls, plans):
        ref = ogft.decompose(L, g.phis)
        assert plan.leaves() == [b.labels for b in ref.leaves]
        for s, pairs in enumerate(ref.stages):
            assert plan.stage_pairs(s).tolist() == [list(p) for p in pairs]
    bad = [list(range(6))[::-1], [1, 2, 0, 3, 4, 5]]
    p6 = ograph.laplacian(W.path(6).W, W.path(6).s)
    with pytest.raises(gft.GftError) as e:
        gft.plans_from_laplacians([p6, p6], [[bad[0]], [bad[1]]], analyze_only=True)
    assert e.value.status == "GFT_ERR_NOT_INVOLUTION"


def test_normalized_laplacian_matches_oracle(gft):
    for g in (W.random_bipartite(7, 4, 0.4, seed=2103), W.krbg(8, 3, seed=2101), W.skeleton25()):
        N = gft.normalized_laplacian(g.W, g.s)
        assert np.allclose(N, ograph.normalized_laplacian(g.W, g.s), rtol=0, atol=1e-15)
    Wm = np.zeros((3, 3))
    Wm[0, 1] = Wm[1, 0] = 1.0                                      # node 2 isolated
    with pytest.raises(gft.GftError) as e:
        gft.normalized_laplacian(Wm)
    assert e.value.status == "GFT_ERR_NOT_LAPLACIAN"


@pytest.mark.parametrize("case", range(len(W.right_haar_graphs())))
def test_bipartite_plan_structure(gft, case):
    """Parts (two-colouring or given), E / F leaf node lists, the number of
    right Haar units and the operation counts equal the oracle's."""
    from oracle import right_haar as orh
    g, normalised = W.right_haar_graphs()[case]
    L = ograph.normalized_laplacian(g.W, g.s) if normalised else ograph.laplacian(g.W, g.s)
    ref = orh.right_haar_gft(L, g.meta.get("side"))
    for side in (g.meta.get("side"), None):
        plan = gft.Plan.bipartite(L, side, analyze_only=True)
        inf = plan.info
        if side is None and g.meta.get("side") is not None:
            # two-colouring may name the parts the other way round; the
            # larger part is E's either way (ties: colour 0 of the colouring)
            auto = ograph.bipartition(L, 1e-12 * max(1.0, np.abs(L).max()))
            assert orh.right_structure(L, auto)[1] == plan.leaves()[0]
            continue
        assert plan.leaves() == [ref.big, ref.small]
        assert inf["right_pairs"] == ref.p and inf["n_stages"] == 0 and inf["n_pairs"] == 0
        assert (inf["fast_adds"], inf["fast_mults"]) == orh.op_counts(ref)
        with pytest.raises(gft.GftError) as e:
            plan.leaf_laplacian(0)
        assert e.value.status == "GFT_ERR_UNSUPPORTED"


def test_bipartite_plan_errors(gft):
    def status(L, side=None, **kw):
        with pytest.raises(gft.GftError) as e:
            gft.Plan.bipartite(L, side, analyze_only=True, **kw)
        return e.value.status
    assert status(ograph.laplacian(W.cycle(7).W, W.cycle(7).s)) == "GFT_ERR_NOT_BIPARTITE"     # odd cycle
    assert status(ograph.laplacian(W.path(6).W, W.path(6).s)) == "GFT_ERR_NOT_BIPARTITE"       # degrees 1 and 2
    g = W.krbg(4, 2, seed=1, shuffle=False)
    L = ograph.laplacian(g.W, g.s)
    bad = g.meta["side"].copy()
    bad[0], bad[4] = bad[4], bad[0]
    assert status(L, bad) == "GFT_ERR_NOT_BIPARTITE"                                          # edge inside a part
    assert status(L, np.full(8, 2)) == "GFT_ERR_INVALID_ARG"
    assert status(L + np.triu(np.ones((8, 8)) * 1e-3, 1)) == "GFT_ERR_NOT_LAPLACIAN"
    import ctypes as C
    lib = gft.lib()
    h = C.c_void_p()
    assert lib.gft_plan_create_bipartite(8, L.ctypes.data, None, 0x1, C.byref(h)) == 1          # SPLIT flag
    assert lib.gft_plan_create_bipartite(8, None, None, 0, C.byref(h)) == 1


def _leaf_runs(lib_layers, n_haar, leaves):
    """Split the library's Givens layers into per-leaf layer lists (leaf
    node sets from the oracle's decomposition)."""
    owner = {}
    for k, leaf in enumerate(leaves):
        for lab in leaf.labels:
            owner[lab] = k
    runs = [[] for _ in leaves]
    for layer in lib_layers[n_haar:]:
        per = [[] for _ in leaves]
        for p, q, m in layer:
            assert owner[p] == owner[q]                 # a rotation never leaves its leaf
            per[owner[p]].append((p, q, m))
        for k in range(len(leaves)):
            if per[k]:
                runs[k].append(per[k])
    return runs


def _check_greedy_run(Lk, labels, layers, tol_rel=1e-9):
    """Replays one leaf's layers on the oracle's leaf Laplacian: every layer
    is disjoint, greedy (each pair has the largest |a_pq| among pairs of free
    nodes, up to rounding), maximal, and its rotations zero the chosen
    entries (with equal diagonal entries both angles +-pi/4 do); returns the
    final matrix."""
    from oracle import approx as oap
    A = np.array(Lk, dtype=np.float64, copy=True)
    m = A.shape[0]
    scale = max(1.0, np.abs(A).max())
    zero = oap.ZERO_TOL * scale
    eps = tol_rel * scale
    loc = {lab: i for i, lab in enumerate(labels)}
    for layer in layers:
        free = np.ones(m, dtype=bool)
        rots = []
        for gp, gq, (m00, m01, m10, m11) in layer:
            p, q = sorted((loc[gp], loc[gq]))
            assert free[p] and free[q]
            up = np.abs(np.triu(A, 1))
            best = max((up[r, t] for r in range(m) for t in range(r + 1, m) if free[r] and free[t]), default=0.0)
            assert up[p, q] >= best - eps and up[p, q] > zero - eps
            # a rotation (the entry it must zero is checked after the update),
            # the smaller angle of the symmetric Schur step: |theta| <= pi/4
            assert m01 == -m10 and m11 == m00 and abs(m00 * m00 + m10 * m10 - 1) <= 1e-15
            assert m00 >= abs(m10) - 1e-15
            free[p] = free[q] = False
            rots.append((loc[gp], loc[gq], m00, m10))
        up = np.abs(np.triu(A, 1))
        assert all(up[r, t] <= zero + eps for r in range(m) for t in range(r + 1, m) if free[r] and free[t])
        for p, q, c, s_ in rots:
            ap, aq = A[:, p].copy(), A[:, q].copy()
            A[:, p] = c * ap - s_ * aq
            A[:, q] = s_ * ap + c * aq
        for p, q, c, s_ in rots:
            ap, aq = A[p, :].copy(), A[q, :].copy()
            A[p, :] = c * ap - s_ * aq
            A[q, :] = s_ * ap + c * aq
        for p, q, _, _ in rots:
            assert abs(A[p, q]) <= 1e-9 * scale
            A[p, q] = A[q, p] = 0.0
    return A


APPROX_CASES = [(W.grid6_bidiag(8), 20), (W.zgrid(8), 20), (W.skeleton25(), 8),
                (W.near_symmetric_path(16, 0.05, seed=1), 30), (W.grid6_bidiag(4), 0),
                (W.grid(6, weights="sym_uniform", seed=9), 12)]


@pytest.mark.parametrize("g,J", APPROX_CASES, ids=lambda v: getattr(v, "name", str(v)))
@pytest.mark.parametrize("haar", [True, False])
def test_approx_build_is_a_valid_greedy_run(gft, g, J, haar):
    """The library's host build of the approximate GFT, replayed on the
    oracle's leaf Laplacians: Haar units exactly Eq. 20's, every Givens
    layer a valid greedy Jacobi layer, eigenvalues = the replayed diagonal,
    output order ascending, U_hat = the units applied to the identity.
    (Where magnitudes tie up to rounding the greedy choice can differ from
    the oracle's own run; the test_approx_*_matches_oracle cases have none.)"""
    from oracle import approx as oap
    from oracle import gft as og
    L = ograph.laplacian(g.W, g.s)
    phis = g.phis if haar else []
    a = gft.ApproxGFT(L, phis, J, analyze_only=True)
    lo, pairs, coef, perm = a.units()
    layers = [[(int(pairs[u, 0]), int(pairs[u, 1]), tuple(coef[u])) for u in range(lo[l], lo[l + 1])]
              for l in range(len(lo) - 1)]
    fact = og.decompose(L, phis)
    n_haar = a.info["n_haar_layers"]
    assert n_haar == len(fact.stages)
    r = 1 / np.sqrt(2)
    for st, layer in zip(fact.stages, layers[:n_haar]):
        assert [(p, q) for p, q, _ in layer] == list(st)
        assert all(m == (r, r, r, -r) for _, _, m in layer)
    runs = _leaf_runs(layers, n_haar, fact.leaves)
    diag = {}
    for leaf, run in zip(fact.leaves, runs):
        assert len(run) <= J
        A = _check_greedy_run(leaf.L, leaf.labels, run)
        for i, lab in enumerate(leaf.labels):
            diag[lab] = A[i, i]
    lam = a.eigenvalues()
    assert np.max(np.abs(lam - np.array([diag[int(v)] for v in perm]))) <= 1e-9 * max(1.0, np.abs(L).max())
    assert np.all(np.diff(lam) >= -1e-9 * max(1.0, np.abs(lam).max()))
    assert sorted(perm.tolist()) == list(range(g.n))
    assert np.max(np.abs(a.basis() - oap.apply_units(layers, np.eye(g.n))[:, perm])) <= 1e-13


@pytest.mark.parametrize("g,J", [(W.near_symmetric_path(16, 0.05, seed=1), 30),
                                 (W.grid(6, weights="sym_uniform", seed=9), 12), (W.grid6_bidiag(4), 0)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_approx_build_matches_oracle(gft, g, J):
    """Without ties the library's run and the oracle's are the same: same
    layers, pairs, permutation; coefficients, eigenvalues and U_hat to 1e-12."""
    from oracle import approx as oap
    L = ograph.laplacian(g.W, g.s)
    ref = oap.haar_approx_gft(L, [], J)
    a = gft.ApproxGFT(L, [], J, analyze_only=True)
    lo, pairs, coef, perm = a.units()
    assert lo.tolist() == np.cumsum([0] + [len(layer) for layer in ref.layers]).tolist()
    ref_units = [u for layer in ref.layers for u in layer]
    assert pairs.tolist() == [[p, q] for p, q, _ in ref_units]
    if ref_units:
        assert np.max(np.abs(coef - np.array([m for _, _, m in ref_units]))) <= 1e-12
    assert perm.tolist() == ref.perm.tolist()
    assert np.max(np.abs(a.eigenvalues() - ref.lam)) <= 1e-12 * max(1.0, np.abs(L).max())
    assert np.max(np.abs(a.basis() - ref.U)) <= 1e-12


@pytest.mark.parametrize("g,split", [(W.skeleton25(), True), (W.grid(6, weights="sym_uniform", seed=9), False),
                                     (W.bipartite(32, 0.2, seed=5), False), (W.zgrid(8), False)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_normalised_laplacian_plan_structure(gft, g, split):
    """The symmetric decomposition of the normalised Laplacian (Sec. II-B;
    Thm. 3 holds for it as well): stage pairs and leaves bit-exact, leaf
    matrices equal to the oracle's."""
    N = ograph.normalized_laplacian(g.W, g.s)
    plan = gft.Plan(N, g.phis, split_components=split, analyze_only=True)
    ref = ogft.decompose(N, g.phis, split_components=split)
    for s, pairs in enumerate(ref.stages):
        assert plan.stage_pairs(s).tolist() == [list(p) for p in pairs]
    assert plan.leaves() == [b.labels for b in ref.leaves]
    for k, b in enumerate(ref.leaves):
        assert np.allclose(plan.leaf_laplacian(k), b.L, rtol=0, atol=1e-13)


def test_approx_errors(gft):
    import ctypes as C
    lib = gft.lib()
    g = W.grid6_bidiag(4)
    L = ograph.laplacian(g.W, g.s)
    h = C.c_void_p()
    ptr = L.ctypes.data
    assert lib.gft_approx_create(16, ptr, 0, None, -1, 0x4, C.byref(h)) == 1          # n_layers < 0
    assert lib.gft_approx_create(16, ptr, 0, None, 4097, 0x4, C.byref(h)) == 1        # n_layers > 4096
    assert lib.gft_approx_create(16, ptr, 0, None, 3, 0x8, C.byref(h)) == 1           # NO_JIT is not an approx flag
    assert lib.gft_approx_create(2000, ptr, 0, None, 3, 0x4, C.byref(h)) == 1         # n > 1024
    assert lib.gft_approx_create(16, None, 0, None, 3, 0x4, C.byref(h)) == 1
    assert lib.gft_approx_create(16, ptr, 1, None, 3, 0x4, C.byref(h)) == 1           # stages without phi
    with pytest.raises(gft.GftError) as e:
        gft.ApproxGFT(L, [[1, 2, 0] + list(range(3, 16))], 3, analyze_only=True)    # not an involution
    assert e.value.status == "GFT_ERR_NOT_INVOLUTION"
    a = gft.ApproxGFT(L, g.phis, 3, analyze_only=True)
    assert a.info["has_device"] == 0
    x = np.zeros((4, 16), dtype=np.float32)
    assert lib.gft_approx_forward(a._h, x.ctypes.data, x.ctypes.data, 4, None) == 12       # GFT_ERR_NO_DEVICE
    assert lib.gft_approx_destroy(None) == 0


@pytest.mark.parametrize("g", [W.skeleton25(), W.grid(6), W.cycle(16), W.grid6_bidiag(4), W.path(12)],
                         ids=lambda g: g.name)
def test_search_flag_equals_explicit_search(gft, g):
    """GFT_SEARCH_STAGES builds the plan on the stages gft_search_stages
    returns (up to 16 stages): same pairs and leaves as passing them."""
    L = ograph.laplacian(g.W, g.s)
    phis = gft.search_stages(L, max_stages=16)
    a = gft.Plan(L, search=True, analyze_only=True)
    b = gft.Plan(L, phis, analyze_only=True)
    assert a.info["n_stages"] == b.info["n_stages"] == len(phis) >= 1
    for s in range(len(phis)):
        assert a.stage_pairs(s).tolist() == b.stage_pairs(s).tolist()
    assert a.leaves() == b.leaves()
    many = gft.plans_from_laplacians([L, L], [[], []], search=True, analyze_only=True)
    assert all(p.leaves() == b.leaves() for p in many)
    with pytest.raises(gft.GftError) as e:
        gft.Plan(L, g.phis or [list(range(g.n))], search=True, analyze_only=True)
    assert e.value.status == "GFT_ERR_INVALID_ARG"


@pytest.mark.parametrize("g", [W.skeleton25(), W.grid(6, weights="sym_uniform", seed=9), W.zgrid(4)],
                         ids=lambda g: g.name)
def test_normalized_flag_equals_normalised_input(gft, g):
    """GFT_NORMALIZED: the plan of L with the flag is the plan of
    D^-1/2 L D^-1/2 (same pairs, leaves and leaf matrices, bit for bit)."""
    L = ograph.laplacian(g.W, g.s)
    a = gft.Plan(L, g.phis, normalized=True, analyze_only=True)
    b = gft.Plan(gft.normalized_laplacian(g.W, g.s), g.phis, analyze_only=True)
    assert a.leaves() == b.leaves()
    for k in range(len(a.leaves())):
        assert np.array_equal(a.leaf_laplacian(k), b.leaf_laplacian(k))
    Z = np.zeros((3, 3))
    Z[0, 1] = Z[1, 0] = -1.0
    Z[0, 0] = Z[1, 1] = 1.0                                          # node 2 has degree 0
    with pytest.raises(gft.GftError) as e:
        gft.Plan(Z, [], normalized=True, analyze_only=True)
    assert e.value.status == "GFT_ERR_NOT_LAPLACIAN"


def test_bipartite_normalized_flag(gft):
    """Thm. 2 from the combinatorial Laplacian: the flag gives the plan of the
    normalised Laplacian (alpha = 1), whose parts need not be regular."""
    g = W.random_bipartite(7, 4, 0.4, seed=2103)
    L = ograph.laplacian(g.W, g.s)
    with pytest.raises(gft.GftError) as e:
        gft.Plan.bipartite(L, g.meta["side"], analyze_only=True)         # unequal degrees
    assert e.value.status == "GFT_ERR_NOT_BIPARTITE"
    a = gft.Plan.bipartite(L, g.meta["side"], normalized=True, analyze_only=True)
    b = gft.Plan.bipartite(gft.normalized_laplacian(g.W, g.s), g.meta["side"], analyze_only=True)
    assert a.leaves() == b.leaves() and a.info["right_pairs"] == 4


def test_batch_flags_and_device_check(gft):
    """gft_batch_create: an unknown flag bit is rejected before anything
    else; GFT_BATCH_NO_JIT or'ed into a precision is a known flag, so a plan
    without device data is then reported as such."""
    import ctypes as C
    g = W.path(8)
    plan = gft.Plan(ograph.laplacian(g.W, g.s), g.phis, analyze_only=True)
    lib = gft.lib()
    arr = (C.c_void_p * 1)(plan.handle)
    b = np.array([16], dtype=np.int64)
    out = C.c_void_p()
    status = lambda flags: lib.gft_batch_create(1, C.cast(arr, C.c_void_p), b.ctypes.data_as(C.c_void_p), flags,
                                                C.byref(out))
    assert gft.STATUS[status(0x200)] == "GFT_ERR_INVALID_ARG"
    assert gft.STATUS[status(4)] == "GFT_ERR_INVALID_ARG"                  # precision past GFT_PREC_FP16X3
    assert gft.STATUS[status(gft.Batch.BATCH_NO_JIT | 3)] == "GFT_ERR_NO_DEVICE"
    assert gft.STATUS[status(gft.Batch.BATCH_NO_JIT)] == "GFT_ERR_NO_DEVICE"
    assert gft.STATUS[status(3)] == "GFT_ERR_NO_DEVICE"
