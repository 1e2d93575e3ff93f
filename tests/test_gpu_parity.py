"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

FP32 outputs: relative L2 error <= 2e-6 against the FP64 oracle after
eigenspace alignment (bases are unique only up to rotations inside repeated
eigenvalues, Sec. III).  FP64 outputs: <= 1e-13.  Integer plan data (stage
pairs, leaves, output map) bit-exact.  Eigenvalues within 1e-12 * max(1,
max|lambda|); basis projectors within 1e-10; columns of simple eigenvalues
equal to the oracle's entry by entry (the sign rule), within 1e-9.
"""
import numpy as np
import pytest

import gft_workloads as W
from oracle import gft as ogft
from oracle import graph as ograph
from _helpers import align, projector_distance, rel_l2, simple_column_sign_error

pytestmark = pytest.mark.gpu

FP32_TOL = 2e-6
FP64_TOL = 1e-13


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1907_07875_gb300.build import build
    build()
    import paper_1907_07875_gb300 as gft
    return gft, torch


_REF_CACHE = {}


def oracle_ref(g, split):
    key = (g.W.tobytes(), g.s.tobytes(), split, tuple(tuple(int(v) for v in p) for p in g.phis))
    if key not in _REF_CACHE:
        _REF_CACHE[key] = ogft.fast_gft(ograph.laplacian(g.W, g.s), g.phis, split_components=split)
    return _REF_CACHE[key]


def make_plan(gft, g, split, **kw):
    return gft.Plan(gft.laplacian(g.W, g.s), g.phis, split_components=split, **kw)


def check_plan_against_oracle(plan, ref):
    lam = plan.eigenvalues()
    scale = max(1.0, float(np.abs(ref.lam).max()))
    assert np.max(np.abs(lam - ref.lam)) <= 1e-12 * scale
    assert plan.output_map().tolist() == ref.pos.tolist()
    for s, pairs in enumerate(ref.fact.stages):
        assert plan.stage_pairs(s).tolist() == [list(p) for p in pairs]
    assert plan.leaves() == [b.labels for b in ref.fact.leaves]
    U = plan.basis()
    assert np.max(np.abs(U.T @ U - np.eye(plan.n))) <= 1e-12
    assert projector_distance(U, ref.U, ref.lam) <= 1e-10
    # simple eigenvalues: the library's sign rule gives the oracle's vector
    assert simple_column_sign_error(U, ref.U, ref.lam) <= 1e-9
    return U


def forward_error(gft, torch, plan, ref, U_gpu, x32, dtype="f32"):
    xt = torch.from_numpy(x32 if dtype == "f32" else x32.astype(np.float64)).cuda()
    y = plan.forward(xt).cpu().numpy().astype(np.float64)
    y_ref = align(ogft.forward_dense(ref.U, x32.astype(np.float64)), U_gpu, ref.U, ref.lam)
    return rel_l2(y, y_ref), y


FAMILIES = [
    (W.path(8), False), (W.path(9), False), (W.path(16), False), (W.cycle(12), False),
    (W.cycle(64), False), (W.grid(4), False), (W.grid(5, 3), False), (W.grid(8), False),
    (W.grid(8, weights="sym_uniform", seed=3), False), (W.skeleton25(), True), (W.skeleton25(), False),
    (W.bipartite(64, 0.1, seed=2), True), (W.bipartite(30, 0.3, seed=4), False),
    (W.planted_symmetric(11, np.array([10, 9, 2, 7, 4, 5, 6, 3, 8, 1, 0]), seed=2), False),
    (W.star(7), False), (W.complete(6), False), (W.near_symmetric_path(32, 0.05, seed=1), False),
    (W.grid6_bidiag(4), False), (W.grid6_bidiag(8), False), (W.zgrid(4), False), (W.zgrid(8), False),
    (W.cycle(80), False), (W.cycle(128), False), (W.grid(10), False), (W.bipartite(72, 0.2, seed=5), False),
    (W.path(100), False), (W.bipartite(128, 0.1, seed=3), False),
    (W.path_recursive(64), False), (W.path_recursive(100), False), (W.path_recursive(256), False),
    (W.cycle_recursive(64), False),
]


@pytest.mark.parametrize("g,split", FAMILIES, ids=lambda v: getattr(v, "name", str(v)))
@pytest.mark.parametrize("batch", [1, 37, 1000])
def test_forward_inverse_families(env, g, split, batch):
    gft, torch = env
    plan = make_plan(gft, g, split)
    ref = oracle_ref(g, split)
    U = check_plan_against_oracle(plan, ref)
    x = W.signals(batch, g.n, 11 + batch)
    err, y = forward_error(gft, torch, plan, ref, U, x)
    assert err <= FP32_TOL, err
    xb = plan.inverse(torch.from_numpy(y.astype(np.float32)).cuda()).cpu().numpy()
    x_ref = ogft.inverse_staged(ref, align(y, ref.U, U, ref.lam))
    assert rel_l2(xb, x_ref) <= FP32_TOL
    assert rel_l2(xb, x) <= 2 * FP32_TOL
    assert plan.device_error() == 0


@pytest.mark.parametrize("g,split", [(W.path(8), False), (W.skeleton25(), True), (W.grid(8), False),
                                     (W.cycle(12), False), (W.cycle(80), False), (W.cycle(128), False)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_fp64_path(env, g, split):
    gft, torch = env
    plan = make_plan(gft, g, split)
    ref = oracle_ref(g, split)
    U = plan.basis()
    x = W.signals(513, g.n, 5)
    err, y = forward_error(gft, torch, plan, ref, U, x, dtype="f64")
    assert err <= FP64_TOL, err
    back = plan.inverse(torch.from_numpy(y).cuda()).cpu().numpy()
    assert rel_l2(back, x.astype(np.float64)) <= FP64_TOL


def test_config1_path8_full(env):
    """Path N=8, 4096 signals, FP64 and FP32; the basis is DCT-II."""
    gft, torch = env
    (g, batch, seed), = W.config1()
    plan = make_plan(gft, g, False)
    ref = oracle_ref(g, False)
    U = check_plan_against_oracle(plan, ref)
    N = 8
    dct = np.array([[np.sqrt((1 if k == 0 else 2) / N) * np.cos(np.pi * k * (i + 0.5) / N) for k in range(N)]
                    for i in range(N)])
    assert np.allclose(np.abs(U), np.abs(dct), atol=1e-13)
    x = W.signals(batch, g.n, seed)
    e32, _ = forward_error(gft, torch, plan, ref, U, x)
    e64, _ = forward_error(gft, torch, plan, ref, U, x, dtype="f64")
    assert e32 <= FP32_TOL and e64 <= FP64_TOL


def test_config2_skeleton_full_batch(env):
    """25-joint skeleton, all 2^20 signals, in the launch configuration the
    benchmark times; every output compared with the oracle."""
    gft, torch = env
    (g, batch, seed), = W.config2()
    plan = make_plan(gft, g, True)
    ref = oracle_ref(g, True)
    U = check_plan_against_oracle(plan, ref)
    x = W.signals(batch, g.n, seed)
    err, y = forward_error(gft, torch, plan, ref, U, x)
    assert err <= FP32_TOL, err
    # worst single signal stays within a few times the global bound
    y_ref = align(ogft.forward_dense(ref.U, x.astype(np.float64)), U, ref.U, ref.lam)
    per = np.linalg.norm(y - y_ref, axis=1) / np.linalg.norm(y_ref, axis=1)
    assert per.max() <= 20 * FP32_TOL
    assert plan.device_error() == 0


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 6, 7])
def test_config3_core_kinds_full(env, kind):
    """Grids 8x8 / 16x16 (unit and symmetrised weights) and cycles 64 / 256
    at 2^23 coefficients each; every 7th signal compared with the oracle."""
    gft, torch = env
    g, batch, seed = W.config3()[kind]
    plan = make_plan(gft, g, False)
    ref = oracle_ref(g, False)
    U = check_plan_against_oracle(plan, ref)
    x = W.signals(batch, g.n, seed)
    y = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    idx = np.arange(0, batch, 7)
    y_ref = align(ogft.forward_dense(ref.U, x[idx].astype(np.float64)), U, ref.U, ref.lam)
    assert rel_l2(y[idx], y_ref) <= FP32_TOL


@pytest.mark.parametrize("n", [16, 32, 64])
def test_dense_plans_no_stages(env, n):
    """Zero stages = the dense GFT (one leaf of n nodes), as used for the
    nearly symmetric graphs of the learned-surrogate workload."""
    gft, torch = env
    g = W.near_symmetric_path(n, 0.05, seed=n) if n < 64 else W.near_symmetric_grid(8, 0.05, seed=3)
    plan = make_plan(gft, g, False)
    ref = oracle_ref(g, False)
    U = check_plan_against_oracle(plan, ref)
    x = W.signals(3001, g.n, 2)
    err, _ = forward_error(gft, torch, plan, ref, U, x)
    assert err <= FP32_TOL


def test_edge_cases(env):
    gft, torch = env
    g = W.skeleton25()
    plan = make_plan(gft, g, True)
    ref = oracle_ref(g, True)
    U = plan.basis()
    # batch 0 is a no-op
    e = torch.empty(0, 25, device="cuda")
    assert plan.forward(e).shape == (0, 25)
    # in place
    x = W.signals(777, 25, 3)
    xt = torch.from_numpy(x).cuda()
    plan.forward(xt, out=xt)
    y_ref = align(ogft.forward_dense(ref.U, x.astype(np.float64)), U, ref.U, ref.lam)
    assert rel_l2(xt.cpu().numpy(), y_ref) <= FP32_TOL
    # misaligned pointer is rejected before any launch
    big = torch.zeros(10 * 25 + 1, device="cuda")
    with pytest.raises(gft.GftError) as ex:
        plan.forward(big[1:].view(10, 25))
    assert ex.value.status == "GFT_ERR_MISALIGNED"
    # one-node and two-node graphs
    for gg in (W.Graph("single", np.zeros((1, 1)), np.array([0.5])), W.path(2), W.path(3)):
        p = gft.Plan(gft.laplacian(gg.W, gg.s), gg.phis if gg.n > 1 else [])
        xs = W.signals(65, gg.n, 1)
        r = ogft.fast_gft(ograph.laplacian(gg.W, gg.s), gg.phis if gg.n > 1 else [])
        err, _ = forward_error(gft, torch, p, r, p.basis(), xs)
        assert err <= FP32_TOL
    assert plan.device_error() == 0


def test_order_block_flag(env):
    gft, torch = env
    g = W.cycle(12)
    plan = make_plan(gft, g, False, order_block=True)
    assert plan.output_map().tolist() == list(range(12))
    ref = ogft.fast_gft(ograph.laplacian(g.W, g.s), g.phis)
    x = W.signals(100, 12, 4)
    y = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    U = plan.basis()
    assert rel_l2(y, x.astype(np.float64) @ U) <= FP32_TOL
    assert projector_distance(U[:, np.argsort(plan.eigenvalues(), kind="stable")],
                              ref.U, ref.lam) <= 1e-10


def test_forward_host_matches_device(env):
    gft, torch = env
    g = W.skeleton25()
    plan = make_plan(gft, g, True)
    x = W.signals(300001, 25, 9)
    y_dev = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    # pinned, device-mapped buffers: the kernel reads and writes host memory
    y_pinned = plan.forward_host(torch.from_numpy(x).pin_memory(), out=torch.empty(300001, 25).pin_memory()).numpy()
    assert np.array_equal(y_pinned, y_dev)
    # pageable buffers: chunked copies through device staging
    y_pageable = plan.forward_host(torch.from_numpy(x.copy())).numpy()
    assert np.array_equal(y_pageable, y_dev)
    assert plan.device_error() == 0


def test_plan_jacobi_matches_oracle_leaves(env):
    """Leaf eigenvalues from the GPU Jacobi equal the oracle's Jacobi."""
    gft, torch = env
    for g in (W.grid(8, weights="sym_uniform", seed=7), W.cycle(256), W.bipartite(200, 0.1, seed=1)):
        plan = make_plan(gft, g, True)
        ref = oracle_ref(g, True)
        lam = plan.eigenvalues()
        assert np.max(np.abs(lam - ref.lam)) <= 1e-12 * max(1.0, np.abs(ref.lam).max())
        assert plan.info["jacobi_sweeps"] <= 30


@pytest.mark.parametrize("g,split", [(W.path(8), False), (W.skeleton25(), True), (W.grid(8), False),
                                     (W.cycle(12), False), (W.path(9), False), (W.path(6), False),
                                     (W.grid(8, weights="sym_uniform", seed=3), False)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_specialised_kernel_matches_interpreter(env, g, split):
    """The plan-specialised (NVRTC) kernel and the table-driven kernel run
    the same FMA sequence, so their outputs agree bit for bit."""
    gft, torch = env
    pj = make_plan(gft, g, split)
    pi = make_plan(gft, g, split, jit=False)
    assert pj.info["jit"] in (1, 2) and pi.info["jit"] == 0
    x = torch.from_numpy(W.signals(4099, g.n, 21)).cuda()
    assert torch.equal(pj.forward(x), pi.forward(x))
    assert torch.equal(pj.inverse(x), pi.inverse(x))
    xd = x.double()
    assert torch.equal(pj.forward(xd), pi.forward(xd))
    assert torch.equal(pj.inverse(xd), pi.inverse(xd))
    src = pj.kernel_source()
    assert "gft_jit_fwd_0" in src and "body_fwd" in src


@pytest.mark.parametrize("g", [W.skeleton25(), W.grid(8), W.cycle(16), W.path(12),
                               W.grid(6, weights="sym_uniform", seed=4)], ids=lambda g: g.name)
def test_searched_stages_parity(env, g):
    """Plans whose stages come from the involution search (Sec. V-F) --
    deeper than the hand-given ones for grids and the skeleton -- against the
    oracle built on the same stages, and against the dense GFT's eigenspaces."""
    gft, torch = env
    L = gft.laplacian(g.W, g.s)
    phis = gft.search_stages(L, max_stages=6)
    plan = gft.Plan(L, phis)
    ref = ogft.fast_gft(ograph.laplacian(g.W, g.s), phis)
    U = check_plan_against_oracle(plan, ref)
    lam_d, U_d = ogft.dense_gft(ograph.laplacian(g.W, g.s))
    assert projector_distance(U, U_d, lam_d) <= 1e-10
    x = W.signals(1001, g.n, 17)
    err, y = forward_error(gft, torch, plan, ref, U, x)
    assert err <= FP32_TOL
    xb = plan.inverse(torch.from_numpy(y.astype(np.float32)).cuda()).cpu().numpy()
    assert rel_l2(xb, x) <= 2 * FP32_TOL


@pytest.mark.parametrize("g,split", [(W.skeleton25(), True), (W.grid(8, weights="sym_uniform", seed=3), False),
                                     (W.bipartite(64, 0.2, seed=2), False), (W.cycle(80), False),
                                     (W.grid6_bidiag(8), False)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_normalised_laplacian_plans(env, g, split):
    """GFTs of the normalised Laplacian D^-1/2 L D^-1/2 (Sec. II-B): the
    block diagonalisation holds for it too (Sec. IV-B, Thm. 3), so
    a plan built on it must match the oracle's fast GFT of the same matrix."""
    gft, torch = env
    Ln = gft.normalized_laplacian(g.W, g.s)
    assert np.allclose(Ln, ograph.normalized_laplacian(g.W, g.s), rtol=0, atol=1e-15)
    plan = gft.Plan(Ln, g.phis, split_components=split)
    ref = ogft.fast_gft(ograph.normalized_laplacian(g.W, g.s), g.phis, split_components=split)
    U = check_plan_against_oracle(plan, ref)
    x = W.signals(1000, g.n, 55)
    err, y = forward_error(gft, torch, plan, ref, U, x)
    assert err <= FP32_TOL, err
    xb = plan.inverse(torch.from_numpy(y.astype(np.float32)).cuda()).cpu().numpy()
    assert rel_l2(xb, x) <= 2 * FP32_TOL
    assert plan.device_error() == 0
