"""Wide-leaf CUDA-core kernel (leaves of 33..512 nodes) against the FP64
oracle: FP32 forward and inverse within relative L2 2e-6, FP64 within 1e-13,
after eigenspace alignment; ragged batches hit partial tiles.  Plan-specialised
kernels are switched off here (they would take the plans of at most 128
nodes); plans whose leaves also fit the table-driven kernel (at most 64
nodes) are run with both kernels forced.  The largest leaf width (512, a 1024-node path) is pinned
to the closed form instead: the uniform path's GFT is the DCT-II (Sec. V-B),
whatever the leaf width."""
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
    assert torch.cuda.is_available()
    from paper_1907_07875_gb300.build import build
    build()
    import paper_1907_07875_gb300 as gft
    return gft, torch


_REF = {}


def ref_of(g, split):
    key = (g.W.tobytes(), g.s.tobytes(), split, tuple(tuple(int(v) for v in p) for p in g.phis))
    if key not in _REF:
        _REF[key] = ogft.fast_gft(ograph.laplacian(g.W, g.s), g.phis, split_components=split)
    return _REF[key]


CASES = [(W.grid(16), False, True), (W.cycle(256), False, True), (W.path(100), False, True),
         (W.grid(12), False, True), (W.bipartite(160, 0.1, seed=3), True, False),
         (W.near_symmetric_grid(8, 0.05, seed=3), False, True), (W.bipartite(72, 0.2, seed=5), False, False)]


def _check(gft, torch, plan, ref, batch, seed):
    U = plan.basis()
    assert projector_distance(U, ref.U, ref.lam) <= 1e-10
    assert simple_column_sign_error(U, ref.U, ref.lam) <= 1e-9
    x = W.signals(batch, plan.n, seed)
    xt = torch.from_numpy(x).cuda()
    y = plan.forward(xt).cpu().numpy().astype(np.float64)
    y_ref = align(ogft.forward_dense(ref.U, x.astype(np.float64)), U, ref.U, ref.lam)
    assert rel_l2(y, y_ref) <= FP32_TOL
    xb = plan.inverse(torch.from_numpy(y.astype(np.float32)).cuda()).cpu().numpy()
    x_ref = ogft.inverse_staged(ref, align(y, ref.U, U, ref.lam))
    assert rel_l2(xb, x_ref) <= FP32_TOL
    yd = plan.forward(xt.double()).cpu().numpy()
    assert rel_l2(yd, x.astype(np.float64) @ U) <= FP64_TOL      # kernel arithmetic, FP64
    assert rel_l2(yd, y_ref) <= 1e-10                             # and the oracle's basis
    xd = plan.inverse(torch.from_numpy(yd).cuda()).cpu().numpy()
    assert rel_l2(xd, x.astype(np.float64)) <= FP64_TOL
    assert plan.device_error() == 0


@pytest.mark.parametrize("g,split,table_ok", CASES, ids=lambda v: getattr(v, "name", str(v)))
@pytest.mark.parametrize("batch", [1, 37, 1000])
def test_wide_kernel_vs_oracle(env, g, split, table_ok, batch):
    gft, torch = env
    ref = ref_of(g, split)
    kernels = ("wide", "table") if table_ok else ("wide", "auto")
    for kernel in kernels:
        plan = gft.Plan(gft.laplacian(g.W, g.s), g.phis, split_components=split, kernel=kernel, jit=False)
        assert plan.info["jit"] == 0
        if kernel == "wide":
            assert plan.info["wide"] == 1
        if kernel == "table":
            assert plan.info["wide"] == 0
        _check(gft, torch, plan, ref, batch, 300 + batch)


@pytest.mark.parametrize("kind", [4, 5])
def test_grid32_fp32_full_size(env, kind):
    """32x32 grids (leaves of 256 nodes) at the mixed-batch size of 2^23
    coefficients (8192 signals); every 5th signal compared with the oracle,
    FP64 on the first 256 signals."""
    gft, torch = env
    g, batch, seed = W.config3()[kind]
    plan = gft.Plan(gft.laplacian(g.W, g.s), g.phis)
    assert plan.info["wide"] == 1
    ref = ref_of(g, False)
    U = plan.basis()
    x = W.signals(batch, g.n, seed)
    xt = torch.from_numpy(x).cuda()
    y = plan.forward(xt).cpu().numpy().astype(np.float64)
    idx = np.arange(0, batch, 5)
    y_ref = align(ogft.forward_dense(ref.U, x[idx].astype(np.float64)), U, ref.U, ref.lam)
    assert rel_l2(y[idx], y_ref) <= FP32_TOL
    yd = plan.forward(xt[:256].double()).cpu().numpy()
    assert rel_l2(yd, x[:256].astype(np.float64) @ U) <= FP64_TOL
    xb = plan.inverse(torch.from_numpy(y.astype(np.float32)).cuda()).cpu().numpy()
    assert rel_l2(xb, x) <= 2 * FP32_TOL
    assert plan.device_error() == 0


def test_path1024_leaves_of_512_are_dct(env):
    """Uniform path, n = 1024, one reversal stage: two leaves of 512 nodes
    (the widest the kernel takes).  The plan's basis must be the DCT-II up to
    column signs (Sec. V-B, simple spectrum), and the FP32 / FP64 transforms
    must match x times that closed-form basis."""
    gft, torch = env
    n = 1024
    g = W.path(n)
    plan = gft.Plan(gft.laplacian(g.W, g.s), g.phis)
    assert plan.info["wide"] == 1 and plan.info["max_leaf"] == 512
    k = np.arange(n)
    D = np.sqrt(np.where(k == 0, 1.0, 2.0) / n)[None, :] * np.cos(np.pi * np.outer(np.arange(n) + 0.5, k) / n)
    U = plan.basis()
    S = np.sign(np.sum(D * U, axis=0))
    DS = D * S[None, :]
    assert np.max(np.abs(U - DS)) <= 1e-10
    lam = plan.eigenvalues()
    assert np.max(np.abs(lam - (2 - 2 * np.cos(np.pi * k / n)))) <= 1e-12
    x = W.signals(777, n, 8)
    xt = torch.from_numpy(x).cuda()
    y = plan.forward(xt).cpu().numpy().astype(np.float64)
    y_ref = x.astype(np.float64) @ DS
    assert rel_l2(y, y_ref) <= FP32_TOL
    yd = plan.forward(xt.double()).cpu().numpy()
    assert rel_l2(yd, x.astype(np.float64) @ U) <= FP64_TOL
    xb = plan.inverse(torch.from_numpy(y.astype(np.float32)).cuda()).cpu().numpy()
    assert rel_l2(xb, x) <= 2 * FP32_TOL
    assert plan.device_error() == 0
