"""Bipartite plans with a right Haar stage (Sec. III-A, Lemma 1, Thms. 1-2)
on the GPU against the FP64 oracle (oracle.right_haar): the plan's
eigenvalues and eigenspaces, FP32 forward and inverse within relative L2
2e-6 after eigenspace alignment, FP64 within 1e-13 of x times the plan's
own basis and within 1e-10 of the oracle's; every CUDA-core kernel
(plan-specialised, table-driven, wide-leaf) and the mixed-batch kernels;
ragged batches hit partial tiles.  Cases: k-regular bipartite graphs
(combinatorial Laplacian, alpha = k), even cycles, hypercubes (highly
repeated spectrum, zero singular values), and random bipartite graphs with
unequal parts (normalised Laplacian, alpha = 1, unpaired columns)."""
import numpy as np
import pytest

import gft_workloads as W
from oracle import graph as ograph
from oracle import right_haar as orh
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


def _lap(g, normalised):
    return ograph.normalized_laplacian(g.W, g.s) if normalised else ograph.laplacian(g.W, g.s)


_REF = {}


def ref_of(g, normalised):
    key = (g.name, normalised, g.W.tobytes())
    if key not in _REF:
        _REF[key] = orh.right_haar_gft(_lap(g, normalised), g.meta.get("side"))
    return _REF[key]


def _check(torch, plan, ref, batch, seed, tol32=FP32_TOL):
    lam = plan.eigenvalues()
    assert np.max(np.abs(lam - ref.lam)) <= 1e-10 * max(1.0, ref.alpha)
    U = plan.basis()
    assert np.max(np.abs(U.T @ U - np.eye(ref.n))) <= 1e-12
    assert projector_distance(U, ref.U, ref.lam) <= 1e-9
    # simple eigenvalues, sum and difference vectors of the right units
    # alike: the sign rule fixes the sum vector and the difference follows
    assert simple_column_sign_error(U, ref.U, ref.lam) <= 1e-8
    x = W.signals(batch, ref.n, seed)
    xt = torch.from_numpy(x).cuda()
    y = plan.forward(xt).cpu().numpy().astype(np.float64)
    y_ref = align(orh.forward_staged(ref, x.astype(np.float64)), U, ref.U, ref.lam)
    assert rel_l2(y, y_ref) <= tol32
    xb = plan.inverse(torch.from_numpy(y.astype(np.float32)).cuda()).cpu().numpy()
    x_ref = orh.inverse_staged(ref, align(y, ref.U, U, ref.lam))
    assert rel_l2(xb, x_ref) <= tol32
    yd = plan.forward(xt.double()).cpu().numpy()
    assert rel_l2(yd, x.astype(np.float64) @ U) <= FP64_TOL
    assert rel_l2(yd, y_ref) <= 1e-10
    xd = plan.inverse(torch.from_numpy(yd).cuda()).cpu().numpy()
    assert rel_l2(xd, x.astype(np.float64)) <= FP64_TOL
    assert plan.device_error() == 0


CASES = W.right_haar_graphs()


@pytest.mark.parametrize("case", range(len(CASES)), ids=[g.name for g, _ in CASES])
@pytest.mark.parametrize("batch", [1, 37, 1000])
def test_bipartite_plan_vs_oracle(env, case, batch):
    gft, torch = env
    g, normalised = CASES[case]
    ref = ref_of(g, normalised)
    L = _lap(g, normalised)
    plan = gft.Plan.bipartite(L, g.meta.get("side"))
    assert plan.info["right_pairs"] == ref.p
    if g.n <= 128 and len(ref.big) ** 2 + ref.p ** 2 <= 8192:
        assert plan.info["jit"] in (1, 2)
    _check(torch, plan, ref, batch, 500 + batch)
    # the table-driven kernel (leaves of at most 64 nodes), plan-specialised kernels off
    if max(len(ref.big), ref.p) <= 64:
        pt = gft.Plan.bipartite(L, g.meta.get("side"), jit=False, kernel="table")
        assert pt.info["jit"] == 0 and pt.info["wide"] == 0
        _check(torch, pt, ref, batch, 600 + batch)
    # the wide-leaf kernel (a part of more than 32 nodes)
    if len(ref.big) > 32:
        pw = gft.Plan.bipartite(L, g.meta.get("side"), jit=False, kernel="wide")
        assert pw.info["wide"] == 1
        _check(torch, pw, ref, batch, 700 + batch)


@pytest.mark.parametrize("which", ["krbg512_k8", "rbip300x212"])
def test_large_bipartite_wide_kernel(env, which):
    """n = 512: a 8-regular bipartite graph (parts of 256) and a normalised
    random bipartite graph with parts 300 / 212 (88 unpaired columns); 2^21
    coefficients, every 7th signal compared with the oracle."""
    gft, torch = env
    if which == "krbg512_k8":
        g, normalised = W.krbg(256, 8, seed=2201), False
    else:
        g, normalised = W.random_bipartite(300, 212, 0.05, seed=2202), True
    ref = ref_of(g, normalised)
    plan = gft.Plan.bipartite(_lap(g, normalised), g.meta["side"])
    assert plan.info["wide"] == 1 and plan.info["right_pairs"] == ref.p
    assert np.max(np.abs(plan.eigenvalues() - ref.lam)) <= 1e-10 * max(1.0, ref.alpha)
    U = plan.basis()
    assert projector_distance(U, ref.U, ref.lam) <= 1e-8
    assert simple_column_sign_error(U, ref.U, ref.lam) <= 1e-7
    batch = (1 << 21) // g.n
    x = W.signals(batch, g.n, 33)
    xt = torch.from_numpy(x).cuda()
    y = plan.forward(xt).cpu().numpy().astype(np.float64)
    idx = np.arange(0, batch, 7)
    y_ref = align(orh.forward_staged(ref, x[idx].astype(np.float64)), U, ref.U, ref.lam)
    assert rel_l2(y[idx], y_ref) <= FP32_TOL
    xb = plan.inverse(torch.from_numpy(y.astype(np.float32)).cuda()).cpu().numpy()
    assert rel_l2(xb, x) <= 2 * FP32_TOL
    yd = plan.forward(xt[:128].double()).cpu().numpy()
    assert rel_l2(yd, x[:128].astype(np.float64) @ U) <= FP64_TOL
    assert plan.device_error() == 0


def test_bipartite_in_mixed_batch(env):
    """Bipartite plans in one graph launch with a symmetric-graph plan: the
    table-driven batch kernel (parts of at most 64) and the wide-leaf batch
    kernel (a part of 80) apply the right Haar units too."""
    gft, torch = env
    items = [(W.krbg(20, 4, seed=2102, weighted=False), False), (W.random_bipartite(80, 48, 0.1, seed=2203), True)]
    plans, refs, xs, ys = [], [], [], []
    for k, (g, nz) in enumerate(items):
        plans.append(gft.Plan.bipartite(_lap(g, nz), g.meta["side"]))
        refs.append(ref_of(g, nz))
    gs = W.skeleton25()
    plans.append(gft.Plan(gft.laplacian(gs.W, gs.s), gs.phis, split_components=True))
    batches = [1000, 333, 700]
    for p, b in zip(plans, batches):
        xs.append(torch.from_numpy(W.signals(b, p.n, 90 + b)).cuda())
        ys.append(torch.empty_like(xs[-1]))
    for prec in ("fp32", "bf16x3"):
        bt = gft.Batch(plans, batches, precision=prec)
        bt.forward(xs, ys)
        torch.cuda.synchronize()
        for p, ref, x, y in zip(plans[:2], refs, xs, ys):
            U = p.basis()
            y_ref = align(orh.forward_staged(ref, x.cpu().numpy().astype(np.float64)), U, ref.U, ref.lam)
            assert rel_l2(y.cpu().numpy(), y_ref) <= FP32_TOL
            assert p.device_error() == 0
        single = plans[2].forward(xs[2])
        assert rel_l2(ys[2].cpu().numpy(), single.cpu().numpy()) <= 1e-6
        bt.close()


def test_tensor_core_precision_is_unsupported(env):
    gft, torch = env
    g = W.krbg(32, 5, seed=2105)
    plan = gft.Plan.bipartite(_lap(g, False), g.meta["side"])
    x = torch.randn(256, g.n, device="cuda")
    with pytest.raises(gft.GftError) as e:
        plan.forward(x, precision="bf16x3")
    assert e.value.status == "GFT_ERR_UNSUPPORTED"
