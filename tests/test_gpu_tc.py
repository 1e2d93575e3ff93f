"""Tensor-core (tcgen05) leaf products: BF16, BF16 hi+lo and scaled FP16
hi+lo split precisions against the FP64 oracle, after eigenspace alignment.
Stated error bounds (relative L2 over the output): BF16 5e-3, BF16 split 1e-5,
FP16 split 2e-6 (the FP32 bound)."""
import numpy as np
import pytest

import gft_workloads as W
from oracle import gft as ogft
from oracle import graph as ograph
from _helpers import align, rel_l2

pytestmark = pytest.mark.gpu

BOUNDS = {"bf16": 5e-3, "bf16x3": 1e-5, "fp16x3": 2e-6}


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
    key = (g.W.tobytes(), g.s.tobytes(), split)
    if key not in _REF:
        _REF[key] = ogft.fast_gft(ograph.laplacian(g.W, g.s), g.phis, split_components=split)
    return _REF[key]


CASES = [(W.path(8), False), (W.skeleton25(), True), (W.grid(8), False), (W.grid(16), False),
         (W.grid(16, weights="sym_uniform", seed=2), False), (W.cycle(64), False), (W.cycle(256), False),
         (W.grid(32), False), (W.bipartite(160, 0.1, seed=3), True)]


@pytest.mark.parametrize("g,split", CASES, ids=lambda v: getattr(v, "name", str(v)))
@pytest.mark.parametrize("batch", [1, 129, 1000])
def test_tensor_core_precisions_vs_oracle(env, g, split, batch):
    gft, torch = env
    plan = gft.Plan(gft.laplacian(g.W, g.s), g.phis, split_components=split)
    ref = ref_of(g, split)
    U = plan.basis()
    x = W.signals(batch, g.n, 40 + batch)
    y_ref = align(ogft.forward_dense(ref.U, x.astype(np.float64)), U, ref.U, ref.lam)
    xt = torch.from_numpy(x).cuda()
    for prec, bound in BOUNDS.items():
        y = plan.forward(xt, precision=prec).cpu().numpy()
        err = rel_l2(y, y_ref)
        assert err <= bound, (prec, err)
    assert plan.device_error() == 0


def test_tensor_core_full_size_grid32(env):
    """32x32 grid at 2^23 coefficients (8192 signals), every 5th signal checked."""
    gft, torch = env
    g, batch, seed = W.config3()[4]
    plan = gft.Plan(gft.laplacian(g.W, g.s), g.phis)
    ref = ref_of(g, False)
    U = plan.basis()
    x = W.signals(batch, g.n, seed)
    idx = np.arange(0, batch, 5)
    y_ref = align(ogft.forward_dense(ref.U, x[idx].astype(np.float64)), U, ref.U, ref.lam)
    xt = torch.from_numpy(x).cuda()
    for prec in ("bf16x3", "fp16x3"):
        y = plan.forward(xt, precision=prec).cpu().numpy()[idx]
        assert rel_l2(y, y_ref) <= BOUNDS[prec]


def test_tensor_core_unsupported_cases(env):
    gft, torch = env
    g = W.grid(16)
    plan = gft.Plan(gft.laplacian(g.W, g.s), g.phis)
    x = torch.zeros(256, g.n, device="cuda")
    for call in (lambda: plan.inverse(x, precision="bf16x3"), lambda: plan.forward(x, out=x, precision="bf16x3")):
        with pytest.raises(gft.GftError) as e:
            call()
        assert e.value.status == "GFT_ERR_UNSUPPORTED"
    big = W.bipartite(1024, 0.1, seed=1)                # leaves of 512 nodes
    p2 = gft.Plan(gft.laplacian(big.W, big.s), big.phis)
    with pytest.raises(gft.GftError) as e:
        p2.forward(torch.zeros(128, 1024, device="cuda"), precision="bf16x3")
    assert e.value.status == "GFT_ERR_UNSUPPORTED"
