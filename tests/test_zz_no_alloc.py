"""The allocation-free Givens backward entry point (gft_givens_backward_noalloc),
called through the C ABI, against the allocating gft_givens_backward.

It exists for callers that cannot allocate device memory while running (a
program whose own pool owns the GPU's memory, a real-time loop that must not
allocate mid-step, a thin C host without an allocator): it keeps its scratch
in a fixed array inside the library.  Several calls in a row with
different network shapes (butterfly and random-matching wirings, ragged
batches, a single signal, batch 0) check that the shared scratch carries
nothing over.  This file sorts last so that a run stopping at the first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import gft_workloads as W

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4      # angle-gradient tolerance used by the Givens tests


def _xor_pairs(n, S):
    lg = int(np.log2(n))
    out = np.zeros((S, n // 2, 2), dtype=np.int32)
    for t in range(S):
        bit = 1 << (t % lg)
        lo = [i for i in range(n) if not i & bit]
        out[t, :, 0] = lo
        out[t, :, 1] = [i | bit for i in lo]
    return out


def _random_pairs(n, S, seed):
    """S stages, each a random perfect matching of the n nodes (the general,
    non-butterfly wiring)."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.permutation(n).reshape(n // 2, 2) for _ in range(S)]).astype(np.int32)


def test_noalloc_backward_matches_allocating_backward():
    import torch
    assert torch.cuda.is_available()
    from paper_1907_07875_gb300.build import build
    build()
    import paper_1907_07875_gb300 as gft
    lib = gft.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = ((32, 10, 5003, 1, _xor_pairs(32, 10)), (16, 8, 777, 2, _xor_pairs(16, 8)),
             (16, 8, 1, 3, _xor_pairs(16, 8)), (24, 7, 1000, 4, _random_pairs(24, 7, 40)),
             (64, 12, 129, 5, _random_pairs(64, 12, 41)))
    for n, S, B, seed, pairs in cases:
        rng = np.random.default_rng(seed)
        theta = torch.from_numpy(rng.uniform(-1, 1, (S, n // 2)).astype(np.float32)).cuda()
        net = gft.Givens(n, pairs)
        y = net.forward(theta, torch.from_numpy(W.signals(B, n, seed)).cuda())
        gy = torch.from_numpy(rng.standard_normal((B, n)).astype(np.float32)).cuda()
        gx_ref, gth_ref = net.backward(theta, y, gy)
        gx = torch.empty_like(gy)
        gth = torch.empty_like(theta)
        st = lib.gft_givens_backward_noalloc(n, S, C.c_void_p(pairs.ctypes.data), C.c_void_p(theta.data_ptr()),
                                             C.c_void_p(y.data_ptr()), C.c_void_p(gy.data_ptr()),
                                             C.c_void_p(gx.data_ptr()), C.c_void_p(gth.data_ptr()), B, stream)
        assert st == 0, lib.gft_last_error()
        torch.cuda.synchronize()
        assert torch.equal(gx, gx_ref)
        err = float(torch.linalg.norm(gth - gth_ref) / torch.linalg.norm(gth_ref))
        assert err <= GRAD_TOL, err
    # batch = 0: the pair table is copied and gtheta is zeroed (filled with
    # garbage first so that a skipped clear shows)
    gth.fill_(7.0)
    st = lib.gft_givens_backward_noalloc(n, S, C.c_void_p(pairs.ctypes.data), C.c_void_p(theta.data_ptr()),
                                         C.c_void_p(y.data_ptr()), C.c_void_p(gy.data_ptr()),
                                         C.c_void_p(gx.data_ptr()), C.c_void_p(gth.data_ptr()), 0, stream)
    assert st == 0, lib.gft_last_error()
    torch.cuda.synchronize()
    assert torch.count_nonzero(gth).item() == 0
    # a network that is not a perfect matching is rejected before any launch
    bad = _xor_pairs(16, 8)
    bad[0, 0] = bad[0, 1]
    st = lib.gft_givens_backward_noalloc(16, 8, C.c_void_p(bad.ctypes.data), C.c_void_p(theta.data_ptr()),
                                         C.c_void_p(y.data_ptr()), C.c_void_p(gy.data_ptr()),
                                         C.c_void_p(gx.data_ptr()), C.c_void_p(gth.data_ptr()), 777, stream)
    assert st == 1
