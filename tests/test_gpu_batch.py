"""Mixed batches: one persistent, graph-captured launch over many plans.
Every plan's output must equal its own single-plan forward bit for bit (the
batch kernel runs the same FMA sequence), and the single-plan forward is
pinned to the oracle by test_gpu_parity."""
import numpy as np
import pytest

import gft_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_1907_07875_gb300.build import build
    build()
    import paper_1907_07875_gb300 as gft
    return gft, torch


def _plans(gft, graphs, split=False):
    # the table-driven kernel runs the batch kernel's FMA sequence
    return [gft.Plan(gft.laplacian(g.W, g.s), g.phis, split_components=split, jit=False, kernel="table")
            for g in graphs]


def test_config3_core_kinds_in_one_launch(env):
    gft, torch = env
    kinds = [W.config3(coeffs_per_kind=1 << 18)[k] for k in (0, 1, 2, 3, 6, 7)]
    graphs = [k[0] for k in kinds]
    batches = [k[1] + 13 for k in kinds]            # ragged tails
    plans = _plans(gft, graphs)
    b = gft.Batch(plans, batches)
    xs = [torch.from_numpy(W.signals(bt, g.n, 100 + i)).cuda() for i, (g, bt) in enumerate(zip(graphs, batches))]
    ys = [torch.empty_like(x) for x in xs]
    for rep in range(3):                               # capture, then replays
        b.forward(xs, ys)
    torch.cuda.synchronize()
    for p, x, y in zip(plans, xs, ys):
        assert torch.equal(y, p.forward(x))
    for p, i in zip(plans, range(len(plans))):
        tile, threads = b.tile(i)
        if p.n <= 256:        # node-major kernel: a power-of-two tile
            assert threads == 256 and tile in (16, 32, 64, 128, 256, 512, 1024)
        else:                 # thread-per-signal kernel (autotuned tile) or wide-leaf kernel
            assert (threads, tile) == (0, 0) or (threads == 128 and tile in (128, 256, 512))


def test_pointer_change_reuses_graph(env):
    gft, torch = env
    graphs = [W.skeleton25(), W.path(8), W.cycle(12)]
    plans = _plans(gft, graphs)
    batches = [1000, 5000, 333]
    b = gft.Batch(plans, batches)
    for seed in (1, 2):
        xs = [torch.from_numpy(W.signals(bt, g.n, seed * 10 + i)).cuda() for i, (g, bt) in enumerate(zip(graphs, batches))]
        ys = [torch.full_like(x, float("nan")) for x in xs]
        b.forward(xs, ys)
        torch.cuda.synchronize()
        for p, x, y in zip(plans, xs, ys):
            assert torch.equal(y, p.forward(x))


def test_many_small_graphs_and_empty_batches(env):
    """A sweep-like batch: 120 graphs of 6..64 nodes from every family."""
    gft, torch = env
    rng = np.random.default_rng(5)
    graphs = []
    for i in range(120):
        fam = i % 5
        n = int(rng.integers(6, 65))
        if fam == 0:
            graphs.append(W.path(n))
        elif fam == 1:
            graphs.append(W.cycle(max(4, n - n % 4)))
        elif fam == 2:
            graphs.append(W.grid(max(2, int(np.sqrt(n)))))
        elif fam == 3:
            graphs.append(W.skeleton25())
        else:
            graphs.append(W.bipartite(max(8, min(64, n - n % 2)), 0.2, seed=int(rng.integers(1 << 30))))
    plans = _plans(gft, graphs)
    batches = [int(rng.integers(0, 700)) for _ in graphs]
    batches[3] = 0
    b = gft.Batch(plans, batches)
    xs = [torch.from_numpy(W.signals(max(bt, 1), g.n, i)).cuda()[:bt] for i, (g, bt) in enumerate(zip(graphs, batches))]
    ys = [torch.empty_like(x) for x in xs]
    b.forward(xs, ys)
    torch.cuda.synchronize()
    for p, x, y in zip(plans, xs, ys):
        if x.shape[0]:
            assert torch.equal(y, p.forward(x))


def test_batch_rejects_leaves_over_512(env):
    gft, torch = env
    g = W.path(1100)                                   # two leaves of 550 nodes
    p = gft.Plan(gft.laplacian(g.W, g.s), g.phis)
    with pytest.raises(gft.GftError) as e:
        gft.Batch([p], [10])
    assert e.value.status == "GFT_ERR_UNSUPPORTED"


TC_BOUNDS = {"bf16": 5e-3, "bf16x3": 1e-5, "fp16x3": 2e-6}


def _check_tc_entry(p, x, y, prec):
    """A tensor-core batch entry: plans whose leaves reach 64 nodes run on
    the tensor cores (the 128-signal kernel for large batches of leaves of
    64..256, else the signals-as-N kernel, whose sums are ordered
    differently), the others on CUDA cores bit for bit like their own FP32
    forward.  Tensor-core entries are held to the precision's bound against
    x U in FP64 with the plan's basis (oracle parity: test_gpu_batch_oracle)."""
    import torch
    if p.info["max_leaf"] < 64:
        assert torch.equal(y, p.forward(x))
        return
    ref = x.double().cpu().numpy() @ p.basis()
    got = y.double().cpu().numpy()
    err = float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))
    assert err <= TC_BOUNDS[prec], (p.n, prec, err)


def _config3_plans(gft, coeffs):
    kinds = W.config3(coeffs_per_kind=coeffs)
    graphs = [k[0] for k in kinds]
    batches = [k[1] + 5 for k in kinds]                # ragged tails
    plans = [gft.Plan(gft.laplacian(g.W, g.s), g.phis) for g in graphs]
    return graphs, batches, plans


def test_config3_all_kinds_fp32_one_graph(env):
    """All eight grid / cycle kinds of the mixed workload, grid32 (leaves of
    256) included, in one graph launch: table-driven and wide-leaf groups.
    Every output equals its plan's own forward bit for bit (same kernel code
    and tile shape), which the single-plan tests pin to the oracle."""
    gft, torch = env
    graphs, batches, plans = _config3_plans(gft, 1 << 18)
    b = gft.Batch(plans, batches)
    xs = [torch.from_numpy(W.signals(bt, g.n, 60 + i)).cuda() for i, (g, bt) in enumerate(zip(graphs, batches))]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    for _ in range(2):
        b.forward(xs, ys)
    torch.cuda.synchronize()
    for p, x, y in zip(plans, xs, ys):
        assert torch.equal(y, p.forward(x))
    assert any(p.info["wide"] for p in plans)


@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "fp16x3"])
def test_config3_tensor_core_precisions_one_graph(env, prec):
    """The mixed workload in a tensor-core precision: grids 16/32 and the
    256-cycle (leaves of 64 and 256) on the tensor cores, the rest on CUDA
    cores, in one graph launch; a plan appears twice (its two entries share
    its scratch and run in order).  Outputs are within the precision's bound
    of x U (FP64, the plan's basis); new pointers reuse the captured graph."""
    gft, torch = env
    graphs, batches, plans = _config3_plans(gft, 1 << 17)
    graphs.append(graphs[2])
    plans.append(plans[2])
    batches.append(300)
    b = gft.Batch(plans, batches, precision=prec)
    for rep in range(2):
        xs = [torch.from_numpy(W.signals(bt, g.n, 90 + 7 * rep + i)).cuda()
              for i, (g, bt) in enumerate(zip(graphs, batches))]
        ys = [torch.full_like(x, float("nan")) for x in xs]
        b.forward(xs, ys)
        b.forward(xs, ys)
        torch.cuda.synchronize()
        for p, x, y in zip(plans, xs, ys):
            _check_tc_entry(p, x, y, prec)


def test_create_many_matches_single_plans(env):
    """Plans built together (one batched Jacobi solve over all leaves, grouped
    by size) agree with plans built one at a time: same structure and output
    map, eigenvalues within 1e-12, eigenspace projectors within 1e-10."""
    from _helpers import projector_distance
    gft, torch = env
    graphs = [W.path(9), W.cycle(64), W.grid(8, weights="sym_uniform", seed=4), W.skeleton25(),
              W.bipartite(300, 0.1, seed=6), W.path(600), W.grid(12), W.cycle(8), W.bipartite(40, 0.3, seed=8)]
    many = gft.plans_from_laplacians([gft.laplacian(g.W, g.s) for g in graphs], [g.phis for g in graphs])
    for g, pm in zip(graphs, many):
        ps = gft.Plan(gft.laplacian(g.W, g.s), g.phis)
        assert pm.leaves() == ps.leaves()
        assert pm.output_map().tolist() == ps.output_map().tolist()
        lam = ps.eigenvalues()
        assert np.max(np.abs(pm.eigenvalues() - lam)) <= 1e-12 * max(1.0, np.abs(lam).max())
        assert projector_distance(pm.basis(), ps.basis(), lam) <= 1e-10


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_size_sweep_sample_one_graph(env, prec):
    """A 400-graph slice of the size sweep (families path, cycle, grid,
    skeleton, bipartite; sizes 8..1024; 2^22 coefficients), plans built in
    one call and shared between identical graphs, transformed in one graph
    launch; every output equals its plan's own forward bit for bit."""
    gft, torch = env
    specs = W.config5_specs(n_graphs=400, total_coeffs=1 << 22)
    keys, graphs = {}, []
    for fam, n, gs, b, ss in specs:
        if (fam, n, gs) not in keys:
            keys[(fam, n, gs)] = len(graphs)
            graphs.append(W.make_graph(fam, n, gs))
    plans = gft.plans_from_laplacians([gft.laplacian(g.W, g.s) for g in graphs], [g.phis for g in graphs],
                                      jit=False)
    entry_plans = [plans[keys[(f, n, gs)]] for f, n, gs, b, ss in specs]
    batches = [b for f, n, gs, b, ss in specs]
    bt = gft.Batch(entry_plans, batches, precision=prec)
    xs = [torch.from_numpy(W.signals(b, n, ss % 100000)).cuda() for f, n, gs, b, ss in specs]
    ys = [torch.empty_like(x) for x in xs]
    bt.forward(xs, ys)
    torch.cuda.synchronize()
    for p, x, y in zip(entry_plans, xs, ys):
        if prec == "fp32":
            assert torch.equal(y, p.forward(x))
        else:
            _check_tc_entry(p, x, y, prec)


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
def test_tensor_core_batch_with_odd_largest_graph(env, prec):
    """Tensor-core batch whose largest graph has n % 4 != 0 (a 257-node path,
    leaves of 129 and 128) beside graphs with n % 4 == 0 (16x16 grid, 256-
    cycle), whose rows are staged with 16-byte copies: the staging row stride
    must stay a multiple of four floats.  Outputs within the precision's
    bound."""
    gft, torch = env
    graphs = [W.path(257), W.grid(16), W.cycle(256), W.path(130)]
    plans = [gft.Plan(gft.laplacian(g.W, g.s), g.phis) for g in graphs]
    batches = [301, 517, 129, 260]
    b = gft.Batch(plans, batches, precision=prec)
    xs = [torch.from_numpy(W.signals(bt, g.n, 70 + i)).cuda() for i, (g, bt) in enumerate(zip(graphs, batches))]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    b.forward(xs, ys)
    torch.cuda.synchronize()
    for p, x, y in zip(plans, xs, ys):
        _check_tc_entry(p, x, y, prec)


def test_small_graph_batch_sizes_and_item_edges(env):
    """Small graphs in one batch: zero to two stages, batches on both sides of
    every tile size (128, 256, 512 signals) and of the cost-balanced CTA
    ranges, a single signal, an empty entry; outputs equal the table-driven
    single-plan forward bit for bit."""
    gft, torch = env
    graphs = [W.path(2), W.path(3), W.cycle(8), W.grid(4), W.path(16), W.path(17), W.grid(5, 3), W.cycle(32),
              W.bipartite(32, 0.3, seed=11), W.skeleton25(), W.star(9), W.complete(6)]
    plans = _plans(gft, graphs)
    batches = [1, 127, 128, 129, 511, 512, 513, 1537, 100, 4099, 33, 0]
    b = gft.Batch(plans, batches)
    xs = [torch.from_numpy(W.signals(max(bt, 1), g.n, 300 + i)).cuda()[:bt] for i, (g, bt) in
          enumerate(zip(graphs, batches))]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    b.bind(xs, ys).forward()
    torch.cuda.synchronize()
    for p, x, y in zip(plans, xs, ys):
        if x.shape[0]:
            assert torch.equal(y, p.forward(x)), p.n


def test_node_major_kernel_tiles_and_leaf_widths(env):
    """The node-major table-driven kernel: graphs of 2..256 nodes (tiles of
    1024 down to 16 signals), leaves from 1 to 64 nodes (widths that are not
    multiples of four included), zero to several Haar stages, batches on
    both sides of every tile size and a single signal, mixed with a plan
    that has right Haar units (thread-per-signal kernel) in one launch.
    Outputs equal the table-driven single-plan forward bit for bit (the same
    FMA chain per output)."""
    gft, torch = env
    graphs = [W.path(2), W.path(3), W.path(5), W.cycle(12), W.path(33), W.grid(6), W.path(70), W.cycle(100),
              W.path(128), W.grid(11), W.bipartite(90, 0.2, seed=3), W.skeleton25(), W.path(127), W.cycle(256),
              W.grid(14), W.path(130)]
    plans = _plans(gft, graphs)
    right = W.krbg(16, 3, seed=7)
    plans.append(gft.Plan.bipartite(gft.laplacian(right.W, right.s), right.meta["side"]))
    graphs.append(right)
    batches = [1025, 1024, 255, 1, 129, 128, 65, 64, 33, 31, 97, 1025, 2, 17, 16, 15, 300]
    b = gft.Batch(plans, batches)
    xs = [torch.from_numpy(W.signals(bt, g.n, 700 + i)).cuda() for i, (g, bt) in enumerate(zip(graphs, batches))]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    b.bind(xs, ys).forward()
    torch.cuda.synchronize()
    for p, x, y, i in zip(plans, xs, ys, range(len(plans))):
        assert torch.equal(y, p.forward(x)), (p.n, p.info["max_leaf"])
    tiles = [b.tile(i) for i in range(len(plans))]
    assert tiles[0] == (1024, 256) and tiles[8] == (32, 256) and tiles[13] == (16, 256)   # 2, 128, 256 nodes
    assert tiles[-1][1] != 256                                     # right Haar plan: not node-major
    b.forward()                                                    # replay: same bits
    torch.cuda.synchronize()
    for p, x, y in zip(plans, xs, ys):
        assert torch.equal(y, p.forward(x))


def test_plan_specialised_group_for_shared_small_plans(env):
    """Small plans shared by many entries (at least 2^19 coefficients per plan
    over its entries) run in the batch's plan-specialised group: one module
    with the straight-line forward of each such plan and one persistent
    kernel over all their (entry, tile) items.  Entries: eight skeletons,
    five cycles, a path, a grid of odd size, a right Haar plan (three
    entries), batches on both sides of the tile sizes; next to them a plan
    below the threshold (node-major kernel).  Every output equals the plan's
    own table-driven forward bit for bit, with the group and without it."""
    gft, torch = env
    sk, cy, pa, gr = W.skeleton25(), W.cycle(16), W.path(40), W.grid(7)
    rb = W.krbg(16, 3, seed=9)
    p_sk, p_cy, p_pa, p_gr, p_small = _plans(gft, [sk, cy, pa, gr, W.path(12)])
    p_rb = gft.Plan.bipartite(gft.laplacian(rb.W, rb.s), rb.meta["side"])
    entries = [(p_sk, sk.n, b) for b in (6000, 5999, 6001, 256, 257, 4096, 8000, 1)]      # 778 K coefficients
    entries += [(p_cy, cy.n, b) for b in (14000, 13999, 14001, 511, 512)]                # 704 K
    entries += [(p_pa, pa.n, 14000), (p_gr, gr.n, 11000), (p_small, 12, 300)]
    entries += [(p_rb, rb.n, b) for b in (6000, 6001, 5999)]
    plans = [e[0] for e in entries]
    xs = [torch.from_numpy(W.signals(b, n, 900 + i)).cuda() for i, (_, n, b) in enumerate(entries)]
    outs = {}
    for jit in (True, False):
        bt = gft.Batch(plans, [e[2] for e in entries], jit=jit)
        ys = [torch.full_like(x, float("nan")) for x in xs]
        bt.bind(xs, ys).forward()
        bt.forward()
        torch.cuda.synchronize()
        for p, x, y in zip(plans, xs, ys):
            assert torch.equal(y, p.forward(x)), (p.n, jit)
        outs[jit] = ys
        tiles = [bt.tile(i) for i in range(len(plans))]
        group = [t[1] == 128 and t[0] in (128, 256, 512) for t in tiles]
        if jit:
            assert all(group[:-4]) and all(group[-3:])     # the group, right Haar plan included
            assert tiles[-4][1] == 256                      # below the threshold: node-major kernel
        else:
            assert all(t[1] == 256 for t in tiles[:-3])     # node-major kernel
    assert all(torch.equal(a, b) for a, b in zip(outs[True], outs[False]))
