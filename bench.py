"""Benchmark of the batched fast GFT on GB300.

Workload (default): the 25-joint skeleton graph (spine 0-4, arms and legs of
5 joints, left/right involution), 2^20 FP32 signals drawn i.i.d. N(0,1) --
one Haar stage and leaf blocks of 15, 5 and 5 nodes.  A step is one forward
fast GFT of the whole batch (Haar stage, leaf products, output permutation:
one kernel launch).  Metric: coefficients per second (batch * n per step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank transforms its own batch (independent problems:
weak scaling, no collective on the data path); the time is the max over
ranks.  `--impl reference` times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gft_workloads as W  # noqa: E402

WORKLOAD = "skeleton25_2^20_fp32"
METRIC = "fast-GFT coeffs/s vs dense GFT, same GB300, at stated err vs FP64; %HBM roof"
UNIT = "coeffs/s"
L2_BYTES = 129 * 1024 * 1024


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_hash(plan):
    """Hash of the CUDA source of the plan-specialised kernel module that the
    timed step launches (the text NVRTC compiles)."""
    return hashlib.sha256(plan.kernel_source().encode()).hexdigest()[:16]


def _traffic_from_profile(kernel_hash):
    """DRAM bytes per launch from the committed ncu summary of the forward
    kernel, if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "skeleton25_fwd_2e20.md")
    vals = {}
    try:
        with open(path) as fh:
            for line in fh:
                if ":" in line and line.strip().startswith("- "):
                    k, v = line.strip()[2:].split(":", 1)
                    vals[k.strip()] = v.strip().strip("`")
        if vals.get("kernel_hash") == kernel_hash:
            return int(vals["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (spawned process: no fork after CUDA initialisation)
# ---------------------------------------------------------------------------
def _oracle_worker(batch, seconds, q):
    from oracle import gft as ogft
    from oracle import graph as ograph
    (g, _, seed), = W.config2()
    f = ogft.fast_gft(ograph.laplacian(g.W, g.s), g.phis, split_components=True)
    x = W.signals(batch, g.n, seed).astype(np.float64)
    reps, t0 = 0, time.perf_counter()
    while True:
        ogft.forward_staged(f, x)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    q.put((reps * batch * g.n / el, reps, el))


def oracle_rate(batch, seconds):
    cores = os.cpu_count() or 1
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = str(cores)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_oracle_worker, args=(batch, seconds, q))
    p.start()
    rate, reps, el = q.get()
    p.join()
    return rate, reps, el, cores


# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    batch = 1 << 18
    rates = []
    for _ in range(args.warmup):
        oracle_rate(batch, 0.5)
    for _ in range(args.steps):
        r, _, _, cores = oracle_rate(batch, 2.0)
        rates.append(r)
    value = statistics.median(rates)
    cores = os.cpu_count() or 1
    sample = f"oracle.forward_staged (FP64 numpy) on 2^18 of the 2^20 signals, repeated for 2 s per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "graph": "skeleton25", "signals": 1 << 20, "n": 25},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _timed(torch, fn, reps=10):
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps / 1e3


def _rel(a, b):
    return float((a - b).norm() / b.norm())


def extras(torch, gft, dev):
    """Context numbers after the timed region (each kernel timed with CUDA
    events, 3 warm-up + 10 timed launches, inputs larger than L2 unless
    stated).  Errors are relative L2 against the plan's FP64 basis applied in
    FP64 on the GPU to the first 2048 signals."""
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    # ---- config 1: path N=8, FP64 and FP32, 4096 signals (launch-bound) and 2^26 coefficients
    (g, batch, seed), = W.config1()
    plan = gft.Plan(gft.laplacian(g.W, g.s), g.phis)
    U = torch.from_numpy(plan.basis()).to(dev)
    c1 = {}
    for nb, tag in ((batch, "4096_signals"), ((1 << 26) // 8, "2^26_coeffs")):
        x = torch.from_numpy(W.signals(nb, 8, seed)).to(dev)
        ref = x[:2048].double() @ U
        row = {}
        for dt, xx in (("fp32", x), ("fp64", x.double())):
            y = torch.empty_like(xx)
            t = _timed(torch, lambda: plan.forward(xx, out=y))
            row[dt] = {"gcoeffs_s": round(nb * 8 / t / 1e9, 2),
                       "err_vs_fp64": float(f"{_rel(plan.forward(xx[:2048].contiguous()).double(), ref):.2e}")}
        yd = torch.empty_like(x)
        t = _timed(torch, lambda: torch.matmul(x, U.float(), out=yd))
        row["dense_fp32_gcoeffs_s"] = round(nb * 8 / t / 1e9, 2)
        c1[tag] = row
    c1["note"] = "4096 signals = 128 KiB: launch-bound and L2-resident"
    out["config1_path8"] = c1
    # ---- config 3 kinds alone, 2^26 coefficients each (256 MiB in: > L2)
    kinds = {}
    for k, (g, _, seed) in enumerate(W.config3()):
        batch = (1 << 26) // g.n
        plan = gft.Plan(gft.laplacian(g.W, g.s), g.phis)
        x = torch.from_numpy(W.signals(batch, g.n, seed)).to(dev)
        y = torch.empty_like(x)
        U = torch.from_numpy(plan.basis()).to(dev)
        ref = x[:2048].double() @ U
        inf = plan.info
        row = {"n": g.n, "signals": batch, "max_leaf": inf["max_leaf"],
               "fp32_kernel": "plan-specialised" if inf["jit"] else ("wide-leaf" if inf["wide"] else "table-driven")}
        coeffs = batch * g.n
        for prec in ("fp32", "bf16", "bf16x3", "fp16x3"):
            try:
                t = _timed(torch, lambda: plan.forward(x, out=y, precision=prec))
                err = _rel(plan.forward(x[:2048].contiguous(), precision=prec).double(), ref)
                row[prec] = {"gcoeffs_s": round(coeffs / t / 1e9, 1), "err_vs_fp64": float(f"{err:.2e}")}
            except gft.GftError:
                row[prec] = "unsupported"
        Uf = U.float()
        t = _timed(torch, lambda: torch.matmul(x, Uf, out=y))
        row["dense_fp32_gcoeffs_s"] = round(coeffs / t / 1e9, 1)
        xb, Ub = x.bfloat16(), Uf.bfloat16()
        t = _timed(torch, lambda: torch.matmul(xb, Ub))
        row["dense_bf16_gcoeffs_s"] = round(coeffs / t / 1e9, 1)
        kinds[g.name] = row
        del x, y, U
    out["config3_kinds_2^26"] = kinds
    # ---- config 3 as specified: eight kinds x 2^23 coefficients in ONE graph launch
    sel = W.config3()
    plans = [gft.Plan(gft.laplacian(g.W, g.s), g.phis) for g, _, _ in sel]
    xs = [torch.from_numpy(W.signals(b, g.n, s)).to(dev) for g, b, s in sel]
    ys = [torch.empty_like(v) for v in xs]
    tot = sum(b * g.n for g, b, _ in sel)
    mixed = {"coeffs": tot, "graph_launches_per_step": 1}
    for prec in ("fp32", "bf16", "bf16x3"):
        bat = gft.Batch(plans, [b for _, b, _ in sel], precision=prec)
        t = _timed(torch, lambda: bat.forward(xs, ys))
        mixed[prec] = {"gcoeffs_s": round(tot / t / 1e9, 1), "ms": round(t * 1e3, 3)}
        del bat
    out["config3_mixed_one_graph"] = mixed
    del xs, ys, plans
    # ---- the paper's runtime table (Sec. VI-A): fast vs matrix GFT on the same graphs
    out["paper_runtime_table"] = runtime_table_extras(torch, gft, dev)
    # ---- right Haar stage (Sec. III-A): bipartite plans vs the matrix GFT
    out["right_haar_bipartite"] = right_haar_extras(torch, gft, dev)
    # ---- Sec. VI-B: approximate GFTs (greedy Jacobi layers) with and without the Haar stages
    out["approx_vs_exact"] = approx_extras(torch, gft, dev)
    # ---- config 4: learned Givens surrogates on the nine nearly symmetric graphs
    out["config4_learned"] = learned_extras(torch, gft, dev)
    torch.backends.cuda.matmul.allow_tf32 = prev
    return out


def runtime_table_extras(torch, gft, dev):
    """The graphs of the paper's runtime table: operation counts (ours, from
    the plan; printed, from the paper) and the runtime reduction of the fast
    GFT over the matrix GFT (torch.matmul FP32, TF32 off) on the same GB300 --
    on the paper's workload (20000 i.i.d. U[0,1] signals: launch-bound here)
    and on 2^26 coefficients (above L2)."""
    res = {}
    for g, split, printed in W.runtime_table_graphs():
        plan = gft.Plan(gft.laplacian(g.W, g.s), g.phis, split_components=split)
        inf = plan.info
        U = torch.from_numpy(plan.basis()).float().to(dev)
        row = {"n": g.n, "leaves": [len(l) for l in plan.leaves()], "fast_adds": inf["fast_adds"],
               "fast_mults": inf["fast_mults"], "printed_fast_adds_mults": list(printed[2:4]),
               "printed_reduction": printed[4]}
        for tag, nb in (("paper_20000", 20000), ("2^26", (1 << 26) // g.n)):
            x = torch.from_numpy(W.signals(nb, g.n, 7, dist="uniform")).to(dev)
            y = torch.empty_like(x)
            t_f = _timed(torch, lambda: plan.forward(x, out=y))
            t_d = _timed(torch, lambda: torch.matmul(x, U, out=y))
            row[tag] = {"fast_gcoeffs_s": round(nb * g.n / t_f / 1e9, 2),
                        "dense_gcoeffs_s": round(nb * g.n / t_d / 1e9, 2),
                        "reduction": round(1.0 - t_f / t_d, 3)}
        res[g.name] = row
    return res


def right_haar_extras(torch, gft, dev):
    """Bipartite plans with a right Haar stage (Sec. III-A): k-regular
    bipartite graphs (combinatorial Laplacian) and random bipartite graphs
    (normalised Laplacian), 2^26 coefficients each; the fast FP32 transform
    (kernel as chosen by the plan) against the matrix GFT (torch.matmul
    FP32) on the same basis, and the error against the FP64 basis."""
    res = {}
    cases = [(W.krbg(32, 5, seed=2105), False), (W.random_bipartite(40, 24, 0.15, seed=2301), True),
             (W.krbg(64, 6, seed=2302), False), (W.krbg(256, 8, seed=2201), False),
             (W.random_bipartite(300, 212, 0.05, seed=2202), True)]
    for g, normalised in cases:
        L = gft.normalized_laplacian(g.W, g.s) if normalised else gft.laplacian(g.W, g.s)
        plan = gft.Plan.bipartite(L, g.meta["side"])
        inf = plan.info
        U = torch.from_numpy(plan.basis()).to(dev)
        nb = (1 << 26) // g.n
        x = torch.from_numpy(W.signals(nb, g.n, 9)).to(dev)
        y = torch.empty_like(x)
        t_f = _timed(torch, lambda: plan.forward(x, out=y))
        t_i = _timed(torch, lambda: plan.inverse(x, out=y))
        Uf = U.float()
        t_d = _timed(torch, lambda: torch.matmul(x, Uf, out=y))
        ref = x[:2048].double() @ U
        res[g.name] = {"n": g.n, "parts": [len(v) for v in plan.leaves()], "right_pairs": inf["right_pairs"],
                       "laplacian": "normalised" if normalised else "combinatorial",
                       "fp32_kernel": "plan-specialised" if inf["jit"] else ("wide-leaf" if inf["wide"] else "table-driven"),
                       "fast_mults": inf["fast_mults"], "dense_mults": g.n * g.n,
                       "fast_gcoeffs_s": round(nb * g.n / t_f / 1e9, 1),
                       "inverse_gcoeffs_s": round(nb * g.n / t_i / 1e9, 1),
                       "dense_gcoeffs_s": round(nb * g.n / t_d / 1e9, 1),
                       "err_vs_fp64": float(f"{_rel(plan.forward(x[:2048].contiguous()).double(), ref):.2e}")}
    return res


def approx_extras(torch, gft, dev):
    """The comparison of Sec. VI-B on its two graphs (8x8 bi-diagonal grid,
    a = 0.5; 8x8 z-shaped grid, w = 2): matrix GFT, Haar + matrix GFT (the
    exact fast plan), approximate GFT and Haar + approximate GFT with J
    Givens layers.  Per implementation: the sign-normalised error delta and
    the empirical error epsilon against the exact GFT (2000 U[0,1] signals,
    FP64 on the host from the FP64 bases), and G coeff/s on the paper's
    20000 signals and on 2^26 coefficients."""
    res = {}
    for g in (W.grid6_bidiag(8), W.zgrid(8)):
        n = g.n
        L = gft.laplacian(g.W, g.s)
        exact = gft.Plan(L, g.phis)
        dense = gft.Plan(L, [], jit=False)
        U = dense.basis()
        Uf = torch.from_numpy(U).float().to(dev)
        xe = W.signals(2000, n, 77, dist="uniform").astype(np.float64)
        ye = np.abs(xe @ U)

        def errs(Uh):
            d = float(np.linalg.norm(np.abs(Uh.T @ U) - np.eye(n)) / np.sqrt(n))
            e = float(np.mean(np.sum((ye - np.abs(xe @ Uh)) ** 2, axis=1)))
            return round(d, 4), float(f"{e:.3e}")

        def speeds(fn):
            out = {}
            for tag, nb in (("paper_20000", 20000), ("2^26", (1 << 26) // n)):
                x = torch.from_numpy(W.signals(nb, n, 7, dist="uniform")).to(dev)
                y = torch.empty_like(x)
                out[tag] = round(nb * n / _timed(torch, lambda: fn(x, y)) / 1e9, 1)
            return out
        rows = {"matrix": {"delta": 0.0, "epsilon": 0.0,
                           "gcoeffs_s": speeds(lambda x, y: torch.matmul(x, Uf, out=y))},
                "haar_matrix": {"delta": errs(exact.basis())[0], "epsilon": errs(exact.basis())[1],
                                "gcoeffs_s": speeds(lambda x, y: exact.forward(x, out=y))}}
        for J in (0, 5, 10, 20, 30, 40):
            for tag, phis in (("approx", []), ("haar_approx", g.phis)):
                a = gft.ApproxGFT(L, phis, J)
                d, e = errs(a.basis())
                inf = a.info
                rows[f"{tag}_J{J}"] = {"delta": d, "epsilon": e, "layers": inf["n_layers"], "units": inf["n_units"],
                                       "gcoeffs_s": speeds(lambda x, y: a.forward(x, out=y))}
        res[g.name] = rows
    return res


def learned_extras(torch, gft, dev, steps=1500):
    """Per nearly symmetric graph: the surrogate trained on the GPU against
    the exact basis, its sign-normalised error delta (Sec. VI-B) before and
    after training, the error of the method without it (the exact butterfly
    of the graph with its weights symmetrised under the involutions), and
    coefficients/s of the surrogate, the exact dense GFT and that butterfly
    on 2^24 coefficients."""
    from paper_1907_07875_gb300.learned import LearnedGFT, delta
    res = {}
    for g in W.config4():
        n = g.n
        phis = [W.grid_lr(int(round(n ** 0.5))), W.grid_ud(int(round(n ** 0.5)))] if "grid" in g.name \
            else [W.reversal(n)]
        Ws = g.W.copy()
        for _ in range(2):
            for ph in phis:
                Ws = 0.5 * (Ws + Ws[np.ix_(ph, ph)])
        exact = gft.Plan(gft.laplacian(g.W, g.s), [])
        sym = gft.Plan(gft.laplacian(Ws, g.s), phis)
        U = exact.basis()
        model = LearnedGFT(n, device=dev)
        d0 = delta(model.matrix(), U)
        model.train(U, steps=steps, lr=0.05)
        d1 = delta(model.matrix(), U)
        nb = (1 << 24) // n
        x = torch.from_numpy(W.signals(nb, n, 5)).to(dev)
        y = torch.empty_like(x)
        t_l = _timed(torch, lambda: model.forward(x, out=y))
        t_e = _timed(torch, lambda: exact.forward(x, out=y))
        t_s = _timed(torch, lambda: sym.forward(x, out=y))
        res[g.name] = {"delta_untrained": round(d0, 4), "delta_learned": round(d1, 4),
                       "delta_symmetrised_butterfly": round(delta(sym.basis(), U), 4),
                       "learned_gcoeffs_s": round((1 << 24) / t_l / 1e9, 1),
                       "exact_dense_gcoeffs_s": round((1 << 24) / t_e / 1e9, 1),
                       "symmetrised_butterfly_gcoeffs_s": round((1 << 24) / t_s / 1e9, 1)}
    return res


def sweep(torch, gft, dev, precisions=("fp32", "bf16x3"), n_graphs=10000, total=1 << 28, reps=5):
    """Config-5 size sweep: 10^4 graphs (path, cycle, grid, skeleton,
    bipartite; n = 8..1024 log-uniform), 2^28 FP32 coefficients, in one graph
    launch per precision; plans built in one batched call, identical graphs
    share a plan.  Dense baseline: torch.bmm of each size class against its
    graphs' FP32 bases (TF32 off)."""
    import collections
    t0 = time.perf_counter()
    specs = W.config5_specs(n_graphs=n_graphs, total_coeffs=total)
    keys, graphs = {}, []
    for fam, n, gs, b, ss in specs:
        if (fam, n, gs) not in keys:
            keys[(fam, n, gs)] = len(graphs)
            graphs.append((fam, n, gs))
    Ls, phis = [], []
    for fam, n, gs in graphs:
        g = W.make_graph(fam, n, gs)
        Ls.append(gft.laplacian(g.W, g.s))
        phis.append(g.phis)
    t1 = time.perf_counter()
    plans = gft.plans_from_laplacians(Ls, phis, jit=False)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del Ls
    entry = [keys[(f, n, gs)] for f, n, gs, b, ss in specs]
    batches = [b for f, n, gs, b, ss in specs]
    ns = [n for f, n, gs, b, ss in specs]
    # one input and one output buffer; entry views start 16-byte aligned
    offs, o = [], 0
    for b, n in zip(batches, ns):
        offs.append(o)
        o += (b * n + 3) & ~3
    X = torch.randn(o, device=dev)
    Y = torch.empty(o, device=dev)
    xs = [X[a:a + b * n].view(b, n) for a, b, n in zip(offs, batches, ns)]
    ys = [Y[a:a + b * n].view(b, n) for a, b, n in zip(offs, batches, ns)]
    coeffs = sum(b * n for b, n in zip(batches, ns))
    out = {"graphs": len(specs), "distinct_plans": len(graphs), "coeffs": coeffs,
           "build_graphs_s": round(t1 - t0, 1), "build_plans_s": round(t2 - t1, 1)}
    for prec in precisions:
        t3 = time.perf_counter()
        bt = gft.Batch([plans[i] for i in entry], batches, precision=prec)
        bt.forward(xs, ys)
        torch.cuda.synchronize()
        t4 = time.perf_counter()
        t = _timed(torch, lambda: bt.forward(xs, ys), reps=reps)
        out[prec] = {"gcoeffs_s": round(coeffs / t / 1e9, 1), "ms": round(t * 1e3, 2),
                     "batch_create_s": round(t4 - t3, 1)}
        del bt
    # dense baseline: grouped by size
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    by_n = collections.defaultdict(list)
    for j, n in enumerate(ns):
        by_n[n].append(j)
    groups, basis = [], {}
    for n, js in by_n.items():
        for j in js:
            if entry[j] not in basis:
                basis[entry[j]] = torch.from_numpy(plans[entry[j]].basis()).float().to(dev)
        U = torch.stack([basis[entry[j]] for j in js])
        Xg = torch.stack([xs[j] for j in js])
        groups.append((Xg, U, torch.empty_like(Xg)))
    t = _timed(torch, lambda: [torch.bmm(a, u, out=c) for a, u, c in groups], reps=reps)
    out["dense_bmm_fp32"] = {"gcoeffs_s": round(coeffs / t / 1e9, 1), "ms": round(t * 1e3, 2),
                             "size_classes": len(groups)}
    torch.backends.cuda.matmul.allow_tf32 = prev
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1907_07875_gb300 as gft
    from paper_1907_07875_gb300 import sharding
    from paper_1907_07875_gb300.build import build
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if rank == 0 or world == 1:
        build()
    if dist is not None:
        dist.barrier()
    (g, batch, seed), = W.config2()
    n = g.n
    plan = gft.Plan(gft.laplacian(g.W, g.s), g.phis, split_components=True)
    stream = torch.cuda.current_stream()
    # rotating input/output sets, together larger than L2, so every step reads
    # its input from HBM
    x_host = W.signals(batch, n, sharding.rank_seed(seed, rank))
    nbytes = batch * n * 4
    nsets = 2 if args.profile else max(2, -(-4 * L2_BYTES // (2 * nbytes)))
    xs = [torch.from_numpy(x_host).to(dev) for _ in range(nsets)]
    for i in range(1, nsets):
        xs[i].mul_(1.0 + 1e-3 * i)
    ys = [torch.empty_like(xs[0]) for _ in range(nsets)]

    # parity spot check against the FP64 oracle (rank 0, 2^14 signals)
    err = None
    if rank == 0 and not args.profile:
        from oracle import gft as ogft
        from oracle import graph as ograph
        ref = ogft.fast_gft(ograph.laplacian(g.W, g.s), g.phis, split_components=True)
        U = plan.basis()
        k = 1 << 14
        y = plan.forward(xs[0][:k].contiguous()).cpu().numpy().astype(np.float64)
        yo = ogft.forward_dense(ref.U, x_host[:k].astype(np.float64))
        lam = ref.lam
        tol = 1e-9 * max(1.0, float(np.abs(lam).max()))
        ya, start = np.empty_like(yo), 0
        for j in range(1, n + 1):
            if j == n or lam[j] - lam[j - 1] > tol:
                S = list(range(start, j))
                ya[:, S] = yo[:, S] @ (U[:, S].T @ ref.U[:, S]).T
                start = j
        err = float(np.linalg.norm(y - ya) / np.linalg.norm(ya))

    def step(i):
        plan.forward(xs[i % nsets], out=ys[i % nsets], stream=stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    # per-launch durations: events around a sample of about 256 launches
    # spread over the timed region (an event pair around every launch would
    # put its own gap between consecutive kernels)
    every = max(1, args.steps // 256)
    sampled = list(range(0, args.steps, every))
    starts = {i: torch.cuda.Event(enable_timing=True) for i in sampled}
    ends = {i: torch.cuda.Event(enable_timing=True) for i in sampled}
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            if i in starts:
                starts[i].record(stream)
                step(i)
                ends[i].record(stream)
            else:
                step(i)
        t1.record(stream)
        torch.cuda.synchronize()
        total_ms = t0.elapsed_time(t1)
    launch_ms = [starts[i].elapsed_time(ends[i]) for i in sampled]
    if args.profile:
        if rank == 0:
            inf = plan.info
            print(json.dumps({"profile_run": True, "ms_per_step": total_ms / args.steps,
                              "kernel_hash": _kernel_hash(plan), "tile_signals": inf["tile_signals"],
                              "threads": inf["threads"], "jit": inf["jit"],
                              "config": {"workload": WORKLOAD, "sets": nsets}}), flush=True)
        return
    total_ms = sharding.max_over_ranks(total_ms, dist, dev)
    ms_per_step = total_ms / args.steps
    coeffs_per_step = batch * n
    value = coeffs_per_step * world / (total_ms / 1e3) * args.steps

    # dominant (only) kernel: the fused transform, one launch per step
    avg_launch_s = statistics.mean(launch_ms) / 1e3
    alg_bytes = 8 * coeffs_per_step          # FP32 read + write per coefficient
    peak, peak_kind = _peaks()
    achieved = alg_bytes / avg_launch_s / 1e9
    khash = _kernel_hash(plan)
    traffic = _traffic_from_profile(khash)

    # inverse and the dense GEMM on the same data (context)
    def timed(fn, reps=20):
        for i in range(3):
            fn(i)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(reps):
            fn(i)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps / 1e3

    inv_s = timed(lambda i: plan.inverse(ys[i % nsets], out=xs[(i + 1) % nsets], stream=stream))
    Ut = torch.from_numpy(plan.basis()).float().to(dev)
    prev_tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    dense_s = timed(lambda i: torch.matmul(xs[i % nsets], Ut, out=ys[i % nsets]))
    torch.backends.cuda.matmul.allow_tf32 = prev_tf32

    # end to end through the public API with host buffers (pinned)
    xh = torch.from_numpy(x_host).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    plan.forward_host(xh, out=yh)
    e2e_steps = max(3, min(args.steps, 20))
    t = time.perf_counter()
    for _ in range(e2e_steps):
        plan.forward_host(xh, out=yh)
    e2e_s = (time.perf_counter() - t) / e2e_steps

    if dist is not None:
        dist.barrier()
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rate, reps, el, cores = oracle_rate(1 << 18, 10.0)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"oracle.forward_staged (FP64 numpy) on 2^18 of the 2^20 signals x {reps} reps "
                         f"({el:.1f} s)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "graph": "skeleton25 (1 Haar stage, leaves 15/5/5)",
                   "signals_per_gpu": batch, "n": n, "precision": "fp32",
                   "l2": f"{nsets} rotating input/output sets ({nsets * 2 * nbytes / 2**20:.0f} MiB) > L2"},
        "err_vs_fp64": err,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                     "alg_bytes_per_launch": alg_bytes, "launches_timed": len(launch_ms),
                     "kernel": "gft_jit_fwd_* (plan-specialised)" if plan.info["jit"] else "gft_apply_kernel"},
        "e2e": {"value": coeffs_per_step / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": args.steps,
        "inverse": {"value": coeffs_per_step / inv_s, "unit": UNIT},
        "dense_gemm_fp32": {"value": coeffs_per_step / dense_s, "unit": UNIT,
                            "what": "torch.matmul(x, U) FP32, TF32 off"},
        "clocks": clk.summary(),
        "kernel_hash": khash,
        "cpu_baseline": cpu,
    }
    if not args.no_extras and world == 1:
        line["extras"] = extras(torch, gft, dev)
        if not args.no_sweep:
            line["extras"]["config5_sweep"] = sweep(torch, gft, dev)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_probe(args):
    """ncu capture helper: one plan (or Givens network), three forward calls
    of 2^25 coefficients, nothing timed.  Used by the commands recorded in
    profiles/."""
    import torch
    import paper_1907_07875_gb300 as gft
    from paper_1907_07875_gb300.build import build
    build()
    dev = torch.device("cuda", 0)
    if args.probe.startswith("givens"):
        import math
        from paper_1907_07875_gb300.learned import xor_pairs
        n = int(args.probe[len("givens"):])
        S = 2 * int(math.log2(n))
        net = gft.Givens(n, xor_pairs(n, S))
        th = torch.rand(S, n // 2, device=dev)
        x = torch.from_numpy(W.signals((1 << 25) // n, n, 1)).to(dev)
        y = torch.empty_like(x)
        for _ in range(3):
            net.forward(th, x, out=y)
    else:
        g = {"skeleton25": W.skeleton25(), "grid16": W.grid(16), "grid32": W.grid(32), "cycle256": W.cycle(256),
             "grid8": W.grid(8)}[args.probe]
        plan = gft.Plan(gft.laplacian(g.W, g.s), g.phis, kernel=args.kernel)
        x = torch.from_numpy(W.signals((1 << 25) // g.n, g.n, 1)).to(dev)
        y = torch.empty_like(x)
        for _ in range(3):
            plan.forward(x, out=y, precision=args.precision)
    torch.cuda.synchronize()
    print(json.dumps({"probe": args.probe, "precision": args.precision, "kernel": args.kernel}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the context measurements")
    ap.add_argument("--no-sweep", action="store_true", help="skip the 10^4-graph size sweep in the extras")
    ap.add_argument("--probe", choices=["skeleton25", "grid8", "grid16", "grid32", "cycle256", "givens16", "givens64"],
                    help="ncu capture helper: one plan, three forwards of 2^25 coefficients, nothing timed")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "bf16x3", "fp16x3"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "table", "wide"])
    ap.add_argument("--profile", action="store_true",
                    help="forward steps only, 2 buffer sets (for ncu captures)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if args.probe:
        run_probe(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
