"""GB300-native batched fast graph Fourier transform (Lu & Ortega, "Fast
Graph Fourier Transforms Based on Graph Symmetry and Bipartition").

Thin Python binding over the C-ABI library ``libgft.so`` (include/gft.h).
PyTorch supplies device memory and streams; every step of a transform runs
in the library's CUDA kernels, and a missing library raises instead of
falling back to anything else.

    import numpy as np, torch, paper_1907_07875_gb300 as gft
    L = gft.laplacian(W, s)                       # Eq. 5
    plan = gft.Plan(L, [phi], split_components=True)
    y = plan.forward(x)                           # x: cuda float32 [batch, n]
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import _native

SPLIT_COMPONENTS = 0x1
ORDER_BLOCK = 0x2
ANALYZE_ONLY = 0x4
NO_JIT = 0x8
KERNEL_TABLE = 0x10
KERNEL_WIDE = 0x20
SEARCH_STAGES = 0x40
NORMALIZED = 0x80
PRECISIONS = {"fp32": 0, "bf16": 1, "bf16x3": 2, "fp16x3": 3}

STATUS = {0: "GFT_OK", 1: "GFT_ERR_INVALID_ARG", 2: "GFT_ERR_NOT_INVOLUTION", 3: "GFT_ERR_NOT_SYMMETRIC",
          4: "GFT_ERR_NOT_LAPLACIAN", 5: "GFT_ERR_NO_CONVERGENCE", 6: "GFT_ERR_CUDA", 7: "GFT_ERR_OOM",
          8: "GFT_ERR_TIMEOUT", 9: "GFT_ERR_UNSUPPORTED", 10: "GFT_ERR_MISALIGNED", 11: "GFT_ERR_BLOCK_LEAK",
          12: "GFT_ERR_NO_DEVICE", 13: "GFT_ERR_NOT_BIPARTITE"}


class GftError(RuntimeError):
    def __init__(self, code: int, message: str):
        self.code = code
        self.status = STATUS.get(code, str(code))
        super().__init__(f"{self.status}: {message}")


def lib():
    return _native.load()


def _check(code: int) -> None:
    if code != 0:
        raise GftError(code, lib().gft_last_error().decode())


def _ptr(a) -> C.c_void_p:
    """Address of a numpy array or a torch tensor (no copy)."""
    if a is None:
        return C.c_void_p(0)
    if isinstance(a, np.ndarray):
        return C.c_void_p(a.ctypes.data)
    return C.c_void_p(a.data_ptr())


def _stream_ptr(stream) -> C.c_void_p:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _as_f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def laplacian(W, s=None) -> np.ndarray:
    """Eq. 5: Laplacian from symmetric weights W and self-loops s (host)."""
    W = _as_f64(W)
    n = W.shape[0]
    sv = None if s is None else _as_f64(s, (n,))
    L = np.empty((n, n))
    _check(lib().gft_laplacian_from_weights(n, _ptr(W), _ptr(sv), _ptr(L)))
    return L


def normalized_laplacian(W, s=None) -> np.ndarray:
    """Symmetric normalised Laplacian D^-1/2 L D^-1/2 (Sec. II-B), host."""
    W = _as_f64(W)
    n = W.shape[0]
    sv = None if s is None else _as_f64(s, (n,))
    L = np.empty((n, n))
    _check(lib().gft_normalized_laplacian_from_weights(n, _ptr(W), _ptr(sv), _ptr(L)))
    return L


class Plan:
    """A fast-GFT plan for one graph (gft_plan_create)."""

    def __init__(self, L, phis: Optional[Sequence] = None, *, split_components: bool = False,
                 order_block: bool = False, analyze_only: bool = False, jit: bool = True,
                 kernel: str = "auto", search: bool = False, normalized: bool = False):
        """L: Laplacian (n x n); phis: stage involutions on the original labels
        (or search=True to find them, Sec. V-F); normalized=True builds the
        plan for D^-1/2 L D^-1/2."""
        L = _as_f64(L)
        n = L.shape[0]
        if L.shape != (n, n):
            raise ValueError("L must be square")
        phis = [] if phis is None else list(phis)
        ph = (np.ascontiguousarray(np.stack([np.asarray(p, dtype=np.int32) for p in phis]))
              if phis else None)
        flags = ((SPLIT_COMPONENTS if split_components else 0) | (ORDER_BLOCK if order_block else 0)
                 | (ANALYZE_ONLY if analyze_only else 0) | (0 if jit else NO_JIT)
                 | {"auto": 0, "table": KERNEL_TABLE, "wide": KERNEL_WIDE}[kernel]
                 | (SEARCH_STAGES if search else 0) | (NORMALIZED if normalized else 0))
        h = C.c_void_p()
        self._h = None
        _check(lib().gft_plan_create(n, _ptr(L), len(phis), _ptr(ph), flags, C.byref(h)))
        self._h = h
        self.n = n

    @classmethod
    def bipartite(cls, L, side=None, *, order_block: bool = False, analyze_only: bool = False,
                  jit: bool = True, kernel: str = "auto", normalized: bool = False) -> "Plan":
        """Plan with a right Haar stage for a bipartite graph (Sec. III-A,
        gft_plan_create_bipartite): side = None (two-colouring) or 0 / 1 per node."""
        L = _as_f64(L)
        n = L.shape[0]
        if L.shape != (n, n):
            raise ValueError("L must be square")
        sd = None if side is None else np.ascontiguousarray(np.asarray(side, dtype=np.int32))
        if sd is not None and sd.shape != (n,):
            raise ValueError("side must have n entries")
        flags = ((ORDER_BLOCK if order_block else 0) | (ANALYZE_ONLY if analyze_only else 0)
                 | (0 if jit else NO_JIT) | {"auto": 0, "table": KERNEL_TABLE, "wide": KERNEL_WIDE}[kernel]
                 | (NORMALIZED if normalized else 0))
        h = C.c_void_p()
        _check(lib().gft_plan_create_bipartite(n, _ptr(L), _ptr(sd), flags, C.byref(h)))
        return cls._wrap(h, n)

    @classmethod
    def _wrap(cls, handle, n):
        obj = cls.__new__(cls)
        obj._h = handle
        obj.n = n
        return obj

    # -- lifetime ------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().gft_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- introspection ---------------------------------------------------------
    @property
    def info(self) -> dict:
        inf = _native.PlanInfo()
        _check(lib().gft_plan_get_info(self._h, C.byref(inf)))
        return {f: getattr(inf, f) for f, _ in _native.PlanInfo._fields_}

    def stage_pairs(self, stage: int) -> np.ndarray:
        cnt = C.c_int32(0)
        _check(lib().gft_plan_get_stage_pairs(self._h, stage, None, C.byref(cnt)))
        out = np.zeros((cnt.value, 2), dtype=np.int32)
        if cnt.value:
            _check(lib().gft_plan_get_stage_pairs(self._h, stage, _ptr(out), C.byref(cnt)))
        return out

    def leaves(self):
        inf = self.info
        sizes = np.zeros(inf["n_leaves"], dtype=np.int32)
        labels = np.zeros(self.n, dtype=np.int32)
        _check(lib().gft_plan_get_leaves(self._h, _ptr(sizes), _ptr(labels)))
        out, o = [], 0
        for m in sizes:
            out.append(labels[o:o + m].tolist())
            o += m
        return out

    def leaf_laplacian(self, k: int) -> np.ndarray:
        m = len(self.leaves()[k])
        out = np.zeros((m, m))
        _check(lib().gft_plan_get_leaf_laplacian(self._h, k, _ptr(out)))
        return out

    def output_map(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int32)
        _check(lib().gft_plan_get_output_map(self._h, _ptr(out)))
        return out

    def eigenvalues(self) -> np.ndarray:
        out = np.zeros(self.n)
        _check(lib().gft_plan_eigenvalues(self._h, _ptr(out)))
        return out

    def basis(self) -> np.ndarray:
        out = np.zeros((self.n, self.n))
        _check(lib().gft_plan_basis(self._h, _ptr(out)))
        return out

    # -- transforms ------------------------------------------------------------
    def _run(self, fn_name, x, out, precision, stream):
        import torch
        if not (isinstance(x, torch.Tensor) and x.is_cuda):
            raise TypeError("x must be a CUDA tensor")
        if x.dim() != 2 or x.shape[1] != self.n or not x.is_contiguous():
            raise ValueError(f"x must be a contiguous [batch, {self.n}] tensor")
        if out is None:
            out = torch.empty_like(x)
        f = getattr(lib(), fn_name)
        if fn_name.endswith("_f64"):
            _check(f(self._h, _ptr(x), _ptr(out), x.shape[0], _stream_ptr(stream)))
        else:
            _check(f(self._h, _ptr(x), _ptr(out), x.shape[0], _stream_ptr(stream), PRECISIONS[precision]))
        return out

    def forward(self, x, out=None, precision: str = "fp32", stream=None):
        """y = U^T x for every row of a CUDA tensor (float32, or float64)."""
        import torch
        if x.dtype == torch.float64:
            return self._run("gft_plan_forward_f64", x, out, precision, stream)
        return self._run("gft_plan_forward", x, out, precision, stream)

    def inverse(self, y, out=None, precision: str = "fp32", stream=None):
        import torch
        if y.dtype == torch.float64:
            return self._run("gft_plan_inverse_f64", y, out, precision, stream)
        return self._run("gft_plan_inverse", y, out, precision, stream)

    def forward_host(self, x, out=None, precision: str = "fp32"):
        """Forward transform of a host batch (numpy float32 or CPU tensor);
        the library pipelines host-device copies with the kernels."""
        import torch
        if isinstance(x, np.ndarray):
            x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
        if x.dtype != torch.float32 or x.is_cuda or x.dim() != 2 or x.shape[1] != self.n:
            raise ValueError("x must be a host float32 [batch, n] array")
        x = x.contiguous()
        if out is None:
            out = torch.empty_like(x)
        _check(lib().gft_plan_forward_host(self._h, _ptr(x), _ptr(out), x.shape[0], PRECISIONS[precision]))
        return out

    def kernel_source(self, f64: bool = False) -> str:
        """Source of the plan-specialised kernel module (NVRTC input)."""
        n = C.c_int64(0)
        _check(lib().gft_plan_kernel_source(self._h, int(f64), None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(lib().gft_plan_kernel_source(self._h, int(f64), buf, C.byref(n)))
        return buf.value.decode()

    def device_error(self) -> int:
        v = C.c_int32(0)
        _check(lib().gft_device_error(self._h, C.byref(v)))
        return v.value


def find_involution(L, classes=None, max_steps: int = 0):
    """Involution search (gft_find_involution): (phi, pairs)."""
    L = _as_f64(L)
    n = L.shape[0]
    cl = None if classes is None else np.ascontiguousarray(np.asarray(classes, dtype=np.int32))
    phi = np.zeros(n, dtype=np.int32)
    pairs = C.c_int32(0)
    _check(lib().gft_find_involution(n, _ptr(L), _ptr(cl), int(max_steps), _ptr(phi), C.byref(pairs)))
    return phi, pairs.value


def search_stages(L, max_stages: int = 8, max_steps: int = 0):
    """Stage involutions found by search (gft_search_stages), for Plan()."""
    L = _as_f64(L)
    n = L.shape[0]
    out = np.zeros((max(max_stages, 1), n), dtype=np.int32)
    cnt = C.c_int32(0)
    _check(lib().gft_search_stages(n, _ptr(L), int(max_stages), int(max_steps), _ptr(out), C.byref(cnt)))
    return [out[s].copy() for s in range(cnt.value)]


def plans_from_laplacians(Ls, phis_list, *, split_components: bool = False, order_block: bool = False,
                          analyze_only: bool = False, jit: bool = True, kernel: str = "auto",
                          search: bool = False, normalized: bool = False):
    """Many plans at once (gft_plan_create_many): every graph's leaves are
    eigendecomposed in one batched Jacobi solve on the device."""
    k = len(Ls)
    Ls = [_as_f64(L) for L in Ls]
    phs = [(np.ascontiguousarray(np.stack([np.asarray(p, dtype=np.int32) for p in ph])) if len(ph) else None)
           for ph in phis_list]
    ns = np.array([L.shape[0] for L in Ls], dtype=np.int32)
    st = np.array([len(ph) for ph in phis_list], dtype=np.int32)
    Lp = (C.c_void_p * k)(*[L.ctypes.data for L in Ls])
    Pp = (C.c_void_p * k)(*[(p.ctypes.data if p is not None else None) for p in phs])
    flags = ((SPLIT_COMPONENTS if split_components else 0) | (ORDER_BLOCK if order_block else 0)
             | (ANALYZE_ONLY if analyze_only else 0) | (0 if jit else NO_JIT)
             | {"auto": 0, "table": KERNEL_TABLE, "wide": KERNEL_WIDE}[kernel]
             | (SEARCH_STAGES if search else 0) | (NORMALIZED if normalized else 0))
    out = (C.c_void_p * k)()
    _check(lib().gft_plan_create_many(k, _ptr(ns), C.cast(Lp, C.c_void_p), _ptr(st), C.cast(Pp, C.c_void_p),
                                      flags, C.cast(out, C.c_void_p)))
    return [Plan._wrap(C.c_void_p(out[i]), int(ns[i])) for i in range(k)]


class ApproxGFT:
    """Approximate GFT by greedy layers of Jacobi rotations, alone (phis =
    []) or after the Haar stages of the symmetric decomposition (Sec. VI-B,
    gft_approx_create)."""

    def __init__(self, L, phis: Optional[Sequence] = None, n_layers: int = 10, *,
                 split_components: bool = False, analyze_only: bool = False):
        L = _as_f64(L)
        n = L.shape[0]
        if L.shape != (n, n):
            raise ValueError("L must be square")
        phis = [] if phis is None else list(phis)
        ph = (np.ascontiguousarray(np.stack([np.asarray(p, dtype=np.int32) for p in phis]))
              if phis else None)
        flags = (SPLIT_COMPONENTS if split_components else 0) | (ANALYZE_ONLY if analyze_only else 0)
        h = C.c_void_p()
        self._h = None
        _check(lib().gft_approx_create(n, _ptr(L), len(phis), _ptr(ph), int(n_layers), flags, C.byref(h)))
        self._h = h
        self.n = n

    def close(self):
        if getattr(self, "_h", None):
            lib().gft_approx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self) -> dict:
        inf = _native.ApproxInfo()
        _check(lib().gft_approx_get_info(self._h, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in inf._fields_}

    def units(self):
        """(layer_off, pairs [units, 2], coef [units, 4], perm)."""
        inf = self.info
        lo = np.zeros(inf["n_layers"] + 1, dtype=np.int32)
        pr = np.zeros((max(1, inf["n_units"]), 2), dtype=np.int32)
        cf = np.zeros((max(1, inf["n_units"]), 4))
        pm = np.zeros(self.n, dtype=np.int32)
        _check(lib().gft_approx_get_units(self._h, _ptr(lo), _ptr(pr), _ptr(cf), _ptr(pm)))
        return lo, pr[:inf["n_units"]], cf[:inf["n_units"]], pm

    def eigenvalues(self) -> np.ndarray:
        lam = np.zeros(self.n)
        _check(lib().gft_approx_eigenvalues(self._h, _ptr(lam)))
        return lam

    def basis(self) -> np.ndarray:
        U = np.zeros((self.n, self.n))
        _check(lib().gft_approx_basis(self._h, _ptr(U)))
        return U

    def forward(self, x, out=None, stream=None):
        import torch
        if x.dtype != torch.float32 or not x.is_cuda or x.dim() != 2 or x.shape[1] != self.n:
            raise ValueError("x must be a CUDA float32 tensor [batch, n]")
        x = x.contiguous()
        y = torch.empty_like(x) if out is None else out
        _check(lib().gft_approx_forward(self._h, _ptr(x), _ptr(y), x.shape[0], _stream_ptr(stream)))
        return y


class Batch:
    """Many plans transformed by one graph-captured launch (gft_batch_create):
    persistent kernels over (plan, tile) work lists, plus the tensor-core
    kernels of wide plans when a tensor-core precision is asked for.
    ``jit=False`` keeps every plan off the plan-specialised group (small
    plans shared by many entries, compiled into one module at creation)."""

    BATCH_NO_JIT = 0x100

    def __init__(self, plans: Sequence[Plan], batches: Sequence[int], precision: str = "fp32", jit: bool = True):
        self.plans = list(plans)
        arr = (C.c_void_p * len(plans))(*[p.handle for p in plans])
        b = np.ascontiguousarray(np.asarray(batches, dtype=np.int64))
        h = C.c_void_p()
        self._h = None
        flags = PRECISIONS[precision] | (0 if jit else self.BATCH_NO_JIT)
        _check(lib().gft_batch_create(len(plans), C.cast(arr, C.c_void_p), _ptr(b), flags, C.byref(h)))
        self._h = h
        self.batches = b

    def bind(self, xs, ys):
        """Marshal the signal and coefficient tensors once (one per plan);
        ``forward()`` without arguments then replays the batch on them.  The
        caller keeps the tensors alive while they are bound."""
        k = len(self.plans)
        if len(xs) != k or len(ys) != k:
            raise ValueError("one input and one output tensor per plan")
        self._bound = ((C.c_void_p * k)(*[t.data_ptr() for t in xs]),
                       (C.c_void_p * k)(*[t.data_ptr() for t in ys]), list(xs), list(ys))
        return self

    def forward(self, xs=None, ys=None, stream=None):
        if xs is None and ys is None:
            if getattr(self, "_bound", None) is None:
                raise ValueError("no tensors bound: pass xs and ys or call bind() first")
            xa, ya, _, ys = self._bound
        else:
            k = len(self.plans)
            xa = (C.c_void_p * k)(*[t.data_ptr() for t in xs])
            ya = (C.c_void_p * k)(*[t.data_ptr() for t in ys])
        _check(lib().gft_batch_forward(self._h, C.cast(xa, C.c_void_p), C.cast(ya, C.c_void_p),
                                       _stream_ptr(stream)))
        return ys

    def tile(self, i: int):
        t, th = C.c_int32(), C.c_int32()
        _check(lib().gft_batch_get_tile(self._h, i, C.byref(t), C.byref(th)))
        return t.value, th.value

    @property
    def launches(self) -> int:
        """Kernel launches of this library per forward (graph nodes)."""
        n = C.c_int32()
        _check(lib().gft_batch_get_launches(self._h, C.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "_h", None):
            lib().gft_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Givens:
    """Layered Givens rotations (Eq. 1, Fig. 1) on fixed pairings."""

    def __init__(self, n: int, pairs):
        pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32))
        if pairs.ndim != 3 or pairs.shape[1:] != (n // 2, 2):
            raise ValueError("pairs must have shape (n_stages, n/2, 2)")
        h = C.c_void_p()
        self._h = None
        _check(lib().gft_givens_create(n, pairs.shape[0], _ptr(pairs), C.byref(h)))
        self._h = h
        self.n = n
        self.n_stages = pairs.shape[0]
        self.pairs = pairs

    def forward(self, theta, x, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(x)
        _check(lib().gft_givens_forward(self._h, _ptr(theta), _ptr(x), _ptr(out), x.shape[0],
                                        _stream_ptr(stream)))
        return out

    def backward(self, theta, y, gy, stream=None):
        import torch
        gx = torch.empty_like(gy)
        gth = torch.empty_like(theta)
        _check(lib().gft_givens_backward(self._h, _ptr(theta), _ptr(y), _ptr(gy), _ptr(gx), _ptr(gth),
                                         y.shape[0], _stream_ptr(stream)))
        return gx, gth

    def close(self):
        if getattr(self, "_h", None):
            lib().gft_givens_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _givens_function():
    import torch

    class GivensFunction(torch.autograd.Function):
        """y = G_S ... G_1 x with hand-written forward and backward kernels."""

        @staticmethod
        def forward(ctx, x, theta, net):
            y = net.forward(theta.detach().contiguous(), x.detach().contiguous())
            ctx.save_for_backward(y, theta)
            ctx.net = net
            return y

        @staticmethod
        def backward(ctx, gy):
            y, theta = ctx.saved_tensors
            gx, gth = ctx.net.backward(theta.detach().contiguous(), y, gy.contiguous())
            return gx, gth, None

    return GivensFunction


_GF = None


def givens_apply(x, theta, net: Givens):
    """Differentiable Givens surrogate (autograd through the CUDA kernels)."""
    global _GF
    if _GF is None:
        _GF = _givens_function()
    return _GF.apply(x, theta, net)


__all__ = ["Plan", "Batch", "ApproxGFT", "Givens", "givens_apply", "laplacian", "normalized_laplacian", "GftError", "lib",
           "SPLIT_COMPONENTS", "ORDER_BLOCK", "ANALYZE_ONLY", "NO_JIT", "KERNEL_TABLE",
           "KERNEL_WIDE", "SEARCH_STAGES", "NORMALIZED", "PRECISIONS", "plans_from_laplacians", "find_involution", "search_stages"]
