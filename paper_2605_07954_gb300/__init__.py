"""GB300-native iterated explicit 2D stencil sweeps (sm_103a CUDA behind a C ABI).

The computation (Jacobi update, paper Sec. II-C; zero padding as the boundary,
Sec. IV-A) runs entirely in the CUDA library ``libstencil_gb300.so``; this
package only marshals arguments.  PyTorch supplies device memory and the
current stream.  ``_capi`` holds the raw C entry points under their C names;
:class:`Plan` is a thin convenience wrapper over them.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi
from ._capi import StencilError, check

DTYPES = {"f32": _capi.STENCIL_F32, "bf16": _capi.STENCIL_BF16, "f16": _capi.STENCIL_F16}
BOUNDARIES = {"zero": _capi.STENCIL_BOUNDARY_ZERO, "periodic": _capi.STENCIL_BOUNDARY_PERIODIC}
COMPUTES = {"auto": 0, "fp32": 1, "tc_tf32": 2, "tc_bf16": 3, "tc_3xtf32": 4, "lowrank": 5}
KERNELS = {"auto": 0, "naive": 1, "stream": 2, "tc": 3, "tc_warp": 4, "tc_umma": 5, "resident": 6,
           "lowrank": 7}
LOADS = {"auto": 0, "cp_async": 1, "tma": 2}


def _torch_dtype_name(t) -> str:
    import torch
    return {torch.float32: "f32", torch.bfloat16: "bf16", torch.float16: "f16"}[t]


def _current_stream_handle() -> int:
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


class Plan:
    """A plan for T-step sweeps of one (ny, nx) grid with one weight set."""

    def __init__(self, ny: int, nx: int, weights, dtype: str = "f32", boundary: str = "zero",
                 compute: str = "auto", kernel: str = "auto", tb_depth: int = 0,
                 threads: int = 0, tile_rows: int = 0, autotune: bool = False, mma_n: int = 0,
                 timeout_ms: int = 0, debug_withhold: int = 0, load: str = "auto", rank: int = 0):
        lib = _capi.load()
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32))
        d = w.shape[0]
        if w.ndim != 2 or w.shape[1] != d or d % 2 != 1:
            raise ValueError(f"weights must be (2r+1, 2r+1), got {w.shape}")
        self.radius = d // 2
        self.shape = (int(ny), int(nx))
        self.dtype = dtype
        self.weights = w
        opt = _capi.stencil_options_t(COMPUTES[compute], KERNELS[kernel], int(tb_depth),
                                      int(threads), int(tile_rows), int(bool(autotune)), int(mma_n),
                                      int(timeout_ms), int(debug_withhold), LOADS[load], int(rank))
        h = ctypes.c_void_p()
        check(lib.stencil_plan_create(ctypes.byref(h), int(ny), int(nx), self.radius,
                                      w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                      DTYPES[dtype], BOUNDARIES[boundary], ctypes.byref(opt)),
              "stencil_plan_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _capi.load().stencil_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_weights(self, weights) -> None:
        """Replace the weights in place (stencil_plan_set_weights): same footprint class."""
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32))
        if w.shape != self.weights.shape:
            raise ValueError(f"weights must be {self.weights.shape}, got {w.shape}")
        check(_capi.load().stencil_plan_set_weights(self._h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
              "stencil_plan_set_weights")
        self.weights = w

    def info(self) -> dict:
        i = _capi.stencil_plan_info_t()
        check(_capi.load().stencil_plan_info(self._h, ctypes.byref(i)), "stencil_plan_info")
        return {f: getattr(i, f) for f, _ in i._fields_}

    def launches(self, T: int) -> int:
        return int(_capi.load().stencil_run_launches(self._h, int(T)))

    def _check_tensor(self, x):
        import torch
        if not x.is_cuda or not x.is_contiguous() or tuple(x.shape) != self.shape:
            raise ValueError(f"expected a contiguous CUDA tensor of shape {self.shape}")
        if _torch_dtype_name(x.dtype) != self.dtype:
            raise ValueError(f"expected dtype {self.dtype}, got {x.dtype}")
        return torch

    def run(self, x, T: int, out=None):
        """u_T from u_0 = x (device tensor); enqueued on torch's current stream."""
        torch = self._check_tensor(x)
        if out is None:
            out = torch.empty_like(x)
        else:
            self._check_tensor(out)
        check(_capi.load().stencil_run(self._h, x.data_ptr(), out.data_ptr(), int(T),
                                       _current_stream_handle()), "stencil_run")
        return out

    def run_residual(self, x, T: int, m: int, out=None):
        """u_T and the residuals ||u_t - u_{t-1}||_2 after every m-th step (CUDA float64)."""
        torch = self._check_tensor(x)
        if out is None:
            out = torch.empty_like(x)
        else:
            self._check_tensor(out)
        res = torch.empty(max(1, int(T) // int(m)), dtype=torch.float64, device=x.device)
        check(_capi.load().stencil_run_residual(self._h, x.data_ptr(), out.data_ptr(), int(T), int(m),
                                                res.data_ptr(), _current_stream_handle()),
              "stencil_run_residual")
        return out, res[: int(T) // int(m)]

    def run_host(self, x: np.ndarray, T: int, out: np.ndarray | None = None, stream: int = 0):
        """Host in, host out: H2D copy, T steps and D2H copy, synchronised."""
        if x.shape != self.shape or not x.flags["C_CONTIGUOUS"]:
            raise ValueError(f"expected a C-contiguous array of shape {self.shape}")
        if out is None:
            out = np.empty_like(x)
        check(_capi.load().stencil_run_host(self._h, x.ctypes.data, out.ctypes.data, int(T),
                                            stream), "stencil_run_host")
        return out

    def run_host_async(self, x: np.ndarray, T: int, out: np.ndarray, stream: int = 0):
        """Host in, host out, enqueued on `stream` without synchronising
        (stencil_run_host_async): `out` holds u_T once the stream is done.
        Both arrays must stay alive until then; pin them for overlap."""
        if x.shape != self.shape or not x.flags["C_CONTIGUOUS"] or out.shape != self.shape:
            raise ValueError(f"expected C-contiguous arrays of shape {self.shape}")
        check(_capi.load().stencil_run_host_async(self._h, x.ctypes.data, out.ctypes.data, int(T), stream),
              "stencil_run_host_async")
        return out

    def status(self):
        check(_capi.load().stencil_plan_status(self._h), "stencil_plan_status")


def adjoint(plan: Plan, u0, grad_uT, T: int, ckpt_interval: int = 0):
    """(dL/du0, dL/dW) for a loss L(u_T) with dL/du_T = grad_uT (stencil_adjoint).

    Returns a CUDA tensor like u0 and a (2r+1, 2r+1) float64 CUDA tensor.
    Enqueued on torch's current stream.
    """
    import torch
    plan._check_tensor(u0)
    plan._check_tensor(grad_uT)
    g_u0 = torch.empty_like(u0)
    d = 2 * plan.radius + 1
    g_w = torch.empty((d, d), dtype=torch.float64, device=u0.device)
    check(_capi.load().stencil_adjoint(plan.handle, u0.data_ptr(), grad_uT.data_ptr(), int(T),
                                       g_u0.data_ptr(), g_w.data_ptr(), int(ckpt_interval),
                                       _current_stream_handle()), "stencil_adjoint")
    return g_u0, g_w


class _PlanCache:
    """Plans for StencilFn, reused across calls: keyed by (device, shape,
    radius, footprint class, boundary); a hit only replaces the weights
    (stencil_plan_set_weights), so the workspace, the tuned configuration and
    the adjoint's checkpoint scratch are allocated once, not per iteration.
    At most `size` plans are kept (least recently used dropped first)."""

    def __init__(self, size: int = 8):
        self.size = size
        self.plans = {}

    def get(self, device: int, ny: int, nx: int, W: np.ndarray, boundary: str) -> Plan:
        r = W.shape[0] // 2
        star = bool(np.all(W[np.arange(W.shape[0]) != r][:, np.arange(W.shape[1]) != r] == 0))
        key = (device, ny, nx, r, star, boundary)
        plan = self.plans.pop(key, None)
        if plan is None:
            plan = Plan(ny, nx, W, boundary=boundary)
            while len(self.plans) >= self.size:
                self.plans.pop(next(iter(self.plans))).close()
        else:
            plan.set_weights(W)
        self.plans[key] = plan  # most recently used last
        return plan


_PLANS = _PlanCache()


def _stencil_fn():
    import torch

    class StencilFn(torch.autograd.Function):
        """u_T = A^T u0 with gradients for u0 and the weights (sqrt(T) checkpointing).

        apply(u0, weights, T, boundary="zero", ckpt_interval=0): u0 a CUDA FP32
        tensor; weights a (2r+1, 2r+1) tensor on any device (its values are read
        at forward time).  The weight gradient has the weights' dtype and device.
        Plans come from a small per-process cache (see _PlanCache), so repeated
        calls with new weights allocate nothing new.  The backward pass uses the
        weights of its own forward call, read back from the saved copy.
        """

        @staticmethod
        def forward(ctx, u0, weights, T, boundary="zero", ckpt_interval=0):
            W = np.ascontiguousarray(weights.detach().to("cpu", torch.float32).numpy())
            plan = _PLANS.get(u0.device.index if u0.is_cuda else -1, u0.shape[0], u0.shape[1], W, boundary)
            u0c = u0.detach().contiguous()
            y = plan.run(u0c, int(T))
            ctx.save_for_backward(u0c)
            ctx.plan, ctx.W, ctx.T, ctx.ckpt = plan, W, int(T), int(ckpt_interval)
            ctx.wdtype, ctx.wdevice = weights.dtype, weights.device
            return y

        @staticmethod
        def backward(ctx, grad_y):
            (u0,) = ctx.saved_tensors
            # another forward call may have changed the cached plan's weights
            ctx.plan.set_weights(ctx.W)
            g_u0, g_w = adjoint(ctx.plan, u0, grad_y.contiguous(), ctx.T, ctx.ckpt)
            return g_u0, g_w.to(ctx.wdevice, ctx.wdtype), None, None, None

    return StencilFn


def __getattr__(name):
    if name == "StencilFn":
        fn = _stencil_fn()
        globals()["StencilFn"] = fn
        return fn
    raise AttributeError(name)


class Batch:
    """Many independent grids run by one persistent launch (CUDA-graph replayed).

    ``grids`` is a list of dicts with keys ``x`` (input, CUDA tensor), ``out``
    (output tensor, may be ``x``), ``weights`` ((2r+1)^2 array), ``T`` and
    optionally ``boundary``.  The tensors must stay alive while the batch is used.
    """

    def __init__(self, grids, dtype: str = "f32", tb_depth: int = 0, threads: int = 0,
                 tile_rows: int = 0, autotune: bool = False, timeout_ms: int = 0,
                 debug_withhold_item: int = 0):
        lib = _capi.load()
        n = len(grids)
        descs = (_capi.stencil_grid_desc_t * n)()
        self._keep = []
        for i, g in enumerate(grids):
            w = np.ascontiguousarray(np.asarray(g["weights"], dtype=np.float32))
            self._keep.append(w)
            x, out = g["x"], g["out"]
            if _torch_dtype_name(x.dtype) != dtype or out.dtype != x.dtype:
                raise ValueError("grid tensors must match the batch dtype")
            if not (x.is_cuda and x.is_contiguous() and out.is_contiguous() and x.shape == out.shape):
                raise ValueError("grids must be contiguous CUDA tensors of equal shape")
            descs[i] = _capi.stencil_grid_desc_t(
                x.shape[0], x.shape[1], w.shape[0] // 2,
                w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                BOUNDARIES[g.get("boundary", "zero")], int(g["T"]), x.data_ptr(), out.data_ptr())
        opt = _capi.stencil_batch_options_t(int(tb_depth), int(threads), int(tile_rows),
                                            int(bool(autotune)), int(timeout_ms),
                                            int(debug_withhold_item))
        h = ctypes.c_void_p()
        check(lib.stencil_batch_create(ctypes.byref(h), n, descs, DTYPES[dtype], ctypes.byref(opt)),
              "stencil_batch_create")
        self._h = h

    def run(self):
        check(_capi.load().stencil_run_batched(self._h, _current_stream_handle()),
              "stencil_run_batched")

    def status(self):
        check(_capi.load().stencil_batch_status(self._h), "stencil_batch_status")

    def info(self) -> dict:
        i = _capi.stencil_batch_info_t()
        check(_capi.load().stencil_batch_info(self._h, ctypes.byref(i)), "stencil_batch_info")
        return {f: getattr(i, f) for f, _ in i._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _capi.load().stencil_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run(x, weights, T: int, boundary: str = "zero", **options):
    """One-shot convenience: plan, run on the current stream, return u_T."""
    p = Plan(x.shape[0], x.shape[1], weights, dtype=_torch_dtype_name(x.dtype),
             boundary=boundary, **options)
    y = p.run(x, T)
    import torch
    torch.cuda.current_stream().synchronize()
    p.close()
    return y


__all__ = ["Plan", "Batch", "StencilFn", "adjoint", "run", "StencilError", "DTYPES", "BOUNDARIES"]
