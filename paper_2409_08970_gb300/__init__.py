"""GB300 Fast DCT+: batched GFTs of rank-one updates of the path graph.

Python layer over the C ABI in ``include/dctplus.h``. Functions named
``dctplus_*`` mirror the C entry points one to one (handles and raw pointers);
``Plan`` and ``Group`` wrap them for torch tensors. PyTorch supplies device
memory and streams only: every step of the transform runs in the library's
CUDA kernels, and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import weakref
from collections import OrderedDict

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401
    CAUCHY_AUTO, CAUCHY_DENSE, CAUCHY_DENSE_GFT, CAUCHY_HIER, CAUCHY_NFST, CAUCHY_SIMT, ERR_SCRATCH_LIMIT,
    F32, F64,
    SEG_WORDS, DctPlusError, Opts,
    check,
)

__all__ = [
    "Plan", "Group", "DctPlusError", "dctplus_plan", "dctplus_destroy", "dctplus_plan_inspect",
    "dctplus_execute", "dctplus_execute_host", "dctplus_execute_noalloc", "dctplus_execute_pruned",
    "dctplus_backward", "dctplus_group_create", "DctPlusFunction", "dct_plus", "dctplus_group_destroy",
    "dctplus_execute_group", "dctplus_execute_group_host", "dctplus_sync_check",
    "dctplus_launch_count", "dctplus_status_string", "dctplus_trace_begin", "dctplus_trace_end",
    "dctplus_autotune", "dctplus_tune_lookup", "dctplus_tune_record", "library_path",
]


def library_path() -> str:
    return _lib.LIB_PATH


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- raw C names

def dctplus_status_string(status: int) -> str:
    return _lib.load().dctplus_status_string(int(status)).decode()


def dctplus_launch_count() -> int:
    return int(_lib.load().dctplus_launch_count())


def dctplus_plan(n: int, v, rho: float, opts: Opts | None = None) -> ctypes.c_void_p:
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    if v.shape != (n,):
        raise ValueError("v must have shape (n,)")
    h = ctypes.c_void_p()
    st = _lib.load().dctplus_plan(ctypes.byref(h), int(n), v.ctypes.data, float(rho),
                                  ctypes.byref(opts) if opts is not None else None)
    check(st, "dctplus_plan")
    return h


def dctplus_destroy(handle) -> None:
    _lib.load().dctplus_destroy(handle)


def dctplus_plan_inspect(handle, n: int) -> dict:
    out = {k: np.zeros(n) for k in ("eigenvalues", "z", "row_tau", "row_a")}
    out["row_kind"] = np.zeros(n, dtype=np.int32)
    out["row_pole"] = np.zeros(n, dtype=np.int32)
    st = _lib.load().dctplus_plan_inspect(
        handle, out["eigenvalues"].ctypes.data, out["z"].ctypes.data, out["row_kind"].ctypes.data,
        out["row_pole"].ctypes.data, out["row_tau"].ctypes.data, out["row_a"].ctypes.data)
    check(st, "dctplus_plan_inspect")
    return out


def dctplus_execute(handle, dtype: int, x_ptr: int, ldx: int, y_ptr: int, ldy: int, batch: int,
                    stream: int) -> None:
    st = _lib.load().dctplus_execute(handle, int(dtype), x_ptr, int(ldx), y_ptr, int(ldy),
                                     int(batch), stream)
    check(st, "dctplus_execute")


def dctplus_execute_host(handle, dtype: int, x_ptr: int, y_ptr: int, batch: int, stream: int) -> None:
    st = _lib.load().dctplus_execute_host(handle, int(dtype), x_ptr, y_ptr, int(batch), stream)
    check(st, "dctplus_execute_host")


def dctplus_execute_noalloc(handle, x_ptr: int, ldx: int, y_ptr: int, ldy: int, batch: int,
                            stream: int) -> None:
    st = _lib.load().dctplus_execute_noalloc(handle, x_ptr, int(ldx), y_ptr, int(ldy), int(batch),
                                             stream)
    check(st, "dctplus_execute_noalloc")


def dctplus_execute_pruned(handles, x_ptr: int, ldx: int, y_ptr: int, ldy: int, batch: int,
                           m_out: int, c_p: int, stream: int) -> None:
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    st = _lib.load().dctplus_execute_pruned(arr, len(handles), x_ptr, int(ldx), y_ptr, int(ldy),
                                            int(batch), int(m_out), int(c_p), stream)
    check(st, "dctplus_execute_pruned")


def dctplus_execute_multi(handles, x_ptr: int, ldx: int, y_ptr: int, ldy: int, batch: int,
                          stream: int) -> None:
    """Several plans of one length over the same FP32 signals; plan k's coefficients at columns
    k n .. k n + n - 1 of each output row (ldy >= len(handles) n)."""
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    st = _lib.load().dctplus_execute_multi(arr, len(handles), x_ptr, int(ldx), y_ptr, int(ldy), int(batch), stream)
    check(st, "dctplus_execute_multi")


def dctplus_backward(handle, gy_ptr: int, ldg: int, y_ptr: int, ldy: int, gx_ptr: int, ldgx: int,
                     grad_rho_ptr: int, grad_v_ptr: int, batch: int, stream: int) -> None:
    st = _lib.load().dctplus_backward(handle, gy_ptr, int(ldg), y_ptr or None, int(ldy), gx_ptr or None,
                                      int(ldgx), grad_rho_ptr or None, grad_v_ptr or None, int(batch),
                                      stream)
    check(st, "dctplus_backward")


def dctplus_group_create(handles) -> ctypes.c_void_p:
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    g = ctypes.c_void_p()
    check(_lib.load().dctplus_group_create(ctypes.byref(g), len(handles), arr), "dctplus_group_create")
    return g


def dctplus_group_destroy(g) -> None:
    _lib.load().dctplus_group_destroy(g)


def dctplus_execute_group(g, x_ptr: int, y_ptr: int, seg: np.ndarray, stream: int) -> None:
    seg = np.ascontiguousarray(seg, dtype=np.int64).reshape(-1, SEG_WORDS)
    st = _lib.load().dctplus_execute_group(g, x_ptr, y_ptr, seg.ctypes.data, seg.shape[0], stream)
    check(st, "dctplus_execute_group")


def dctplus_execute_group_host(g, x_ptr: int, y_ptr: int, total_elems: int, seg: np.ndarray,
                               stream: int) -> None:
    seg = np.ascontiguousarray(seg, dtype=np.int64).reshape(-1, SEG_WORDS)
    st = _lib.load().dctplus_execute_group_host(g, x_ptr, y_ptr, int(total_elems), seg.ctypes.data,
                                                seg.shape[0], stream)
    check(st, "dctplus_execute_group_host")


def dctplus_sync_check(stream: int = 0) -> int:
    return int(_lib.load().dctplus_sync_check(stream))


CANDIDATES = ("dense", "hier_leaf", "hier_tree", "simt")


def dctplus_autotune(n: int, v, rho: float, batch: int, cache_path: str | None = None,
                     stream: int = 0) -> dict:
    """Times the Cauchy evaluations that apply at length n on this device and returns the
    fastest correct one: {"cauchy_mode", "far_field", "ms": {candidate: ms per call}}; with
    cache_path the choice is recorded there (see include/dctplus.h)."""
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    if v.shape != (n,):
        raise ValueError("v must have shape (n,)")
    mode, far = ctypes.c_int(), ctypes.c_int()
    ms = (ctypes.c_double * 4)()
    st = _lib.load().dctplus_autotune(int(n), v.ctypes.data, float(rho), int(batch),
                                      cache_path.encode() if cache_path else None, stream,
                                      ctypes.byref(mode), ctypes.byref(far), ms)
    check(st, "dctplus_autotune")
    return {"cauchy_mode": mode.value, "far_field": far.value,
            "ms": {k: ms[i] for i, k in enumerate(CANDIDATES)}}


def dctplus_tune_lookup(cache_path: str, device_name: str, n: int, batch: int):
    """(cauchy_mode, far_field) recorded for (device, n, batch bucket), or None."""
    mode, far = ctypes.c_int(), ctypes.c_int()
    st = _lib.load().dctplus_tune_lookup(cache_path.encode(), device_name.encode(), int(n), int(batch),
                                         ctypes.byref(mode), ctypes.byref(far))
    if st == _lib.ERR_UNSUPPORTED:
        return None
    check(st, "dctplus_tune_lookup")
    return mode.value, far.value


def dctplus_tune_record(cache_path: str, device_name: str, n: int, batch: int, cauchy_mode: int,
                        far_field: int, ms: float, candidate_ms=None) -> None:
    cand = None
    if candidate_ms is not None:
        cand = (ctypes.c_double * 4)(*[float(c) for c in candidate_ms])
    check(_lib.load().dctplus_tune_record(cache_path.encode(), device_name.encode(), int(n), int(batch),
                                          int(cauchy_mode), int(far_field), float(ms), cand),
          "dctplus_tune_record")


def dctplus_trace_begin(stream: int) -> None:
    check(_lib.load().dctplus_trace_begin(stream), "dctplus_trace_begin")


def dctplus_trace_end(stream: int, cap: int = 256) -> list:
    """Per traced launch: (kernel name, device ms, algorithmic bytes, flops)."""
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_float * cap)()
    by = (ctypes.c_double * cap)()
    fl = (ctypes.c_double * cap)()
    cnt = _lib.load().dctplus_trace_end(stream, names, ms, by, fl, cap)
    if cnt < 0:
        raise DctPlusError(_lib.ERR_INVALID_ARG, "dctplus_trace_end")
    return [(names[i].decode(), float(ms[i]), float(by[i]), float(fl[i])) for i in range(min(cnt, cap))]


# ---------------------------------------------------------------- wrappers

class Plan:
    """A Fast DCT+ plan: the GFT of L~ + rho v v^T for signals of length n."""

    def __init__(self, n: int, v, rho: float, cauchy_mode: int = CAUCHY_AUTO,
                 max_secular_iter: int = 0, far_field: int = 0, device: int = -1,
                 batch_hint: int = 0, tune_cache: str | None = None):
        self.n = int(n)
        self.rho = float(rho)
        opts = Opts(cauchy_mode, max_secular_iter, far_field, device, int(batch_hint),
                    tune_cache.encode() if tune_cache else None)
        self.handle = dctplus_plan(self.n, v, self.rho, opts)

    @property
    def cauchy_mode(self) -> int:
        return int(_lib.load().dctplus_plan_cauchy_mode(self.handle))

    @property
    def far_field(self) -> int:
        """Far-field form of a hierarchical plan: 1 = leaf level, 2 = tree (0 otherwise)."""
        return int(_lib.load().dctplus_plan_far_field(self.handle))

    def inspect(self) -> dict:
        return dctplus_plan_inspect(self.handle, self.n)

    def forward(self, x, out=None, stream=None):
        """y = X^T x for every row of a CUDA tensor x of shape (batch, n), float32 or float64."""
        import torch
        if x.dim() != 2 or x.shape[1] != self.n or x.stride(1) != 1:
            raise ValueError("x must be (batch, n) with unit stride along n")
        dtype = {torch.float32: F32, torch.float64: F64}.get(x.dtype)
        if dtype is None:
            raise TypeError("x must be float32 or float64")
        if out is None:
            out = torch.empty_like(x, memory_format=torch.contiguous_format)
        dctplus_execute(self.handle, dtype, x.data_ptr(), x.stride(0), out.data_ptr(),
                        out.stride(0), x.shape[0], _stream_handle(stream))
        return out

    def forward_host(self, x: np.ndarray, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        """Same transform on host arrays (copies to and from the GPU inside the call)."""
        x = np.ascontiguousarray(x)
        dtype = {np.dtype(np.float32): F32, np.dtype(np.float64): F64}[x.dtype]
        if out is None:
            out = np.empty_like(x)
        dctplus_execute_host(self.handle, dtype, x.ctypes.data, out.ctypes.data, x.shape[0],
                             _stream_handle(stream) if stream is not None else 0)
        return out

    def backward(self, gy, y=None, want_x: bool = True, want_params: bool = False, stream=None):
        """Reverse-mode derivatives for float32 CUDA tensors gy (and the forward output y when
        the parameter gradients are wanted). Returns (gx or None, grad_rho or None, grad_v or None);
        grad_rho and grad_v are float64 tensors."""
        import torch
        if gy.dtype != torch.float32 or gy.dim() != 2 or gy.shape[1] != self.n or gy.stride(1) != 1:
            raise ValueError("gy must be a float32 (batch, n) tensor with unit stride along n")
        batch = gy.shape[0]
        gx = torch.empty_like(gy, memory_format=torch.contiguous_format) if want_x else None
        grad_rho = grad_v = None
        if want_params:
            if y is None or y.shape != gy.shape or y.dtype != torch.float32 or y.stride(1) != 1:
                raise ValueError("y must be the float32 forward output matching gy")
            grad_rho = torch.empty((), dtype=torch.float64, device=gy.device)
            grad_v = torch.empty(self.n, dtype=torch.float64, device=gy.device)
        dctplus_backward(self.handle, gy.data_ptr(), gy.stride(0), y.data_ptr() if want_params else 0,
                         y.stride(0) if want_params else self.n, gx.data_ptr() if gx is not None else 0,
                         gx.stride(0) if gx is not None else self.n,
                         grad_rho.data_ptr() if grad_rho is not None else 0,
                         grad_v.data_ptr() if grad_v is not None else 0, batch, _stream_handle(stream))
        return gx, grad_rho, grad_v

    def close(self) -> None:
        if getattr(self, "handle", None) is not None and self.handle.value:
            dctplus_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Several plans with n <= 64 run as one persistent launch over segments."""

    def __init__(self, plans):
        self.plans = list(plans)
        self.handle = dctplus_group_create([p.handle for p in self.plans])

    def forward(self, x, seg: np.ndarray, out=None, stream=None):
        import torch
        if x.dtype != torch.float32 or not x.is_contiguous():
            raise TypeError("x must be a contiguous float32 CUDA tensor")
        if out is None:
            out = torch.empty_like(x)
        dctplus_execute_group(self.handle, x.data_ptr(), out.data_ptr(), seg, _stream_handle(stream))
        return out

    def forward_host(self, x: np.ndarray, seg: np.ndarray, out=None, stream=None) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32)
        if out is None:
            out = np.empty_like(x)
        dctplus_execute_group_host(self.handle, x.ctypes.data, out.ctypes.data, x.size, seg,
                                   _stream_handle(stream) if stream is not None else 0)
        return out

    def close(self) -> None:
        if getattr(self, "handle", None) is not None and self.handle.value:
            dctplus_group_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- autograd

# Plans of the autograd function, least recently used first, keyed by the values of
# (n, v, rho, device). Evicting a plan only drops the cache's reference: a forward whose
# backward is still pending keeps its plan alive through ctx.plan, and the plan's
# device tables are freed when the last reference goes (Plan.__del__).
_PLAN_CACHE_MAX = 16
_plan_cache: "OrderedDict[tuple, Plan]" = OrderedDict()
# Per tensor object: (weak reference, version counter, value key). When the same v
# (or rho) tensor comes back unmodified, its value key is reused without copying the
# tensor to the host again.
_value_keys: dict = {}


def _value_key(t, to_host):
    """Host value of tensor ``t`` as a hashable key, memoised while ``t`` is unmodified."""
    import torch
    if not torch.is_tensor(t):
        return to_host(t)
    memo = _value_keys.get(id(t))
    if memo is not None and memo[0]() is t and memo[1] == t._version:
        return memo[2]
    key = to_host(t)
    if len(_value_keys) > 4 * _PLAN_CACHE_MAX:  # drop entries of tensors that are gone
        for k in [k for k, m in _value_keys.items() if m[0]() is None]:
            del _value_keys[k]
    _value_keys[id(t)] = (weakref.ref(t), t._version, key)
    return key


def _cached_plan(n: int, v, rho, device: int) -> "Plan":
    import torch
    v_key = _value_key(v, lambda t: np.ascontiguousarray(
        t.detach().to("cpu", torch.float64).numpy() if torch.is_tensor(t) else t,
        dtype=np.float64).tobytes())
    rho_key = _value_key(rho, lambda t: float(t))
    key = (n, v_key, rho_key, device)
    plan = _plan_cache.get(key)
    if plan is not None:
        _plan_cache.move_to_end(key)
        return plan
    while len(_plan_cache) >= _PLAN_CACHE_MAX:
        _plan_cache.popitem(last=False)  # no close(): pending backwards may still hold it
    plan = Plan(n, np.frombuffer(v_key, dtype=np.float64), rho_key, device=device)
    _plan_cache[key] = plan
    return plan


def _make_function():
    import torch

    class DctPlusFunction(torch.autograd.Function):
        """y = X(v, rho)^T x on float32 CUDA signals (rows of x), differentiable in x, v and rho.

        v (n,) and rho (scalar) are float64 tensors; the plan for (v, rho) is built on the GPU
        (and cached, least recently used out) in the forward, and held by ctx until the
        backward, which calls dctplus_backward. The same unmodified v tensor is not copied
        to the host again."""

        @staticmethod
        def forward(ctx, x, v, rho):
            plan = _cached_plan(x.shape[1], v, rho, x.device.index or 0)
            y = plan.forward(x.contiguous())
            ctx.plan = plan
            ctx.save_for_backward(y)
            ctx.v_dtype, ctx.v_device = v.dtype, v.device
            ctx.rho_dtype = rho.dtype if torch.is_tensor(rho) else torch.float64
            return y

        @staticmethod
        def backward(ctx, gy):
            (y,) = ctx.saved_tensors
            want_x = ctx.needs_input_grad[0]
            want_p = ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
            gx, g_rho, g_v = ctx.plan.backward(gy.contiguous().float(), y, want_x=want_x,
                                               want_params=want_p)
            gv = g_v.to(ctx.v_device, ctx.v_dtype) if (g_v is not None and ctx.needs_input_grad[1]) else None
            gr = g_rho.to(ctx.rho_dtype) if (g_rho is not None and ctx.needs_input_grad[2]) else None
            return gx, gv, gr

    return DctPlusFunction


def __getattr__(name):
    if name == "DctPlusFunction":
        fn = _make_function()
        globals()["DctPlusFunction"] = fn
        return fn
    raise AttributeError(name)


def dct_plus(x, v, rho):
    """Differentiable Fast DCT+ forward: y = X(v, rho)^T x for float32 CUDA rows x."""
    import paper_2409_08970_gb300 as _self
    return _self.DctPlusFunction.apply(x, v, rho)
