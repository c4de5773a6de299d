"""Python binding of the hifcn C ABI (``include/hifcn.h``).

Argument marshalling only: every step of the solver runs in the CUDA library
``_lib/libhifcn.so``.  Vectors are torch CUDA tensors (float64, contiguous,
N = (n-1)^dim elements in lexicographic order, x fastest); PyTorch provides
device memory and the current stream.  The functions carry the names of the C
entry points and raise ``HifError`` on a non-zero status.  There is no CPU
path: if the library is missing, loading fails loudly.
"""

from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, byref, c_double, c_int, c_int64, c_size_t, c_void_p

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libhifcn.so")
_lib = None

HIF_OK, HIF_EINVAL, HIF_ENOMEM, HIF_ENOTSPD, HIF_ENOCONV, HIF_ETIMEOUT, HIF_ECUDA, HIF_EFORMAT = (
    0, -1, -2, -3, -4, -5, -6, -7)
HIF_FP64, HIF_FP32, HIF_FP32_BF16TOP = 0, 1, 2

EXPORTED = ("hif_default_options", "hif_setup", "hif_import_factor", "hif_export_factor",
            "hif_apply", "hif_matvec", "pcg_solve", "cn_step", "hif_set_reaction", "hif_query",
            "hif_destroy", "hif_strerror", "hif_last_error", "hif_stats_enable", "hif_stats_read",
            "hif_launch_count", "hif_apply_noalloc", "cn_step_batched", "hif_set_coefficient",
            "hif_refactor", "hif_autotune", "cn_steps", "hif_inject_flow_stall",
            "hif_apply_multi", "cn_step_multi", "hif_release_fp64", "hif_offload", "hif_reload")


class HifGrid(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n", c_int), ("leaf", c_int)]


class HifOptions(ctypes.Structure):
    _fields_ = [("eps", c_double), ("precision", c_int), ("skel_edges_3d", c_int),
                ("cg_tol", c_double), ("cg_maxit", c_int), ("true_res_period", c_int),
                ("theta", c_double), ("x0_mode", c_int), ("solver", c_int),
                ("bf16_top_levels", c_int)]


class HifInfo(ctypes.Structure):
    _fields_ = [("N", c_int64), ("dim", c_int), ("n", c_int), ("leaf", c_int), ("levels", c_int),
                ("root_size", c_int), ("factor_entries", c_int64), ("apply_bytes", c_int64),
                ("device_bytes", c_int64), ("precision", c_int), ("setup_seconds", c_double),
                ("sform_levels", c_int)]


class HifKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", c_int64), ("ms", c_double),
                ("bytes", c_double)]


class HifError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        detail = lib().hif_last_error().decode() if _lib is not None else ""
        msg = lib().hif_strerror(status).decode()
        super().__init__(f"{fn} failed: {msg} ({status}){': ' + detail if detail else ''}")


def lib():
    """Load libhifcn.so (built by ``paper_2004_05566_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"CUDA library {_LIB_PATH} is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(_LIB_PATH)
    L.hif_default_options.argtypes = [POINTER(HifOptions)]
    L.hif_default_options.restype = None
    L.hif_setup.argtypes = [POINTER(HifGrid), c_void_p, c_double, POINTER(HifOptions), c_void_p,
                            POINTER(c_void_p)]
    L.hif_import_factor.argtypes = [POINTER(HifGrid), c_void_p, c_size_t, c_double, c_void_p,
                                    POINTER(HifOptions), c_void_p, POINTER(c_void_p)]
    L.hif_export_factor.argtypes = [c_void_p, c_void_p, POINTER(c_size_t)]
    L.hif_apply.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_void_p]
    L.hif_matvec.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    L.pcg_solve.argtypes = [c_void_p, c_void_p, c_void_p, POINTER(c_int), POINTER(c_double), c_void_p]
    L.cn_step.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_int), c_void_p]
    L.cn_steps.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p]
    L.hif_set_reaction.argtypes = [c_void_p, c_int, c_double, c_double]
    L.hif_query.argtypes = [c_void_p, POINTER(HifInfo)]
    L.hif_destroy.argtypes = [c_void_p]
    L.hif_strerror.argtypes = [c_int]
    L.hif_strerror.restype = ctypes.c_char_p
    L.hif_last_error.argtypes = []
    L.hif_last_error.restype = ctypes.c_char_p
    L.hif_stats_enable.argtypes = [c_void_p, c_int]
    L.hif_stats_read.argtypes = [c_void_p, POINTER(HifKernelStat), c_int, POINTER(c_int)]
    L.hif_launch_count.argtypes = []
    L.hif_launch_count.restype = c_int64
    L.hif_apply_noalloc.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    L.hif_apply_noalloc.restype = c_int
    L.cn_step_batched.argtypes = [POINTER(c_void_p), c_int, POINTER(c_void_p), POINTER(c_void_p),
                                  POINTER(c_void_p), POINTER(c_int), c_void_p]
    L.cn_step_batched.restype = c_int
    L.hif_set_coefficient.argtypes = [c_void_p, c_void_p, c_void_p]
    L.hif_set_coefficient.restype = c_int
    L.hif_refactor.argtypes = [c_void_p, c_void_p, c_void_p]
    L.hif_refactor.restype = c_int
    L.hif_autotune.argtypes = [c_void_p, c_void_p]
    L.hif_autotune.restype = c_int
    L.hif_apply_multi.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_void_p]
    L.hif_apply_multi.restype = c_int
    L.cn_step_multi.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p]
    L.cn_step_multi.restype = c_int
    for name in ("hif_release_fp64", "hif_offload", "hif_reload"):
        getattr(L, name).argtypes = [c_void_p]
        getattr(L, name).restype = c_int
    L.hif_inject_flow_stall.argtypes = [c_void_p, c_int, ctypes.c_longlong]
    L.hif_inject_flow_stall.restype = c_int
    for name in ("hif_setup", "hif_import_factor", "hif_export_factor", "hif_apply", "hif_matvec",
                 "pcg_solve", "cn_step", "cn_steps", "hif_set_reaction", "hif_query", "hif_destroy",
                 "hif_stats_enable", "hif_stats_read"):
        getattr(L, name).restype = c_int
    _lib = L
    return L


def _check(fn: str, status: int, allow=()):
    if status != HIF_OK and status not in allow:
        raise HifError(fn, status)
    return status


def _stream(stream):
    if stream is None:
        return c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return c_void_p(stream.cuda_stream)
    return c_void_p(int(stream))


def _vec(t: torch.Tensor, N: int, name: str) -> c_void_p:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if not t.is_contiguous() or t.numel() != N:
        raise ValueError(f"{name} must be contiguous with {N} elements")
    if t.device.index != torch.cuda.current_device():  # the library works on the current device
        raise ValueError(f"{name} is on {t.device}, the current device is "
                         f"cuda:{torch.cuda.current_device()}")
    return c_void_p(t.data_ptr())


def default_options(**kw) -> HifOptions:
    """hif_options with the library's defaults, then the given fields set
    (eps, precision, cg_tol, cg_maxit, theta, x0_mode, solver, ...)."""
    o = HifOptions()
    lib().hif_default_options(byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Handle:
    """Owner of a hif_handle*; frees device memory on close()/garbage collection."""

    def __init__(self, ptr: c_void_p, dim: int, n: int, leaf: int):
        self._ptr = ptr
        self.dim, self.n, self.leaf = dim, n, leaf
        self.N = (n - 1) ** dim

    @property
    def ptr(self) -> c_void_p:
        if self._ptr is None:
            raise RuntimeError("handle destroyed")
        return self._ptr

    def close(self):
        if self._ptr is not None and _lib is not None:
            _lib.hif_destroy(self._ptr)
        self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        return hif_query(self)


def _grid(dim, n, leaf) -> HifGrid:
    return HifGrid(dim, n, leaf)


def hif_setup(dim: int, n: int, leaf: int, a_nodes: torch.Tensor, dt: float, opt: HifOptions = None,
              stream=None) -> Handle:
    """Factor A = I - dt/2 M on the GPU (Sec. 2.2); a_nodes: (n+1)^dim float64 CUDA tensor."""
    a = _vec(a_nodes.reshape(-1), (n + 1) ** dim, "a_nodes")
    out = c_void_p()
    g = _grid(dim, n, leaf)
    _check("hif_setup", lib().hif_setup(byref(g), a, c_double(dt), byref(opt) if opt else None,
                                        _stream(stream), byref(out)))
    return Handle(out, dim, n, leaf)


def hif_import_factor(dim: int, n: int, leaf: int, blob: bytes, dt: float, a_nodes: torch.Tensor,
                      opt: HifOptions = None, stream=None) -> Handle:
    """A handle from a factor blob (the interchange format of hif_export_factor)
    instead of factoring; a_nodes and dt give the stencil of A."""
    a = _vec(a_nodes.reshape(-1), (n + 1) ** dim, "a_nodes")
    buf = ctypes.create_string_buffer(blob, len(blob))
    out = c_void_p()
    g = _grid(dim, n, leaf)
    _check("hif_import_factor", lib().hif_import_factor(byref(g), buf, c_size_t(len(blob)),
                                                        c_double(dt), a, byref(opt) if opt else None,
                                                        _stream(stream), byref(out)))
    return Handle(out, dim, n, leaf)


def hif_export_factor(h: Handle) -> bytes:
    """The handle's FP64 factor as an interchange blob (checkpoint)."""
    nb = c_size_t(0)
    _check("hif_export_factor", lib().hif_export_factor(h.ptr, None, byref(nb)))
    buf = ctypes.create_string_buffer(nb.value)
    _check("hif_export_factor", lib().hif_export_factor(h.ptr, buf, byref(nb)))
    return buf.raw[: nb.value]


def hif_apply(h: Handle, x: torch.Tensor, y: torch.Tensor = None, precision: int = HIF_FP64,
              stream=None) -> torch.Tensor:
    """y = F^{-1} x (Eq. Ainv)."""
    if y is None:
        y = torch.empty_like(x)
    _check("hif_apply", lib().hif_apply(h.ptr, _vec(x, h.N, "x"), _vec(y, h.N, "y"), precision,
                                        _stream(stream)))
    return y


def hif_apply_noalloc(h: Handle, x: torch.Tensor, y: torch.Tensor = None,
                      stream=None) -> torch.Tensor:
    """y = F^{-1} x in FP64 with the library's static scratch (no device allocation in the
    call; see include/hifcn.h).  If y is None it is allocated here by torch, before the call."""
    if y is None:
        y = torch.empty_like(x)
    _check("hif_apply_noalloc", lib().hif_apply_noalloc(h.ptr, _vec(x, h.N, "x"), _vec(y, h.N, "y"),
                                                        _stream(stream)))
    return y


HIF_MULTI_MAX_COLS = 64


def hif_apply_multi(h: Handle, X: torch.Tensor, Y: torch.Tensor = None, stream=None) -> torch.Tensor:
    """Y = F^{-1} X for the k columns of X (a (k, N) float64 CUDA tensor, one
    right-hand side per row, i.e. the columns stored one after another); the
    BF16 top levels and the root run as tensor-core products for all k at once.
    Needs a handle set up with HIF_FP32_BF16TOP."""
    if X.dim() != 2 or X.shape[1] != h.N:
        raise ValueError(f"X must have shape (k, {h.N})")
    k = X.shape[0]
    if Y is None:
        Y = torch.empty_like(X)
    _check("hif_apply_multi", lib().hif_apply_multi(h.ptr, _vec(X.reshape(-1), k * h.N, "X"),
                                                    _vec(Y.reshape(-1), k * h.N, "Y"), int(k),
                                                    _stream(stream)))
    return Y


def cn_step_multi(h: Handle, U: torch.Tensor, R: torch.Tensor = None, out: torch.Tensor = None,
                  stream=None):
    """One CN step for each row of U ((k, N) float64 CUDA tensor: k states of
    the same operator), the k PCG solves sharing each multi-column apply;
    returns (U1, iters per state)."""
    if U.dim() != 2 or U.shape[1] != h.N:
        raise ValueError(f"U must have shape (k, {h.N})")
    k = U.shape[0]
    if out is None:
        out = torch.empty_like(U)
    rp = _vec(R.reshape(-1), k * h.N, "R") if R is not None else None
    its = (c_int * k)()
    _check("cn_step_multi", lib().cn_step_multi(h.ptr, _vec(U.reshape(-1), k * h.N, "U"), rp,
                                                _vec(out.reshape(-1), k * h.N, "out"), int(k), its,
                                                _stream(stream)))
    return out, [its[i] for i in range(k)]


def hif_matvec(h: Handle, x: torch.Tensor, y: torch.Tensor = None, stream=None) -> torch.Tensor:
    """y = A x, A = I - dt/2 M (Eq. CN)."""
    if y is None:
        y = torch.empty_like(x)
    _check("hif_matvec", lib().hif_matvec(h.ptr, _vec(x, h.N, "x"), _vec(y, h.N, "y"),
                                          _stream(stream)))
    return y


def pcg_solve(h: Handle, b: torch.Tensor, x: torch.Tensor = None, stream=None, allow_noconv=False):
    """Solve A x = b by F^{-1}-preconditioned CG; returns (x, iters, relres).

    With options.x0_mode = 1 the incoming x is the initial guess (zeros when
    x is None); with options.solver = 1, x = F^{-1} b and iters = 0."""
    if x is None:
        x = torch.zeros_like(b)
    it = c_int(0)
    rr = c_double(0.0)
    _check("pcg_solve", lib().pcg_solve(h.ptr, _vec(b, h.N, "b"), _vec(x, h.N, "x"), byref(it),
                                        byref(rr), _stream(stream)),
           allow=(HIF_ENOCONV,) if allow_noconv else ())
    return x, it.value, rr.value


def cn_step(h: Handle, u: torch.Tensor, r: torch.Tensor = None, out: torch.Tensor = None,
            stream=None):
    """One Crank-Nicolson step (Eq. CN2); returns (u_next, iters)."""
    if out is None:
        out = torch.empty_like(u)
    it = c_int(0)
    rp = _vec(r, h.N, "r") if r is not None else None
    _check("cn_step", lib().cn_step(h.ptr, _vec(u, h.N, "u"), rp, _vec(out, h.N, "out"), byref(it),
                                    _stream(stream)))
    return out, it.value


def cn_steps(h: Handle, u: torch.Tensor, nsteps: int, r: torch.Tensor = None, stream=None) -> list:
    """nsteps CN steps of u in place, queued without host synchronization
    between steps; returns the PCG iterations of each step."""
    its = (c_int * max(nsteps, 1))()
    rp = _vec(r, h.N, "r") if r is not None else None
    _check("cn_steps", lib().cn_steps(h.ptr, _vec(u, h.N, "u"), rp, int(nsteps), its, _stream(stream)))
    return [its[i] for i in range(nsteps)]


def cn_step_batched(hs, us, rs=None, outs=None, stream=None):
    """One CN step for each handle (independent problems, overlapped on the GPU).

    hs: list of Handles; us: list of device vectors; rs: list (entries may be
    None) or None; outs: list of outputs or None (allocated here by torch).
    Returns (outs, iters)."""
    n = len(hs)
    if len(us) != n or (rs is not None and len(rs) != n):
        raise ValueError("hs, us and rs must have the same length")
    if outs is None:
        outs = [torch.empty_like(u) for u in us]
    H = (c_void_p * n)(*[h.ptr for h in hs])
    U = (c_void_p * n)(*[_vec(u, h.N, "u") for u, h in zip(us, hs)])
    O = (c_void_p * n)(*[_vec(o, h.N, "out") for o, h in zip(outs, hs)])
    R = None
    if rs is not None:
        R = (c_void_p * n)(*[(_vec(r, h.N, "r") if r is not None else None) for r, h in zip(rs, hs)])
    it = (c_int * n)()
    _check("cn_step_batched", lib().cn_step_batched(H, n, U, R, O, it, _stream(stream)))
    return outs, list(it)


def hif_set_coefficient(h: Handle, a_nodes: torch.Tensor, stream=None):
    """Replace a(x); the current factor stays as the preconditioner."""
    a = _vec(a_nodes.reshape(-1), (h.n + 1) ** h.dim, "a_nodes")
    _check("hif_set_coefficient", lib().hif_set_coefficient(h.ptr, a, _stream(stream)))


def hif_refactor(h: Handle, a_nodes: torch.Tensor, stream=None):
    """Replace a(x) and factor the new operator in place."""
    a = _vec(a_nodes.reshape(-1), (h.n + 1) ** h.dim, "a_nodes")
    _check("hif_refactor", lib().hif_refactor(h.ptr, a, _stream(stream)))


def hif_autotune(h: Handle, stream=None):
    """Pick the per-level CTA cut of the apply and the leaf kernels' CTAs per SM by timing."""
    _check("hif_autotune", lib().hif_autotune(h.ptr, _stream(stream)))


def hif_release_fp64(h: Handle):
    """Free the FP64 factor values of an FP32 / BF16TOP handle (its solves use FP32)."""
    _check("hif_release_fp64", lib().hif_release_fp64(h.ptr))


def hif_offload(h: Handle):
    """Move the handle's large device allocations to host memory (addresses kept)."""
    _check("hif_offload", lib().hif_offload(h.ptr))


def hif_reload(h: Handle):
    """Map device memory at the same addresses again and copy the contents back."""
    _check("hif_reload", lib().hif_reload(h.ptr))


def hif_inject_flow_stall(h: Handle, unit: int, polls: int = 0):
    """Failure injection (tests): unit `unit` of the dependency-driven sweep never
    publishes its flag, so its dependents' waits expire after `polls` polls and
    the next solve returns HIF_ETIMEOUT; unit = -1 ends the injection."""
    _check("hif_inject_flow_stall", lib().hif_inject_flow_stall(h.ptr, int(unit), int(polls)))


def hif_set_reaction(h: Handle, kind: int, k1: float = 1.0, k2: float = math.inf):
    """Explicit reaction of the right-hand side (Eq. nr): kind 1 is
    k1 u (1 - u/k2) (k2 = inf: linear k1 u), kind 0 none."""
    _check("hif_set_reaction", lib().hif_set_reaction(h.ptr, kind, c_double(k1), c_double(k2)))


def hif_query(h: Handle) -> dict:
    """Sizes of the handle: N, levels, root size, factor entries, apply bytes,
    device bytes, setup seconds, S-form levels."""
    info = HifInfo()
    _check("hif_query", lib().hif_query(h.ptr, byref(info)))
    return {k: getattr(info, k) for k, _ in HifInfo._fields_}


def hif_destroy(h: Handle):
    """Free the handle's device memory (the same as h.close())."""
    h.close()


def hif_stats_enable(h: Handle, on: bool = True):
    """Bracket every apply-path kernel launch with CUDA events (measurement)."""
    _check("hif_stats_enable", lib().hif_stats_enable(h.ptr, 1 if on else 0))


def hif_stats_read(h: Handle) -> list:
    """Per-kernel launches, device ms and algorithmic bytes since the last read."""
    cnt = c_int(0)
    _check("hif_stats_read", lib().hif_stats_read(h.ptr, None, 0, byref(cnt)))
    n = max(cnt.value, 1)
    arr = (HifKernelStat * n)()
    _check("hif_stats_read", lib().hif_stats_read(h.ptr, arr, n, byref(cnt)))
    return [dict(name=a.name.decode(), launches=a.launches, ms=a.ms, bytes=a.bytes)
            for a in arr[: cnt.value]]


def hif_launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().hif_launch_count())
