"""Python binding of libgbpcg.so (ctypes): argument marshalling only.

Every function here converts torch tensors / numbers into the C ABI of
``include/gbpcg.h`` and calls it; all arithmetic runs in the library's CUDA
kernels.  There is no CPU path: if the library cannot be loaded the call
raises.

Grids are torch tensors of shape (nz, ny, nx) (x fastest), matching the
library's index (k*ny + j)*nx + i.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgbpcg.so")

OK, ERR_ARG, ERR_CUDA, NOT_CONVERGED, BREAKDOWN, TIMEOUT, FALLBACK_USED = range(7)
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "NOT_CONVERGED", 4: "BREAKDOWN", 5: "TIMEOUT",
                6: "FALLBACK_USED"}
F32, BF16, F16, F64 = 0, 1, 2, 3
FLAG_HOST_IO = 1
FLAG_PROFILE = 2
FLAG_AUTOTUNE = 4
FLAG_HOST_LOOP = 8
FLAG_SPLIT = 16
FLAG_BATCH_GRAPH = 32
_MODES = {"graph": 0, "host_loop": FLAG_HOST_LOOP, "split": FLAG_SPLIT}

_DTYPES = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16, torch.float64: F64}

EXPORTS = ["gbpcg_version", "gbpcg_last_error", "gbpcg_dot_workspace_size", "gbpcg_stencil_apply", "gbpcg_dot",
           "gbpcg_dot_noalloc", "gbpcg_axpy", "gbpcg_tile_config", "gbpcg_workspace_size", "gbpcg_pcg_solve",
           "gbpcg_workspace_size_batched", "gbpcg_pcg_solve_batched", "gbpcg_autotune", "gbpcg_autotune_record",
           "gbpcg_conv3_workspace_size", "gbpcg_conv3_forward", "gbpcg_conv3_backward_data",
           "gbpcg_conv3_backward_weight", "gbpcg_nn_workspace_size", "gbpcg_nn_forward", "gbpcg_nn_backward",
           "gbpcg_nn_loss", "gbpcg_nn_adam", "gbpcg_nn_train_step", "gbpcg_nn_status", "gbpcg_fcg_workspace_size",
           "gbpcg_fcg_solve", "gbpcg_wait_selftest", "gbpcg_nn_tensor_info", "gbpcg_dot_variant_workspace_size",
           "gbpcg_dot_variant", "gbpcg_stencil_apply_variant", "gbpcg_sell_stencil_layout", "gbpcg_sell_from_stencil",
           "gbpcg_sell_csr_layout", "gbpcg_sell_from_csr", "gbpcg_sell_spmv", "gbpcg_sell_workspace_size",
           "gbpcg_sell_pcg_solve", "gbpcg_mg_workspace_size", "gbpcg_mg_vcycle", "gbpcg_mg_pcg_solve"]
PRECOND_JACOBI, PRECOND_LEARNED, PRECOND_MG = 0, 1, 2

NN_NUM_WEIGHTS = 319248
# (name, input channels, output channels) of the U-net's layers, in weight-array order
NN_LAYERS = [("c1", 2, 16), ("c2", 16, 16), ("c3", 16, 32), ("c4", 32, 32), ("c5", 32, 64), ("c6", 64, 64),
             ("c7", 96, 32), ("c8", 48, 16), ("c9", 16, 1)]


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("k_block", ctypes.c_void_p), ("kbx", ctypes.c_int32), ("kby", ctypes.c_int32),
                ("kbz", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("io_dtype", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("tile_cfg", ctypes.c_int32), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int32), ("fcg_m", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("rel_res_recursive", ctypes.c_double),
                ("rel_res_true", ctypes.c_double), ("time_ms", ctypes.c_double),
                ("pass_ms", ctypes.c_double * 2), ("pass_launches", ctypes.c_int32 * 2),
                ("replacements", ctypes.c_int32), ("refine_steps", ctypes.c_int32),
                ("pass_ctas", ctypes.c_int32 * 2)]

    def as_dict(self):
        return dict(iters=self.iters, status=self.status, status_name=STATUS_NAMES.get(self.status, "?"),
                    rel_res_recursive=self.rel_res_recursive, rel_res_true=self.rel_res_true,
                    time_ms=self.time_ms, pass_ms=list(self.pass_ms), pass_launches=list(self.pass_launches),
                    replacements=self.replacements, refine_steps=self.refine_steps, pass_ctas=list(self.pass_ctas))


class Sell(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("slice", ctypes.c_int32), ("slice_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("inv_diag", ctypes.c_void_p)]


class SellMatrix:
    """Device arrays of a SELL-32 matrix (gbpcg_sell) and the C struct that points at them."""

    def __init__(self, n, slice_ptr, col, val, inv_diag):
        self.n, self.slice_ptr, self.col, self.val, self.inv_diag = n, slice_ptr, col, val, inv_diag
        self.c = Sell(n, 32, slice_ptr.data_ptr(), col.data_ptr(), val.data_ptr(), inv_diag.data_ptr())

    @property
    def nnz_stored(self):
        return self.val.numel()


class GbpcgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gbpcg status {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Loads the CUDA library (building it in-tree first if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            from . import build as _build
            _build.build()
        lib = ctypes.CDLL(path)
        P, I32, I64, D, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
        lib.gbpcg_version.restype = ctypes.c_char_p
        lib.gbpcg_last_error.restype = ctypes.c_char_p
        lib.gbpcg_dot_workspace_size.restype = SZ
        lib.gbpcg_stencil_apply.restype = ctypes.c_int
        lib.gbpcg_stencil_apply.argtypes = [ctypes.POINTER(Grid), I32, P, P, P]
        lib.gbpcg_dot.restype = ctypes.c_int
        lib.gbpcg_dot.argtypes = [I64, I32, P, P, P, P, SZ, P]
        lib.gbpcg_dot_noalloc.restype = ctypes.c_int
        lib.gbpcg_dot_noalloc.argtypes = [I64, I32, P, P, P, P]
        lib.gbpcg_axpy.restype = ctypes.c_int
        lib.gbpcg_axpy.argtypes = [I64, I32, D, P, P, P]
        lib.gbpcg_tile_config.restype = ctypes.c_int
        lib.gbpcg_tile_config.argtypes = [I32, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)]
        lib.gbpcg_workspace_size.restype = ctypes.c_int
        lib.gbpcg_workspace_size.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Opts), ctypes.POINTER(SZ)]
        lib.gbpcg_pcg_solve.restype = ctypes.c_int
        lib.gbpcg_pcg_solve.argtypes = [ctypes.POINTER(Grid), P, P, ctypes.POINTER(Opts), ctypes.POINTER(Result), P]
        lib.gbpcg_workspace_size_batched.restype = ctypes.c_int
        lib.gbpcg_workspace_size_batched.argtypes = [I32, ctypes.POINTER(Grid), ctypes.POINTER(Opts),
                                                     ctypes.POINTER(SZ)]
        lib.gbpcg_pcg_solve_batched.restype = ctypes.c_int
        lib.gbpcg_pcg_solve_batched.argtypes = [I32, ctypes.POINTER(Grid), ctypes.POINTER(P), ctypes.POINTER(P),
                                                ctypes.POINTER(Opts), ctypes.POINTER(Result), P]
        lib.gbpcg_autotune.restype = ctypes.c_int
        lib.gbpcg_autotune.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Opts), P, ctypes.POINTER(I32),
                                       ctypes.POINTER(D), P]
        lib.gbpcg_autotune_record.restype = ctypes.c_int
        lib.gbpcg_autotune_record.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Opts), I32]
        lib.gbpcg_conv3_workspace_size.restype = ctypes.c_int
        lib.gbpcg_conv3_workspace_size.argtypes = [I32, I32, I32, I32, I32, ctypes.POINTER(SZ)]
        for name in ("gbpcg_conv3_backward_data", "gbpcg_conv3_backward_weight"):
            getattr(lib, name).restype = ctypes.c_int
            getattr(lib, name).argtypes = [I32, I32, I32, I32, I32, P, P, P, P, SZ, P]
        lib.gbpcg_conv3_forward.restype = ctypes.c_int
        lib.gbpcg_conv3_forward.argtypes = [I32, I32, I32, I32, I32, P, P, P, I32, P, SZ, P]
        lib.gbpcg_nn_workspace_size.restype = ctypes.c_int
        lib.gbpcg_nn_workspace_size.argtypes = [I32, I32, I32, I32, ctypes.POINTER(SZ)]
        lib.gbpcg_nn_forward.restype = ctypes.c_int
        lib.gbpcg_nn_tensor_info.argtypes = [I32, I32, I32, I32, I32, ctypes.POINTER(SZ), ctypes.POINTER(I32),
                                             ctypes.POINTER(I32), ctypes.POINTER(I32)]
        lib.gbpcg_nn_tensor_info.restype = ctypes.c_int
        lib.gbpcg_dot_variant_workspace_size.restype = SZ
        lib.gbpcg_dot_variant_workspace_size.argtypes = []
        lib.gbpcg_dot_variant.argtypes = [I32, I64, P, P, P, P, SZ, P]
        lib.gbpcg_dot_variant.restype = ctypes.c_int
        lib.gbpcg_stencil_apply_variant.argtypes = [ctypes.POINTER(Grid), I32, P, P, P]
        lib.gbpcg_stencil_apply_variant.restype = ctypes.c_int
        lib.gbpcg_sell_stencil_layout.argtypes = [ctypes.POINTER(Grid), P, ctypes.POINTER(I64), P]
        lib.gbpcg_sell_from_stencil.argtypes = [ctypes.POINTER(Grid), P, P, P, P, P]
        lib.gbpcg_sell_csr_layout.argtypes = [I64, P, P, ctypes.POINTER(I64), P]
        lib.gbpcg_sell_from_csr.argtypes = [I64, P, P, P, P, P, P, P, P]
        lib.gbpcg_sell_spmv.argtypes = [ctypes.POINTER(Sell), P, P, P]
        lib.gbpcg_sell_workspace_size.argtypes = [ctypes.POINTER(Sell), ctypes.POINTER(SZ)]
        lib.gbpcg_sell_pcg_solve.argtypes = [ctypes.POINTER(Sell), P, P, ctypes.POINTER(Opts), ctypes.POINTER(Result),
                                             P]
        for name in ("gbpcg_sell_stencil_layout", "gbpcg_sell_from_stencil", "gbpcg_sell_csr_layout",
                     "gbpcg_sell_from_csr", "gbpcg_sell_spmv", "gbpcg_sell_workspace_size", "gbpcg_sell_pcg_solve"):
            getattr(lib, name).restype = ctypes.c_int
        lib.gbpcg_mg_workspace_size.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(SZ)]
        lib.gbpcg_mg_vcycle.argtypes = [ctypes.POINTER(Grid), P, P, P, SZ, ctypes.POINTER(I32), P]
        lib.gbpcg_mg_pcg_solve.argtypes = [ctypes.POINTER(Grid), P, P, ctypes.POINTER(Opts), ctypes.POINTER(Result), P]
        for name in ("gbpcg_mg_workspace_size", "gbpcg_mg_vcycle", "gbpcg_mg_pcg_solve"):
            getattr(lib, name).restype = ctypes.c_int
        lib.gbpcg_nn_forward.argtypes = [ctypes.POINTER(Grid), P, P, P, P, SZ, P]
        lib.gbpcg_nn_backward.restype = ctypes.c_int
        lib.gbpcg_nn_backward.argtypes = [ctypes.POINTER(Grid), P, P, P, SZ, P]
        lib.gbpcg_nn_loss.restype = ctypes.c_int
        lib.gbpcg_nn_loss.argtypes = [ctypes.POINTER(Grid), P, P, P, P, P, SZ, P]
        lib.gbpcg_nn_adam.restype = ctypes.c_int
        lib.gbpcg_nn_adam.argtypes = [I64, P, P, P, P, I32, D, D, D, D, P]
        lib.gbpcg_nn_train_step.restype = ctypes.c_int
        lib.gbpcg_nn_train_step.argtypes = [ctypes.POINTER(Grid), P, P, P, I32, D, P, P, P, P, P, P, P, SZ, P]
        lib.gbpcg_nn_status.restype = ctypes.c_int
        lib.gbpcg_nn_status.argtypes = [P, P]
        lib.gbpcg_fcg_workspace_size.restype = ctypes.c_int
        lib.gbpcg_fcg_workspace_size.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Opts), ctypes.POINTER(SZ)]
        lib.gbpcg_wait_selftest.restype = ctypes.c_int
        lib.gbpcg_wait_selftest.argtypes = [I32, ctypes.c_uint32, P, ctypes.POINTER(D), P]
        lib.gbpcg_fcg_solve.restype = ctypes.c_int
        lib.gbpcg_fcg_solve.argtypes = [ctypes.POINTER(Grid), P, P, P, ctypes.POINTER(Opts), ctypes.POINTER(Result), P]
        _lib = lib
        return lib


def version() -> str:
    return load().gbpcg_version().decode()


def last_error() -> str:
    return load().gbpcg_last_error().decode()


def _check(rc: int, allowed=(OK,)):
    if rc not in allowed:
        raise GbpcgError(rc, last_error())
    return rc


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _dtype(t: torch.Tensor) -> int:
    try:
        return _DTYPES[t.dtype]
    except KeyError:
        raise GbpcgError(ERR_ARG, f"unsupported dtype {t.dtype}") from None


def make_grid(shape, k_block: torch.Tensor | None = None, kb=8) -> Grid:
    nz, ny, nx = (int(s) for s in shape)
    if isinstance(kb, int):
        kb = (kb, kb, kb)
    g = Grid(nx, ny, nz, None, 1, 1, 1)
    if k_block is not None:
        if k_block.dtype != torch.float32 or not k_block.is_cuda or not k_block.is_contiguous():
            raise GbpcgError(ERR_ARG, "k_block must be a contiguous float32 CUDA tensor")
        g.k_block = k_block.data_ptr()
        g.kbx, g.kby, g.kbz = (int(v) for v in kb)
    return g


def stencil_apply(p: torch.Tensor, q: torch.Tensor | None = None, k_block=None, kb=8, stream=None) -> torch.Tensor:
    """q = A p (gbpcg_stencil_apply)."""
    if p.dim() != 3 or not p.is_contiguous():
        raise GbpcgError(ERR_ARG, "p must be a contiguous (nz, ny, nx) tensor")
    if q is None:
        q = torch.empty_like(p)
    g = make_grid(p.shape, k_block, kb)
    _check(load().gbpcg_stencil_apply(ctypes.byref(g), _dtype(p), _ptr(p), _ptr(q), _stream(stream)))
    return q


def dot_workspace_size() -> int:
    return int(load().gbpcg_dot_workspace_size())


def dot(x: torch.Tensor, y: torch.Tensor, out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
        stream=None) -> torch.Tensor:
    """Device scalar (float64 tensor) x . y (gbpcg_dot)."""
    if x.numel() != y.numel() or x.dtype != y.dtype:
        raise GbpcgError(ERR_ARG, "x and y must have the same size and dtype")
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=x.device)
    if workspace is None:
        workspace = torch.empty(dot_workspace_size(), dtype=torch.uint8, device=x.device)
    _check(load().gbpcg_dot(x.numel(), _dtype(x), _ptr(x), _ptr(y), _ptr(out), _ptr(workspace),
                            workspace.numel(), _stream(stream)))
    return out


def dot_noalloc(x: torch.Tensor, y: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """x . y through gbpcg_dot_noalloc, which takes no workspace and allocates
    nothing: its scratch is a static array inside the library (calls must not
    overlap on the GPU).  ``out`` is the caller's float64 device scalar."""
    if x.numel() != y.numel() or x.dtype != y.dtype:
        raise GbpcgError(ERR_ARG, "x and y must have the same size and dtype")
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=x.device)
    _check(load().gbpcg_dot_noalloc(x.numel(), _dtype(x), _ptr(x), _ptr(y), _ptr(out), _stream(stream)))
    return out


def dot_variant(variant: int, x: torch.Tensor, y: torch.Tensor, out: torch.Tensor | None = None,
                workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """x.y (FP32, 16-byte aligned) with reduction variant 0..4 (gbpcg_dot_variant)."""
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=x.device)
    if workspace is None:
        workspace = torch.empty(load().gbpcg_dot_variant_workspace_size(), dtype=torch.uint8, device=x.device)
    _check(load().gbpcg_dot_variant(int(variant), x.numel(), _ptr(x), _ptr(y), _ptr(out), _ptr(workspace),
                                    workspace.numel(), _stream(stream)))
    return out


def stencil_apply_variant(variant: int, p: torch.Tensor, q: torch.Tensor | None = None, stream=None):
    """q = A p (FP32, constant coefficient) with boundary variant 0..2 (gbpcg_stencil_apply_variant)."""
    if q is None:
        q = torch.empty_like(p)
    g = make_grid(p.shape)
    _check(load().gbpcg_stencil_apply_variant(ctypes.byref(g), int(variant), _ptr(p), _ptr(q), _stream(stream)))
    return q


def sell_from_stencil(shape, k_block=None, kb=8, device="cuda", stream=None) -> SellMatrix:
    """The seven-point operator of a grid as a SELL-32 matrix on the device
    (gbpcg_sell_stencil_layout + gbpcg_sell_from_stencil)."""
    g = make_grid(shape, k_block, kb)
    nnz = ctypes.c_int64(0)
    lib = load()
    _check(lib.gbpcg_sell_stencil_layout(ctypes.byref(g), None, ctypes.byref(nnz), _stream(stream)))
    n = int(np.prod(shape))
    sp = torch.empty((n + 31) // 32 + 1, dtype=torch.int64, device=device)
    _check(lib.gbpcg_sell_stencil_layout(ctypes.byref(g), _ptr(sp), ctypes.byref(nnz), _stream(stream)))
    col = torch.empty(nnz.value, dtype=torch.int32, device=device)
    val = torch.empty(nnz.value, dtype=torch.float32, device=device)
    inv = torch.empty(n, dtype=torch.float32, device=device)
    _check(lib.gbpcg_sell_from_stencil(ctypes.byref(g), _ptr(sp), _ptr(col), _ptr(val), _ptr(inv), _stream(stream)))
    return SellMatrix(n, sp, col, val, inv)


def sell_from_csr(row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, stream=None) -> SellMatrix:
    """A CSR matrix (CUDA row_ptr int64, col int32, val float32) as SELL-32 (gbpcg_sell_csr_layout +
    gbpcg_sell_from_csr)."""
    n = row_ptr.numel() - 1
    lib = load()
    nnz = ctypes.c_int64(0)
    sp = torch.empty((n + 31) // 32 + 1, dtype=torch.int64, device=row_ptr.device)
    _check(lib.gbpcg_sell_csr_layout(n, _ptr(row_ptr), _ptr(sp), ctypes.byref(nnz), _stream(stream)))
    scol = torch.empty(nnz.value, dtype=torch.int32, device=row_ptr.device)
    sval = torch.empty(nnz.value, dtype=torch.float32, device=row_ptr.device)
    inv = torch.empty(n, dtype=torch.float32, device=row_ptr.device)
    _check(lib.gbpcg_sell_from_csr(n, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(sp), _ptr(scol), _ptr(sval),
                                   _ptr(inv), _stream(stream)))
    return SellMatrix(n, sp, scol, sval, inv)


def sell_spmv(m: SellMatrix, x: torch.Tensor, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """y = A x, FP32 (gbpcg_sell_spmv)."""
    if y is None:
        y = torch.empty_like(x)
    _check(load().gbpcg_sell_spmv(ctypes.byref(m.c), _ptr(x), _ptr(y), _stream(stream)))
    return y


def sell_pcg_solve(m: SellMatrix, b: torch.Tensor, x: torch.Tensor | None = None, tol=1e-6, maxit=2000,
                   workspace=None, stream=None):
    """Jacobi-PCG on a SELL matrix (gbpcg_sell_pcg_solve); b, x float64 CUDA vectors."""
    if x is None:
        x = torch.zeros_like(b)
    lib = load()
    if workspace is None:
        nb = ctypes.c_size_t(0)
        _check(lib.gbpcg_sell_workspace_size(ctypes.byref(m.c), ctypes.byref(nb)))
        workspace = torch.empty(nb.value, dtype=torch.uint8, device=b.device)
    o = make_opts(tol, maxit, F32, F64, False, workspace)
    r = Result()
    rc = lib.gbpcg_sell_pcg_solve(ctypes.byref(m.c), _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(r),
                                  _stream(stream))
    _check(rc, allowed=(OK, NOT_CONVERGED, BREAKDOWN, TIMEOUT))
    return x, r.as_dict()


def mg_workspace(shape, k_block=None, kb=8, device="cuda") -> torch.Tensor:
    g = make_grid(shape, k_block, kb)
    n = ctypes.c_size_t(0)
    _check(load().gbpcg_mg_workspace_size(ctypes.byref(g), ctypes.byref(n)))
    return torch.empty(n.value, dtype=torch.uint8, device=device)


def mg_vcycle(r: torch.Tensor, z: torch.Tensor | None = None, k_block=None, kb=8, workspace=None, stream=None):
    """(z = M r, levels): one multigrid V-cycle, r float32 (nz, ny, nx) (gbpcg_mg_vcycle)."""
    if z is None:
        z = torch.empty_like(r)
    ws = workspace if workspace is not None else mg_workspace(r.shape, k_block, kb, r.device)
    g = make_grid(r.shape, k_block, kb)
    lv = ctypes.c_int32(0)
    _check(load().gbpcg_mg_vcycle(ctypes.byref(g), _ptr(r), _ptr(z), _ptr(ws), ws.numel(), ctypes.byref(lv),
                                  _stream(stream)))
    return z, lv.value


def mg_pcg_solve(b: torch.Tensor, x: torch.Tensor | None = None, tol=1e-6, maxit=2000, k_block=None, kb=8,
                 workspace=None, stream=None):
    """PCG with the multigrid preconditioner (gbpcg_mg_pcg_solve); b, x float64 (nz, ny, nx)."""
    if x is None:
        x = torch.zeros_like(b)
    ws = workspace if workspace is not None else mg_workspace(b.shape, k_block, kb, b.device)
    g = make_grid(b.shape, k_block, kb)
    o = make_opts(tol, maxit, F32, F64, False, ws)
    o.precond = PRECOND_MG
    r = Result()
    rc = load().gbpcg_mg_pcg_solve(ctypes.byref(g), _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(r),
                                   _stream(stream))
    _check(rc, allowed=(OK, NOT_CONVERGED, BREAKDOWN, TIMEOUT))
    return x, r.as_dict()


def axpy(alpha: float, x: torch.Tensor, y: torch.Tensor, stream=None) -> torch.Tensor:
    """y = alpha x + y in place (gbpcg_axpy)."""
    if x.numel() != y.numel() or x.dtype != y.dtype:
        raise GbpcgError(ERR_ARG, "x and y must have the same size and dtype")
    _check(load().gbpcg_axpy(x.numel(), _dtype(x), float(alpha), _ptr(x), _ptr(y), _stream(stream)))
    return y


def tile_configs():
    """[(tx, ty, stages), ...] of the data passes' tile configurations."""
    out = []
    lib = load()
    while True:
        tx, ty, st = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        if lib.gbpcg_tile_config(len(out), ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(st)) != OK:
            return out
        out.append((tx.value, ty.value, st.value))


def tile_cfg_code(cfg_a=None, cfg_b=None) -> int:
    """gbpcg_opts.tile_cfg for explicit pass-A / pass-B configuration indices."""
    return (0 if cfg_a is None else cfg_a + 1) | ((0 if cfg_b is None else cfg_b + 1) << 8)


def make_opts(tol=1e-6, maxit=2000, storage=F32, io_dtype=F32, host_io=False, workspace=None,
              profile=False, tile_cfg=0, inner_tol=0.0, max_outer=30, autotune=False, mode="graph") -> Opts:
    """gbpcg_opts; mode "graph" (the device-driven CUDA-graph loop), "host_loop" (GBPCG_FLAG_HOST_LOOP)
    or "split" (GBPCG_FLAG_SPLIT)."""
    o = Opts()
    o.tol = float(tol)
    o.maxit = int(maxit)
    o.precond = 0
    o.storage = storage
    o.io_dtype = io_dtype
    o.flags = (FLAG_HOST_IO if host_io else 0) | (FLAG_PROFILE if profile else 0) | (FLAG_AUTOTUNE if autotune else 0)
    o.flags |= _MODES[mode]
    o.tile_cfg = int(tile_cfg)
    o.inner_tol = float(inner_tol)
    o.max_outer = int(max_outer)
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    return o


def workspace_size(shape, k_block=None, kb=8, **opt_kw) -> int:
    g = make_grid(shape, k_block, kb)
    o = make_opts(**opt_kw)
    n = ctypes.c_size_t(0)
    _check(load().gbpcg_workspace_size(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)))
    return int(n.value)


def alloc_workspace(shape, k_block=None, kb=8, device="cuda", **opt_kw) -> torch.Tensor:
    """Caller-owned device workspace for gbpcg_pcg_solve (make_opts keywords)."""
    return torch.empty(workspace_size(shape, k_block, kb, **opt_kw), dtype=torch.uint8, device=device)


def pcg_solve(b: torch.Tensor, x: torch.Tensor | None = None, tol=1e-6, maxit=2000, k_block=None, kb=8,
              workspace: torch.Tensor | None = None, host_io=False, profile=False, tile_cfg=0, storage=None,
              inner_tol=0.0, max_outer=30, mode="graph", stream=None):
    """Jacobi-PCG solve of A x = b (gbpcg_pcg_solve).  Returns (x, result dict).

    b and x are float32 or float64 (the solution accumulates in that type; the
    iteration vectors are float32 either way).  They may be CPU tensors
    (pinned for speed) when host_io=True; the
    copies then happen inside the library call.  profile=True runs the
    iteration kernels one by one, each timed with CUDA events, and reports
    the summed pass times in result["pass_ms"].  storage=torch.bfloat16 or
    torch.float16 (with float64 b and x) selects mixed precision: FP64
    iterative refinement around 16-bit inner solves to inner_tol (0: the library's default,
    0.1 for BF16 and 1e-2 for FP16).  mode="host_loop" or "split" selects the paper's
    host-readback variants (GBPCG_FLAG_HOST_LOOP, GBPCG_FLAG_SPLIT).
    """
    if b.dim() != 3 or not b.is_contiguous():
        raise GbpcgError(ERR_ARG, "b must be a contiguous (nz, ny, nx) tensor")
    if x is None:
        x = torch.zeros_like(b)
    if x.dtype != b.dtype or x.shape != b.shape or not x.is_contiguous():
        raise GbpcgError(ERR_ARG, "x must be a contiguous tensor of b's shape and dtype")
    io = _dtype(b)
    st = F32 if storage is None else _DTYPES[storage]
    dev = b.device if b.is_cuda else torch.device("cuda", torch.cuda.current_device())
    if workspace is None:
        workspace = alloc_workspace(b.shape, k_block, kb, device=dev, io_dtype=io, host_io=host_io, storage=st,
                                    inner_tol=inner_tol, max_outer=max_outer, mode=mode)
    g = make_grid(b.shape, k_block, kb)
    o = make_opts(tol, maxit, st, io, host_io, workspace, profile, tile_cfg, inner_tol, max_outer, mode=mode)
    r = Result()
    rc = load().gbpcg_pcg_solve(ctypes.byref(g), _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(r),
                                _stream(stream))
    _check(rc, allowed=(OK, NOT_CONVERGED, BREAKDOWN, TIMEOUT))
    return x, r.as_dict()


def pcg_solve_batched(bs, xs=None, tol=1e-6, maxit=2000, tile_cfg=0, autotune=False, workspace=None,
                      graph=False, stream=None):
    """Solves len(bs) independent problems in one launch (gbpcg_pcg_solve_batched): one persistent
    kernel for constant-coefficient grids (tile_cfg 1..3 picks its tiles), or with graph=True
    (GBPCG_FLAG_BATCH_GRAPH) one CUDA graph with a branch per problem.

    bs, xs: lists of contiguous (nz, ny, nx) CUDA tensors (all float32 or all
    float64).  Returns (xs, [result dict per problem]).
    """
    n = len(bs)
    if xs is None:
        xs = [torch.zeros_like(b) for b in bs]
    io = _dtype(bs[0])
    for b, x in zip(bs, xs):
        if b.dtype != bs[0].dtype or x.dtype != b.dtype or x.shape != b.shape or not (b.is_cuda and x.is_cuda):
            raise GbpcgError(ERR_ARG, "b and x must be CUDA tensors of one dtype and matching shapes")
    grids = (Grid * n)(*[make_grid(b.shape) for b in bs])
    o = make_opts(tol, maxit, F32, io, False, None, False, tile_cfg, autotune=autotune)
    if graph:
        o.flags |= FLAG_BATCH_GRAPH
    lib = load()
    if workspace is None:
        nbytes = ctypes.c_size_t(0)
        _check(lib.gbpcg_workspace_size_batched(n, grids, ctypes.byref(o), ctypes.byref(nbytes)))
        workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=bs[0].device)
    o.workspace = workspace.data_ptr()
    o.workspace_bytes = workspace.numel()
    bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    res = (Result * n)()
    rc = lib.gbpcg_pcg_solve_batched(n, grids, bp, xp, ctypes.byref(o), res, _stream(stream))
    _check(rc, allowed=(OK, NOT_CONVERGED, BREAKDOWN, TIMEOUT))
    return xs, [r.as_dict() for r in res]


def autotune(b: torch.Tensor, workspace=None, stream=None):
    """Times the tile configurations on A x = b (x from 0, in scratch) and
    returns (tile_cfg code, microseconds per iteration) (gbpcg_autotune)."""
    g = make_grid(b.shape)
    o = make_opts(io_dtype=_dtype(b), autotune=True)
    if workspace is None:
        workspace = alloc_workspace(b.shape, device=b.device, io_dtype=_dtype(b), autotune=True)
    o.workspace = workspace.data_ptr()
    o.workspace_bytes = workspace.numel()
    code = ctypes.c_int32(0)
    us = ctypes.c_double(0.0)
    _check(load().gbpcg_autotune(ctypes.byref(g), ctypes.byref(o), _ptr(b), ctypes.byref(code), ctypes.byref(us),
                                 _stream(stream)))
    return code.value, us.value


def autotune_record(shape, tile_cfg: int, io_dtype=F32):
    """Seeds the process-wide autotune cache (e.g. from a saved file)."""
    g = make_grid(shape)
    o = make_opts(io_dtype=io_dtype)
    _check(load().gbpcg_autotune_record(ctypes.byref(g), ctypes.byref(o), int(tile_cfg)))


def save_autotune(path, entries):
    """Writes {"nx,ny,nz,io": code} entries (from autotune()) as JSON."""
    import json
    with open(path, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)


def load_autotune(path):
    """Reads a file written by save_autotune and seeds the cache with it."""
    import json
    with open(path) as f:
        entries = json.load(f)
    for key, code in entries.items():
        nx, ny, nz, io = (int(v) for v in key.split(","))
        autotune_record((nz, ny, nx), code, io)
    return entries


# --------------------------------------------------- learned preconditioner --

def conv3_workspace(shape, ci, co, device="cuda") -> torch.Tensor:
    nz, ny, nx = (int(v) for v in shape)
    n = ctypes.c_size_t(0)
    _check(load().gbpcg_conv3_workspace_size(nx, ny, nz, int(ci), int(co), ctypes.byref(n)))
    return torch.empty(int(n.value), dtype=torch.uint8, device=device)


def _conv_check(a: torch.Tensor, name: str):
    if a.dim() != 4 or not a.is_cuda or not a.is_contiguous() or a.dtype != torch.bfloat16:
        raise GbpcgError(ERR_ARG, f"{name} must be a contiguous bfloat16 CUDA tensor (nz, ny, nx, C)")


def conv3_forward(x: torch.Tensor, w: torch.Tensor, relu=False, workspace=None, stream=None) -> torch.Tensor:
    """y = conv3(x, w) in FP32 (gbpcg_conv3_forward); x (nz, ny, nx, ci) and w (co, 27, ci) bfloat16."""
    _conv_check(x, "x")
    co, _, ci = w.shape
    nz, ny, nx, _ = x.shape
    y = torch.empty((nz, ny, nx, co), dtype=torch.float32, device=x.device)
    ws = workspace if workspace is not None else conv3_workspace(x.shape[:3], ci, co, x.device)
    _check(load().gbpcg_conv3_forward(nx, ny, nz, ci, co, _ptr(x), _ptr(w.contiguous()), _ptr(y), int(bool(relu)),
                                      _ptr(ws), ws.numel(), _stream(stream)))
    return y


def conv3_backward_data(gy: torch.Tensor, w: torch.Tensor, workspace=None, stream=None) -> torch.Tensor:
    """gx = conv3 adjoint of gy (gbpcg_conv3_backward_data); gy (.., co), w (co, 27, ci) bfloat16."""
    _conv_check(gy, "gy")
    co, _, ci = w.shape
    nz, ny, nx, _ = gy.shape
    gx = torch.empty((nz, ny, nx, ci), dtype=torch.float32, device=gy.device)
    ws = workspace if workspace is not None else conv3_workspace(gy.shape[:3], ci, co, gy.device)
    _check(load().gbpcg_conv3_backward_data(nx, ny, nz, ci, co, _ptr(gy), _ptr(w.contiguous()), _ptr(gx), _ptr(ws),
                                            ws.numel(), _stream(stream)))
    return gx


def conv3_backward_weight(x: torch.Tensor, gy: torch.Tensor, workspace=None, stream=None) -> torch.Tensor:
    """gw (co, 27, ci) FP32 = sum_v gy[v, o] x[v + off(t), i] (gbpcg_conv3_backward_weight)."""
    _conv_check(x, "x")
    _conv_check(gy, "gy")
    nz, ny, nx, ci = x.shape
    co = gy.shape[3]
    gw = torch.empty((co, 27, ci), dtype=torch.float32, device=x.device)
    ws = workspace if workspace is not None else conv3_workspace(x.shape[:3], ci, co, x.device)
    _check(load().gbpcg_conv3_backward_weight(nx, ny, nz, ci, co, _ptr(x), _ptr(gy), _ptr(gw), _ptr(ws), ws.numel(),
                                              _stream(stream)))
    return gw


def nn_workspace(shape, training=False, device="cuda") -> torch.Tensor:
    nz, ny, nx = (int(v) for v in shape)
    n = ctypes.c_size_t(0)
    _check(load().gbpcg_nn_workspace_size(nx, ny, nz, int(bool(training)), ctypes.byref(n)))
    return torch.empty(int(n.value), dtype=torch.uint8, device=device)


NN_TENSORS = ["xin", "a1", "k8", "p1", "a3", "k7", "p2", "a5", "a6", "a7", "a8", "dsc", "sr", "scale",
              "gout", "ga8", "gk8", "ga7", "gk7", "ga6", "ga5", "t5", "ge1b", "ga3", "t3", "ge0b", "ga1"]


def nn_tensor(workspace: torch.Tensor, shape, name: str, training=False) -> torch.Tensor:
    """A view of tensor `name` (NN_TENSORS) inside a network workspace (gbpcg_nn_tensor_info):
    (nz, ny, nx, C) of its level, channels-last; 'scale' is a 0-d float64."""
    nz, ny, nx = (int(v) for v in shape)
    off, dt, ch, lv = ctypes.c_size_t(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load().gbpcg_nn_tensor_info(nx, ny, nz, int(bool(training)), NN_TENSORS.index(name), ctypes.byref(off),
                                       ctypes.byref(dt), ctypes.byref(ch), ctypes.byref(lv)))
    tdt = {F32: torch.float32, BF16: torch.bfloat16, F64: torch.float64}[dt.value]
    esize = torch.tensor([], dtype=tdt).element_size()
    if lv.value < 0:
        return workspace[off.value:off.value + esize].view(tdt)[0]
    dims = (nz >> lv.value, ny >> lv.value, nx >> lv.value, ch.value)
    nbytes = dims[0] * dims[1] * dims[2] * dims[3] * esize
    return workspace[off.value:off.value + nbytes].view(tdt).reshape(dims)


def nn_pack_weights(ws: dict) -> torch.Tensor:
    """One flat float32 array of the layers' (co, 27, ci) weights, c1..c9 in order (CPU tensor)."""
    parts = [torch.as_tensor(ws[name], dtype=torch.float32).reshape(-1) for name, _, _ in NN_LAYERS]
    return torch.cat(parts)


def nn_unpack_weights(flat: torch.Tensor) -> dict:
    out, o = {}, 0
    for name, ci, co in NN_LAYERS:
        n = co * 27 * ci
        out[name] = flat[o:o + n].reshape(co, 27, ci)
        o += n
    return out


def nn_forward(w: torch.Tensor, r: torch.Tensor, z=None, k_block=None, kb=8, workspace=None, stream=None):
    """z = N(r) (gbpcg_nn_forward); w: float32 CUDA master weights, r (nz, ny, nx) float32."""
    if z is None:
        z = torch.empty_like(r)
    ws = workspace if workspace is not None else nn_workspace(r.shape, False, r.device)
    g = make_grid(r.shape, k_block, kb)
    _check(load().gbpcg_nn_forward(ctypes.byref(g), _ptr(w), _ptr(r), _ptr(z), _ptr(ws), ws.numel(),
                                   _stream(stream)))
    return z


def nn_backward(gz: torch.Tensor, workspace: torch.Tensor, gw=None, k_block=None, kb=8, stream=None):
    """dL/dw from dL/dz after nn_forward on the same training workspace (gbpcg_nn_backward)."""
    if gw is None:
        gw = torch.empty(NN_NUM_WEIGHTS, dtype=torch.float32, device=gz.device)
    g = make_grid(gz.shape, k_block, kb)
    _check(load().gbpcg_nn_backward(ctypes.byref(g), _ptr(gz), _ptr(gw), _ptr(workspace), workspace.numel(),
                                    _stream(stream)))
    return gw


def nn_loss(z: torch.Tensor, e: torch.Tensor, workspace: torch.Tensor, k_block=None, kb=8, stream=None):
    """(loss device scalar, gz) of the scale-free A-norm loss (gbpcg_nn_loss)."""
    gz = torch.empty_like(z)
    loss = torch.empty((), dtype=torch.float64, device=z.device)
    g = make_grid(z.shape, k_block, kb)
    _check(load().gbpcg_nn_loss(ctypes.byref(g), _ptr(z), _ptr(e), _ptr(gz), _ptr(loss), _ptr(workspace),
                                workspace.numel(), _stream(stream)))
    return loss, gz


def nn_adam(w, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """Adam update of w, m, v in place (gbpcg_nn_adam)."""
    _check(load().gbpcg_nn_adam(w.numel(), _ptr(w), _ptr(g), _ptr(m), _ptr(v), int(step), float(lr), float(beta1),
                                float(beta2), float(eps), _stream(stream)))


class NnTrainer:
    """Device state of training (weights, Adam moments, scratch) for one grid
    shape; ``step`` runs gbpcg_nn_train_step on one (r, e) pair."""

    def __init__(self, w: torch.Tensor, shape, k_block=None, kb=8, device="cuda"):
        self.w = w.to(device=device, dtype=torch.float32).contiguous().clone()
        self.m = torch.zeros_like(self.w)
        self.v = torch.zeros_like(self.w)
        self.gw = torch.zeros_like(self.w)
        self.shape = tuple(int(s) for s in shape)
        self.z = torch.empty(self.shape, dtype=torch.float32, device=device)
        self.gz = torch.empty_like(self.z)
        self.loss = torch.zeros((), dtype=torch.float64, device=device)
        self.ws = nn_workspace(self.shape, True, device)
        self.k_block, self.kb = k_block, kb
        self.t = 0

    def set_coefficients(self, k_block, kb=8):
        self.k_block, self.kb = k_block, kb

    def step(self, r: torch.Tensor, e: torch.Tensor, lr=1e-3, stream=None) -> torch.Tensor:
        self.t += 1
        g = make_grid(self.shape, self.k_block, self.kb)
        _check(load().gbpcg_nn_train_step(ctypes.byref(g), _ptr(self.w), _ptr(self.m), _ptr(self.v), self.t,
                                          float(lr), _ptr(r), _ptr(e), _ptr(self.z), _ptr(self.gz), _ptr(self.gw),
                                          _ptr(self.loss), _ptr(self.ws), self.ws.numel(), _stream(stream)))
        return self.loss

    def status(self, stream=None) -> int:
        return _check(load().gbpcg_nn_status(_ptr(self.ws), _stream(stream)))

    def state_dict(self) -> dict:
        """Weights, Adam moments and step count (CPU copies), for torch.save."""
        return {"w": self.w.cpu(), "m": self.m.cpu(), "v": self.v.cpu(), "t": self.t, "shape": self.shape}

    def load_state_dict(self, state: dict):
        """Resumes training from state_dict() output; the grid shape must match."""
        if tuple(state["shape"]) != self.shape:
            raise GbpcgError(ERR_ARG, f"checkpoint is for grid {tuple(state['shape'])}, not {self.shape}")
        for name in ("w", "m", "v"):
            getattr(self, name).copy_(state[name].to(self.w.device))
        self.t = int(state["t"])


def nn_status(workspace: torch.Tensor, stream=None) -> int:
    return _check(load().gbpcg_nn_status(_ptr(workspace), _stream(stream)))


def _fcg_opts(tol, maxit, workspace=None, m=0):
    o = make_opts(tol=tol, maxit=maxit, io_dtype=F64, workspace=workspace)
    o.precond = PRECOND_LEARNED
    o.fcg_m = int(m)
    return o


def fcg_workspace(shape, k_block=None, kb=8, tol=1e-6, maxit=2000, m=0, device="cuda") -> torch.Tensor:
    g = make_grid(shape, k_block, kb)
    o = _fcg_opts(tol, maxit, None, m)
    n = ctypes.c_size_t(0)
    _check(load().gbpcg_fcg_workspace_size(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)))
    return torch.empty(int(n.value), dtype=torch.uint8, device=device)


def fcg_solve(w: torch.Tensor, b: torch.Tensor, x: torch.Tensor | None = None, tol=1e-6, maxit=2000, k_block=None,
              kb=8, m=0, workspace=None, stream=None):
    """Flexible CG with truncation m (0: the library's default) and the learned preconditioner N_w
    (gbpcg_fcg_solve); b, x float64 CUDA (nz, ny, nx).  Returns (x, result dict); FALLBACK_USED,
    NOT_CONVERGED and BREAKDOWN are reported, not raised."""
    if b.dtype != torch.float64 or not b.is_cuda:
        raise GbpcgError(ERR_ARG, "b must be a float64 CUDA tensor")
    if x is None:
        x = torch.zeros_like(b)
    ws = workspace if workspace is not None else fcg_workspace(b.shape, k_block, kb, tol, maxit, m, b.device)
    g = make_grid(b.shape, k_block, kb)
    o = _fcg_opts(tol, maxit, ws, m)
    res = Result()
    _check(load().gbpcg_fcg_solve(ctypes.byref(g), _ptr(w), _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(res),
                                  _stream(stream)), allowed=(OK, NOT_CONVERGED, BREAKDOWN, FALLBACK_USED))
    return x, res.as_dict()


def wait_selftest(arrive: bool, polls: int, stream=None):
    """(status, ms) of the bounded-wait self-test (gbpcg_wait_selftest); status is OK or TIMEOUT."""
    ms = ctypes.c_double(0.0)
    scratch = torch.zeros(16, dtype=torch.uint8, device="cuda")
    rc = _check(load().gbpcg_wait_selftest(int(bool(arrive)), int(polls), _ptr(scratch), ctypes.byref(ms),
                                           _stream(stream)), allowed=(OK, TIMEOUT))
    return rc, ms.value
