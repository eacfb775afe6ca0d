"""Python binding of the LSRN C ABI (include/lsrn.h).

Argument marshalling only: every step of the solver runs in the CUDA library
``_build/liblsrn.so`` built from ``csrc/``.  Arrays may be numpy arrays (host)
or torch tensors (host or CUDA); their data pointers are handed to the library
unchanged.  If the library is missing or the GPU is unusable, the calls raise
-- there is no CPU fallback.

The names follow the C ABI: ``lsrn_plan``, ``lsrn_sketch``, ``lsrn_precond``,
``lsrn_solve_lsqr``, ``lsrn_solve_cs``, ``lsrn_plan_destroy``,
``lsrn_server_create``, ``lsrn_submit``, ``lsrn_poll``, ``lsrn_server_destroy``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblsrn.so")

LSRN_OK = 0
LSRN_PENDING = 1
LSRN_ERR_INVALID_ARG = -1
LSRN_ERR_OOM = -2
LSRN_ERR_CUDA = -3
LSRN_ERR_NOT_CONVERGED = -4
LSRN_ERR_DIVERGED = -5
LSRN_ERR_TIMEOUT = -6
LSRN_ERR_QUEUE_FULL = -7
LSRN_ERR_STATE = -8
LSRN_ERR_UNSUPPORTED = -9
LSRN_ERR_COMM = -10

LSRN_DENSE_ROWMAJOR, LSRN_DENSE_COLMAJOR, LSRN_CSR = 0, 1, 2
LSRN_F64, LSRN_F32 = 0, 1
LSRN_SKETCH_F64, LSRN_SKETCH_TC_SLICED, LSRN_SKETCH_BF16, LSRN_SKETCH_AUTO = 0, 1, 2, 3
LSRN_ITER_F64, LSRN_ITER_F32, LSRN_ITER_F32X2, LSRN_ITER_AUTO = 0, 1, 2, 3
LSRN_KNOB_JACOBI_WAIT_NS, LSRN_KNOB_JACOBI_SKIP_FIRST_ROUND, LSRN_KNOB_QR_ABSENT_CTA = 0, 1, 2
LSRN_PRECOND_SVD, LSRN_PRECOND_QR = 0, 1
LSRN_SVD_F64, LSRN_SVD_DF = 0, 1


class lsrn_matrix(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("format", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("values", ctypes.c_void_p), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p)]


class lsrn_options(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("tol", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("rcond", ctypes.c_double), ("cs_alpha", ctypes.c_double),
                ("refine_tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("refine_max", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("sketch_mode", ctypes.c_int32), ("iter_mode", ctypes.c_int32),
                ("precond_mode", ctypes.c_int32),
                ("svd_mode", ctypes.c_int32)]


class lsrn_info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("s", ctypes.c_int64),
                ("rank", ctypes.c_int64), ("iterations", ctypes.c_int32),
                ("refine_steps", ctypes.c_int32), ("refine_iterations", ctypes.c_int32),
                ("tall", ctypes.c_int32), ("istop", ctypes.c_int32), ("status", ctypes.c_int32),
                ("sigma_max_sketch", ctypes.c_double), ("sigma_min_sketch", ctypes.c_double),
                ("sigma_L", ctypes.c_double), ("sigma_U", ctypes.c_double),
                ("rnorm_est", ctypes.c_double), ("arnorm_est", ctypes.c_double),
                ("anorm_est", ctypes.c_double), ("t_sketch_ms", ctypes.c_float),
                ("t_precond_ms", ctypes.c_float), ("t_iter_ms", ctypes.c_float),
                ("t_refine_ms", ctypes.c_float), ("t_sketch_gemm_ms", ctypes.c_float),
                ("t_pass_ms", ctypes.c_float), ("n_pass", ctypes.c_int32),
                ("t_qr_ms", ctypes.c_float), ("jacobi_sweeps", ctypes.c_int32),
                ("t_jacobi_ms", ctypes.c_float), ("sketch_used", ctypes.c_int32),
                ("sketch_escalated", ctypes.c_int32),
                ("jacobi_sweeps_df", ctypes.c_int32), ("iter_used", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


lsrn_allgather_fn = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int64)


class lsrn_shard(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("world", ctypes.c_int32),
                ("by_columns", ctypes.c_int32), ("long_offset", ctypes.c_int64),
                ("long_total", ctypes.c_int64), ("allgather", lsrn_allgather_fn),
                ("ctx", ctypes.c_void_p)]


lsrn_matmat_fn = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_void_p)


class lsrn_operator(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("matmat", lsrn_matmat_fn),
                ("rmatmat", lsrn_matmat_fn), ("ctx", ctypes.c_void_p)]


class lsrn_gamma_model(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("rank", ctypes.c_int64),
                ("tol", ctypes.c_double), ("solver", ctypes.c_int32),
                ("c_sketch", ctypes.c_double), ("c_qr", ctypes.c_double),
                ("c_svd", ctypes.c_double), ("c_iter", ctypes.c_double),
                ("gamma_min", ctypes.c_double), ("gamma_max", ctypes.c_double)]


class LsrnError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {status_string(status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


_lib = None

_SIGS = {
    "lsrn_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "lsrn_last_error_message": ([], ctypes.c_char_p),
    "lsrn_kernel_launches": ([], ctypes.c_uint64),
    "lsrn_probe_fp64_fma": ([ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "lsrn_default_options": ([ctypes.POINTER(lsrn_options)], ctypes.c_int),
    "lsrn_set_test_knob": ([ctypes.c_int32, ctypes.c_int64], ctypes.c_int),
    "lsrn_plan": ([ctypes.POINTER(lsrn_matrix), ctypes.POINTER(lsrn_options), ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "lsrn_plan_sharded": ([ctypes.POINTER(lsrn_matrix), ctypes.POINTER(lsrn_options),
                           ctypes.POINTER(lsrn_shard), ctypes.c_void_p,
                           ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "lsrn_solve_batch": ([ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.POINTER(lsrn_options), ctypes.c_int32, ctypes.c_int32,
                          ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "lsrn_sketch_group": ([ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "lsrn_plan_set_lambda": ([ctypes.c_void_p, ctypes.c_double], ctypes.c_int),
    "lsrn_choose_gamma": ([ctypes.POINTER(lsrn_gamma_model), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "lsrn_plan_operator": ([ctypes.POINTER(lsrn_operator), ctypes.POINTER(lsrn_options),
                            ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "lsrn_sketch": ([ctypes.c_void_p], ctypes.c_int),
    "lsrn_precond": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "lsrn_solve_lsqr": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.POINTER(lsrn_info)], ctypes.c_int),
    "lsrn_solve_cs": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                       ctypes.POINTER(lsrn_info)], ctypes.c_int),
    "lsrn_plan_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "lsrn_plan_get_sketch": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "lsrn_plan_get_planes": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "lsrn_plan_get_precond": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "lsrn_generate_sketch_block": ([ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64,
                                    ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
                                   ctypes.c_int),
    "lsrn_sketch_f64_noalloc": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p,
                                 ctypes.c_void_p], ctypes.c_int),
    "lsrn_server_create": ([ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)],
                           ctypes.c_int),
    "lsrn_submit": ([ctypes.c_void_p, ctypes.POINTER(lsrn_matrix), ctypes.c_void_p,
                     ctypes.POINTER(lsrn_options), ctypes.c_int32,
                     ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "lsrn_poll": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(lsrn_info)],
                  ctypes.c_int),
    "lsrn_server_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "lsrn_server_set_batching": ([ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    "lsrn_server_stats": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64),
                           ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
}


def library_path() -> str:
    return LIB_PATH


def load_library():
    """Load _build/liblsrn.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"LSRN CUDA library not built: {LIB_PATH} is missing "
                           "(run paper_1109_5981_gb300.build.build())")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(load_library().lsrn_kernel_launches())


def probe_fp64_fma() -> float:
    """FP64 FMA throughput of the current device (TFLOP/s)."""
    v = ctypes.c_double()
    _check(load_library().lsrn_probe_fp64_fma(ctypes.byref(v)), "lsrn_probe_fp64_fma")
    return v.value


def lsrn_set_test_knob(knob: int, value: int) -> None:
    """Set a process-wide test knob (0 turns it off)."""
    _check(load_library().lsrn_set_test_knob(knob, value), "lsrn_set_test_knob")


def status_string(status: int) -> str:
    try:
        return load_library().lsrn_status_string(int(status)).decode()
    except RuntimeError:
        return f"status {status}"


def _check(status: int, where: str, allowed=(LSRN_OK,)) -> int:
    if status not in allowed:
        detail = load_library().lsrn_last_error_message().decode()
        raise LsrnError(status, where, detail)
    return status


def default_options(**kw) -> lsrn_options:
    o = lsrn_options()
    load_library().lsrn_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k in ("lam", "lambda"):
            k = "lambda_"
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


# --------------------------------------------------------------------------- #
# array marshalling                                                            #
# --------------------------------------------------------------------------- #
def _ptr(a) -> int:
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return int(a.data_ptr())
    if isinstance(a, np.ndarray):
        return int(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _dtype_code(a) -> int:
    dt = str(a.dtype)
    if dt in ("float64", "torch.float64"):
        return LSRN_F64
    if dt in ("float32", "torch.float32"):
        return LSRN_F32
    raise TypeError(f"values must be float64 or float32, got {dt}")


def dense_matrix(A, layout: str = "row") -> lsrn_matrix:
    """Descriptor of a dense 2-D array (numpy or torch, host or device).
    layout 'row': A[i, j] at i*ld + j (C order); 'col': A is given as its
    transpose in C order (A^T[j, i]), i.e. A in column-major storage."""
    mat = lsrn_matrix()
    if layout == "row":
        m, n = A.shape
        ld = A.stride(0) if hasattr(A, "stride") and callable(A.stride) else A.strides[0] // A.itemsize
        inner = A.stride(1) if hasattr(A, "stride") and callable(A.stride) else A.strides[1] // A.itemsize
        fmt = LSRN_DENSE_ROWMAJOR
    else:
        n, m = A.shape
        ld = A.stride(0) if hasattr(A, "stride") and callable(A.stride) else A.strides[0] // A.itemsize
        inner = A.stride(1) if hasattr(A, "stride") and callable(A.stride) else A.strides[1] // A.itemsize
        fmt = LSRN_DENSE_COLMAJOR
    if inner != 1:
        raise ValueError("the fastest dimension must be contiguous")
    mat.m, mat.n, mat.ld, mat.nnz = m, n, ld, 0
    mat.format = fmt
    mat.dtype = _dtype_code(A)
    mat.values = _ptr(A)
    return mat


def csr_matrix(m: int, n: int, row_ptr, col_idx, values) -> lsrn_matrix:
    mat = lsrn_matrix()
    mat.m, mat.n, mat.ld = m, n, 0
    mat.nnz = int(values.shape[0])
    mat.format = LSRN_CSR
    mat.dtype = _dtype_code(values)
    mat.values = _ptr(values)
    mat.row_ptr = _ptr(row_ptr)
    mat.col_idx = _ptr(col_idx)
    return mat


class Plan:
    """Owns an lsrn_plan_t; keeps the arrays it was built from alive."""

    def __init__(self, handle: int, keep: tuple, m: int, n: int):
        self.handle = handle
        self._keep = keep
        self.m, self.n = m, n

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self.handle:
            load_library().lsrn_plan_destroy(self.handle)
            self.handle = 0


def lsrn_plan(A, opt: Optional[lsrn_options] = None, stream: int = 0, layout: str = "row",
              csr: Optional[tuple] = None) -> Plan:
    """lsrn_plan(): A is a dense array, or csr=(m, n, row_ptr, col_idx, values)."""
    lib = load_library()
    if csr is not None:
        m, n, rp, ci, vals = csr
        mat = csr_matrix(m, n, rp, ci, vals)
        keep = (rp, ci, vals)
    else:
        mat = dense_matrix(A, layout)
        keep = (A,)
    h = ctypes.c_void_p()
    o = opt if opt is not None else default_options()
    _check(lib.lsrn_plan(ctypes.byref(mat), ctypes.byref(o), ctypes.c_void_p(stream),
                         ctypes.byref(h)), "lsrn_plan")
    return Plan(h.value, keep, mat.m, mat.n)


def shard_rows(m_total: int, world: int, rank: int) -> tuple:
    """Rows of shard `rank` in a partition of m_total rows into `world` blocks
    of consecutive rows whose sizes differ by at most one: (offset, count)."""
    if not (world >= 1 and 0 <= rank < world and m_total >= world):
        raise ValueError("need world >= 1, 0 <= rank < world and m_total >= world")
    base, extra = divmod(m_total, world)
    offset = rank * base + min(rank, extra)
    return offset, base + (1 if rank < extra else 0)


class _DeviceArray:
    """A device buffer the library owns, seen by torch without a copy."""

    def __init__(self, ptr: int, count: int):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": "<f8",
                                         "data": (ptr, False), "version": 3}


def device_view(ptr: int, count: int):
    """torch view (float64, CUDA) of `count` doubles at a library device pointer."""
    import torch
    return torch.as_tensor(_DeviceArray(ptr, count), device="cuda")


def torch_allgather(group=None):
    """allgather callback over a torch.distributed process group: NCCL gathers
    the device buffers in place; other backends (gloo) go through host copies."""
    import torch
    import torch.distributed as dist

    def fn(send_ptr: int, recv_ptr: int, count: int) -> None:
        send = device_view(send_ptr, count)
        recv = device_view(recv_ptr, count * dist.get_world_size(group))
        if dist.get_backend(group) == "nccl":
            dist.all_gather_into_tensor(recv, send, group=group)
            torch.cuda.current_stream().synchronize()
        else:
            out = torch.empty(recv.shape, dtype=torch.float64)
            dist.all_gather_into_tensor(out, send.cpu(), group=group)
            recv.copy_(out)
            torch.cuda.synchronize()
    return fn


def lsrn_plan_sharded(A_local, opt: Optional[lsrn_options], rank: int, world: int,
                      long_offset: int, long_total: int, allgather, stream: int = 0,
                      csr: Optional[tuple] = None, by_columns: bool = False) -> Plan:
    """lsrn_plan_sharded(): one shard -- rows long_offset .. of a tall A, or with
    by_columns columns long_offset .. of a fat A.  allgather(send_ptr, recv_ptr,
    count) fills recv (world * count doubles, rank-major) from every shard's
    send; exceptions become LSRN_ERR_COMM."""
    lib = load_library()
    if csr is not None:
        m, n, rp, ci, vals = csr
        mat = csr_matrix(m, n, rp, ci, vals)
        keep = [rp, ci, vals]
    else:
        mat = dense_matrix(A_local, "row")
        keep = [A_local]

    def _cb(ctx, send, recv, count):
        try:
            allgather(int(send), int(recv), int(count))
            return 0
        except Exception:        # reported to the library as a failed exchange
            import traceback
            traceback.print_exc()
            return 1
    cb = lsrn_allgather_fn(_cb)
    sh = lsrn_shard(rank=rank, world=world, by_columns=1 if by_columns else 0,
                    long_offset=long_offset, long_total=long_total, allgather=cb, ctx=None)
    keep += [cb, sh]
    h = ctypes.c_void_p()
    o = opt if opt is not None else default_options()
    _check(lib.lsrn_plan_sharded(ctypes.byref(mat), ctypes.byref(o), ctypes.byref(sh),
                                 ctypes.c_void_p(stream), ctypes.byref(h)), "lsrn_plan_sharded")
    return Plan(h.value, tuple(keep), mat.m, mat.n)


def lsrn_solve_batch(problems, opt: Optional[lsrn_options] = None, solver: str = "lsqr",
                     threads: int = 0, xs=None):
    """lsrn_solve_batch(): problems is a list of (A, b) with A a dense array or a
    csr tuple (m, n, row_ptr, col_idx, values).  Returns (xs, infos, statuses)."""
    lib = load_library()
    n = len(problems)
    mats = (lsrn_matrix * max(n, 1))()
    keep = []
    if xs is None:
        xs = []
        for A, b in problems:
            cols = A[1] if isinstance(A, tuple) else A.shape[1]
            xs.append(np.empty(cols) if isinstance(b, np.ndarray) else b.new_empty(cols))
    for k, (A, b) in enumerate(problems):
        mats[k] = csr_matrix(*A) if isinstance(A, tuple) else dense_matrix(A, "row")
        keep.append(A)
    bptr = (ctypes.c_void_p * max(n, 1))(*[_ptr(b) for _, b in problems])
    xptr = (ctypes.c_void_p * max(n, 1))(*[_ptr(x) for x in xs])
    infos = (lsrn_info * max(n, 1))()
    stat = (ctypes.c_int32 * max(n, 1))()
    o = opt if opt is not None else default_options()
    code = {"lsqr": 0, "cs": 1}[solver]
    st = lib.lsrn_solve_batch(n, ctypes.byref(mats), ctypes.byref(bptr), ctypes.byref(xptr),
                              ctypes.byref(o), code, threads, ctypes.byref(infos),
                              ctypes.byref(stat))
    out_info = []
    for k in range(n):
        d = infos[k].as_dict()
        d["status"] = int(stat[k])
        out_info.append(d)
    _check(st, "lsrn_solve_batch", (LSRN_OK, LSRN_ERR_NOT_CONVERGED, LSRN_ERR_DIVERGED))
    return xs, out_info, [int(stat[k]) for k in range(n)]


def lsrn_sketch_group(plans) -> list:
    """lsrn_sketch_group(): sketches a list of Plan objects at once; returns their statuses."""
    lib = load_library()
    n = len(plans)
    hs = (ctypes.c_void_p * max(n, 1))(*[p.handle for p in plans])
    stat = (ctypes.c_int32 * max(n, 1))()
    st = lib.lsrn_sketch_group(n, ctypes.byref(hs), ctypes.byref(stat))
    _check(st, "lsrn_sketch_group")
    return [int(stat[k]) for k in range(n)]


def lsrn_choose_gamma(m: int, n: int, rank: int = 0, tol: float = 1e-14, solver: str = "lsqr",
                      c_sketch: float = 0.0, c_qr: float = 0.0, c_svd: float = 0.0,
                      c_iter: float = 0.0, gamma_min: float = 0.0, gamma_max: float = 0.0):
    """Returns (gamma, predicted ms) minimising the section 4.3 cost model."""
    md = lsrn_gamma_model(m=m, n=n, rank=rank, tol=tol, solver={"lsqr": 0, "cs": 1}[solver],
                          c_sketch=c_sketch, c_qr=c_qr, c_svd=c_svd, c_iter=c_iter,
                          gamma_min=gamma_min, gamma_max=gamma_max)
    g, t = ctypes.c_double(), ctypes.c_double()
    _check(load_library().lsrn_choose_gamma(ctypes.byref(md), ctypes.byref(g), ctypes.byref(t)),
           "lsrn_choose_gamma")
    return g.value, t.value


def gamma_costs_from_info(info: dict) -> dict:
    """Per-unit costs of the gamma model from an earlier solve's lsrn_info."""
    s = max(1, info["s"])
    its = max(1, info["iterations"] + info["refine_iterations"])
    return {"c_sketch": info["t_sketch_ms"] / s, "c_qr": info["t_qr_ms"] / s,
            "c_svd": max(0.0, info["t_precond_ms"] - info["t_qr_ms"]),
            "c_iter": (info["t_iter_ms"] + info["t_refine_ms"]) / its}


def lsrn_plan_operator(m: int, n: int, matmat, rmatmat, opt: Optional[lsrn_options] = None,
                       stream: int = 0) -> Plan:
    """lsrn_plan_operator(): A given by products.  matmat(k, x, y) must write
    y = A x (x: n x k, y: m x k, column-major) and rmatmat(k, y, x) x = A^T y;
    both receive torch views of the library's device buffers (float64, CUDA,
    shape (k, rows) -- the column-major block seen row by row) and must finish
    before returning.  Exceptions become LSRN_ERR_COMM."""
    def wrap(fn, rows_in, rows_out):
        def cb(ctx, k, inp, out):
            try:
                x = device_view(int(inp), int(k) * rows_in).view(int(k), rows_in)
                y = device_view(int(out), int(k) * rows_out).view(int(k), rows_out)
                fn(x, y)
                import torch
                torch.cuda.synchronize()
                return 0
            except Exception:
                import traceback
                traceback.print_exc()
                return 1
        return lsrn_matmat_fn(cb)
    cm, cr = wrap(matmat, n, m), wrap(rmatmat, m, n)
    op = lsrn_operator(m=m, n=n, matmat=cm, rmatmat=cr, ctx=None)
    h = ctypes.c_void_p()
    o = opt if opt is not None else default_options()
    _check(load_library().lsrn_plan_operator(ctypes.byref(op), ctypes.byref(o), ctypes.c_void_p(stream),
                                             ctypes.byref(h)), "lsrn_plan_operator")
    return Plan(h.value, (cm, cr, op, matmat, rmatmat), m, n)


def lsrn_plan_set_lambda(plan: Plan, lam: float) -> None:
    _check(load_library().lsrn_plan_set_lambda(plan.handle, float(lam)), "lsrn_plan_set_lambda")


def lsrn_sketch(plan: Plan) -> None:
    _check(load_library().lsrn_sketch(plan.handle), "lsrn_sketch")


def lsrn_precond(plan: Plan) -> int:
    r = ctypes.c_int64()
    _check(load_library().lsrn_precond(plan.handle, ctypes.byref(r)), "lsrn_precond")
    return r.value


def _solve(fn_name: str, plan: Plan, b, x=None, allow=(LSRN_OK,)):
    lib = load_library()
    if x is None:
        x = (np.empty(plan.n, dtype=np.float64) if isinstance(b, np.ndarray)
             else b.new_empty(plan.n))
    info = lsrn_info()
    st = getattr(lib, fn_name)(plan.handle, _ptr(b), _ptr(x), ctypes.byref(info))
    _check(st, fn_name, allow)
    d = info.as_dict()
    d["status"] = st
    return x, d


def lsrn_solve_lsqr(plan: Plan, b, x=None, allow=(LSRN_OK,)):
    """Returns (x, info dict)."""
    return _solve("lsrn_solve_lsqr", plan, b, x, allow)


def lsrn_solve_cs(plan: Plan, b, x=None, allow=(LSRN_OK,)):
    return _solve("lsrn_solve_cs", plan, b, x, allow)


def lsrn_plan_destroy(plan: Plan) -> None:
    plan.close()


def lsrn_plan_get_sketch(plan: Plan) -> np.ndarray:
    lib = load_library()
    rows, cols = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.lsrn_plan_get_sketch(plan.handle, None, ctypes.byref(rows), ctypes.byref(cols)),
           "lsrn_plan_get_sketch")
    out = np.empty((rows.value, cols.value), dtype=np.float64)
    _check(lib.lsrn_plan_get_sketch(plan.handle, out.ctypes.data, None, None),
           "lsrn_plan_get_sketch")
    return out


def lsrn_plan_get_planes(plan: Plan):
    """Returns (hi, lo, x3 as (rows, ld) float32 arrays, scale)."""
    lib = load_library()
    rows, ld, scale = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    _check(lib.lsrn_plan_get_planes(plan.handle, None, None, None, ctypes.byref(rows),
                                    ctypes.byref(ld), ctypes.byref(scale)),
           "lsrn_plan_get_planes")
    planes = [np.empty((rows.value, ld.value), dtype=np.float32) for _ in range(3)]
    _check(lib.lsrn_plan_get_planes(plan.handle, *[a.ctypes.data for a in planes], None, None,
                                    None), "lsrn_plan_get_planes")
    return planes[0], planes[1], planes[2], scale.value


def lsrn_plan_get_precond(plan: Plan):
    """Returns (N or M as (q, r) array, sigma (r,))."""
    lib = load_library()
    r = ctypes.c_int64()
    _check(lib.lsrn_plan_get_precond(plan.handle, None, None, ctypes.byref(r)),
           "lsrn_plan_get_precond")
    rank = r.value
    rows, cols = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.lsrn_plan_get_sketch(plan.handle, None, ctypes.byref(rows), ctypes.byref(cols)),
           "lsrn_plan_get_sketch")
    N = np.empty((cols.value, rank), dtype=np.float64)
    sig = np.empty(rank, dtype=np.float64)
    _check(lib.lsrn_plan_get_precond(plan.handle, N.ctypes.data if rank else None,
                                     sig.ctypes.data if rank else None, None),
           "lsrn_plan_get_precond")
    return N, sig


def lsrn_generate_sketch_block(seed: int, tag: int, i0: int, j0: int, rows: int, cols: int,
                               with_normals: bool = False):
    """Entries of the drawing array of G (and the raw normals) from the GPU."""
    lib = load_library()
    g = np.empty((rows, cols), dtype=np.float64)
    z = np.empty((rows, cols), dtype=np.float32) if with_normals else None
    _check(lib.lsrn_generate_sketch_block(seed, tag, i0, j0, rows, cols, g.ctypes.data,
                                          z.ctypes.data if z is not None else None, None),
           "lsrn_generate_sketch_block")
    return (g, z) if with_normals else g


def lsrn_sketch_f64_noalloc(A, gamma: float, seed: int, out, stream: int = 0) -> None:
    """A~ = G A into `out` (device arrays) without any device allocation."""
    m, n = A.shape
    ld = A.stride(0)
    _check(load_library().lsrn_sketch_f64_noalloc(_ptr(A), m, n, ld, gamma, seed, _ptr(out),
                                                  ctypes.c_void_p(stream)),
           "lsrn_sketch_f64_noalloc")


def solve(A, b, solver: str = "lsqr", layout: str = "row", csr=None, stream: int = 0,
          x=None, allow=(LSRN_OK,), **options):
    """Plan + sketch + precond + solve in one call; returns (x, info)."""
    plan = lsrn_plan(A, default_options(**options), stream, layout, csr)
    try:
        if solver == "lsqr":
            return lsrn_solve_lsqr(plan, b, x, allow)
        if solver == "cs":
            return lsrn_solve_cs(plan, b, x, allow)
        raise ValueError(solver)
    finally:
        plan.close()


# ---- serving ---------------------------------------------------------------
class Server:
    def __init__(self, hbm_budget_bytes: int, max_slots: int = 4):
        h = ctypes.c_void_p()
        _check(load_library().lsrn_server_create(hbm_budget_bytes, max_slots, ctypes.byref(h)),
               "lsrn_server_create")
        self.handle = h.value

    def close(self):
        if self.handle:
            load_library().lsrn_server_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lsrn_server_create(hbm_budget_bytes: int, max_slots: int = 4) -> Server:
    return Server(hbm_budget_bytes, max_slots)


def lsrn_submit(server: Server, A, b, opt: Optional[lsrn_options] = None, solver: int = 0,
                layout: str = "row", csr=None) -> int:
    if csr is not None:
        m, n, rp, ci, vals = csr
        mat = csr_matrix(m, n, rp, ci, vals)
    else:
        mat = dense_matrix(A, layout)
    o = opt if opt is not None else default_options()
    t = ctypes.c_uint64()
    _check(load_library().lsrn_submit(server.handle, ctypes.byref(mat), _ptr(b), ctypes.byref(o),
                                      solver, ctypes.byref(t)), "lsrn_submit")
    return t.value


def lsrn_poll(server: Server, ticket: int, x_out):
    info = lsrn_info()
    st = load_library().lsrn_poll(server.handle, ticket, _ptr(x_out), ctypes.byref(info))
    return st, info.as_dict()


def lsrn_server_destroy(server: Server) -> None:
    server.close()


def lsrn_server_set_batching(server: Server, max_short_side: int) -> None:
    _check(load_library().lsrn_server_set_batching(server.handle, max_short_side),
           "lsrn_server_set_batching")


def lsrn_server_stats(server: Server) -> tuple:
    b, r = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load_library().lsrn_server_stats(server.handle, ctypes.byref(b), ctypes.byref(r)),
           "lsrn_server_stats")
    return b.value, r.value
