"""GB300 sparse operators: SpMV (CSR, ELL, SELL-P), COO->CSR and
CSR->ELL/SELL-P conversion, and CG / BiCGSTAB / GMRES(m) with a Jacobi
preconditioner, behind the C ABI declared in include/gk.h.

This module is a thin ctypes binding: the functions carry the C names and
only marshal arguments (torch tensors or numpy arrays to raw pointers,
enums to ints, structs to dicts).  Every step of the computation runs in
libgk.so; there is no CPU fallback, and importing fails loudly when the
library has not been built (``python -c "import __graft_entry__ as g;
g.build()"``).

Arrays may be CUDA torch tensors (device pointers) or host arrays (numpy or
CPU torch tensors).  The ``Matrix`` class wraps a handle for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgk.so")

GK_F64, GK_F32, GK_BF16, GK_F16 = 0, 1, 2, 3
GK_CSR, GK_ELL, GK_SELLP, GK_COO = 0, 1, 2, 3
GK_CG, GK_BICGSTAB, GK_GMRES, GK_CGS = 0, 1, 2, 3
GK_PRECOND_NONE, GK_PRECOND_JACOBI, GK_PRECOND_BLOCK_JACOBI, GK_PRECOND_ILU = 0, 1, 2, 3
GK_MEM_HOST, GK_MEM_DEVICE = 0, 1
GK_OK, GK_NOT_CONVERGED, GK_BREAKDOWN = 0, 1, 2
GK_ERR_INVALID, GK_ERR_OOM, GK_ERR_CUDA, GK_ERR_TIMEOUT = -1, -2, -3, -4
GK_ERR_ZERO_DIAG, GK_ERR_NAN, GK_ERR_UNSUPPORTED = -5, -6, -7

DTYPES = {"f64": GK_F64, "f32": GK_F32, "bf16": GK_BF16, "f16": GK_F16}
FORMATS = {"csr": GK_CSR, "ell": GK_ELL, "sellp": GK_SELLP, "coo": GK_COO}
METHODS = {"cg": GK_CG, "bicgstab": GK_BICGSTAB, "gmres": GK_GMRES, "cgs": GK_CGS}

EXPORTED = [
    "gk_matrix_create_csr", "gk_matrix_create_coo", "gk_matrix_convert",
    "gk_matrix_describe", "gk_matrix_export", "gk_matrix_destroy", "gk_apply",
    "gk_apply_adv", "gk_solve", "gk_solve_batched", "gk_status_string", "gk_version",
    "gk_spmv_csr_f64_noalloc", "gk_precond_apply", "gk_ilu_factors", "gk_triangular_solve",
    "gk_solve_async",
]
PRECONDS = {"none": GK_PRECOND_NONE, "jacobi": GK_PRECOND_JACOBI,
            "block_jacobi": GK_PRECOND_BLOCK_JACOBI, "ilu": GK_PRECOND_ILU}


class GkError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {status} ({_status_text(status)})")


class gk_matrix_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("ncols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("format", ctypes.c_int), ("dtype", ctypes.c_int), ("max_row", ctypes.c_int32),
                ("ell_width", ctypes.c_int32), ("ell_stride", ctypes.c_int64),
                ("slice_size", ctypes.c_int32), ("stride_factor", ctypes.c_int32),
                ("num_slices", ctypes.c_int32), ("stored", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("spmv_kernel", ctypes.c_int32),
                ("spmv_launches", ctypes.c_int32), ("device_error", ctypes.c_int32),
                ("solve_format", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gk_solve_opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("precond", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_iters", ctypes.c_int32), ("krylov_dim", ctypes.c_int32),
                ("mixed", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int32), ("batch_tols", ctypes.c_void_p),
                ("engine", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("wait_budget_ns", ctypes.c_int64)]


class gk_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("outer_iters", ctypes.c_int32), ("rel_res_recurrence", ctypes.c_double),
                ("rel_res_true", ctypes.c_double), ("device_ms", ctypes.c_float),
                ("spmv_format", ctypes.c_int32), ("slice_size", ctypes.c_int32),
                ("block_threads", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """The loaded libgk.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "paper_2510_08230_gb300._build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        pm = ctypes.POINTER(vp)
        L.gk_matrix_create_csr.argtypes = [i32, i32, i64, vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, pm]
        L.gk_matrix_create_coo.argtypes = [i32, i32, i64, vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, pm]
        L.gk_matrix_convert.argtypes = [vp, ctypes.c_int, ctypes.c_int, i32, i32, vp, pm]
        L.gk_matrix_describe.argtypes = [vp, ctypes.POINTER(gk_matrix_desc)]
        L.gk_matrix_export.argtypes = [vp, vp, vp, vp, vp]
        L.gk_matrix_destroy.argtypes = [vp]
        L.gk_apply.argtypes = [vp, vp, vp, vp]
        L.gk_apply_adv.argtypes = [vp, f64, vp, f64, vp, vp]
        L.gk_solve.argtypes = [vp, vp, vp, ctypes.POINTER(gk_solve_opts),
                               ctypes.POINTER(gk_solve_info), vp]
        L.gk_solve_batched.argtypes = [i32, pm, pm, pm, ctypes.POINTER(gk_solve_opts),
                                       ctypes.POINTER(gk_solve_info), vp]
        L.gk_solve_async.argtypes = [vp, vp, vp, ctypes.POINTER(gk_solve_opts), vp, vp]
        L.gk_spmv_csr_f64_noalloc.argtypes = [i32, i32, i64, vp, vp, vp, f64, vp, f64, vp, vp]
        L.gk_precond_apply.argtypes = [vp, ctypes.c_int, i32, vp, vp, i64, vp]
        L.gk_ilu_factors.argtypes = [vp, vp, vp]
        L.gk_triangular_solve.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, i64, vp]
        L.gk_status_string.argtypes = [ctypes.c_int]
        L.gk_status_string.restype = ctypes.c_char_p
        L.gk_version.argtypes = []
        L.gk_version.restype = i32
        for name in EXPORTED:
            f = getattr(L, name)
            if name not in ("gk_status_string", "gk_version"):
                f.restype = ctypes.c_int
        _lib = L
    return _lib


def _status_text(s):
    try:
        return lib().gk_status_string(int(s)).decode()
    except Exception:
        return "?"


# ------------------------------------------------------------------ marshalling

def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """Raw pointer of a torch tensor / numpy array (None stays None)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if _is_torch(a):
        return a.data_ptr()
    return a.ctypes.data


def _mem(a):
    if _is_torch(a) and a.is_cuda:
        return GK_MEM_DEVICE
    return GK_MEM_HOST


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover
        pass
    return None


def _check(st, what):
    if st != GK_OK:
        raise GkError(st, what)


def _dt(dtype):
    return DTYPES[dtype] if isinstance(dtype, str) else int(dtype)


# ------------------------------------------------------------------ C names

def gk_matrix_create_csr(n, ncols, nnz, row_ptr, col_idx, values, dtype, mem=None, stream=None):
    h = ctypes.c_void_p()
    mem = _mem(row_ptr) if mem is None else mem
    st = lib().gk_matrix_create_csr(n, ncols, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(values),
                                    _dt(dtype), mem, _stream(stream), ctypes.byref(h))
    _check(st, "gk_matrix_create_csr")
    return h.value


def gk_matrix_create_coo(n, ncols, nnz, row, col, values, dtype, mem=None, stream=None):
    h = ctypes.c_void_p()
    mem = _mem(row) if mem is None else mem
    st = lib().gk_matrix_create_coo(n, ncols, nnz, _ptr(row), _ptr(col), _ptr(values), _dt(dtype),
                                    mem, _stream(stream), ctypes.byref(h))
    _check(st, "gk_matrix_create_coo")
    return h.value


def gk_matrix_convert(A, fmt, dtype, slice_size=0, stride_factor=0, stream=None):
    h = ctypes.c_void_p()
    fmt = FORMATS[fmt] if isinstance(fmt, str) else fmt
    st = lib().gk_matrix_convert(A, fmt, _dt(dtype), slice_size, stride_factor, _stream(stream),
                                 ctypes.byref(h))
    _check(st, "gk_matrix_convert")
    return h.value


def gk_matrix_describe(A):
    d = gk_matrix_desc()
    _check(lib().gk_matrix_describe(A, ctypes.byref(d)), "gk_matrix_describe")
    return d.as_dict()


def gk_matrix_export(A, idx_a=None, sets=None, col=None, values=None):
    _check(lib().gk_matrix_export(A, _ptr(idx_a), _ptr(sets), _ptr(col), _ptr(values)),
           "gk_matrix_export")


def gk_matrix_destroy(A):
    _check(lib().gk_matrix_destroy(A), "gk_matrix_destroy")


def gk_apply(A, b, x, stream=None):
    return lib().gk_apply(A, _ptr(b), _ptr(x), _stream(stream))


def gk_apply_adv(A, alpha, b, beta, x, stream=None):
    return lib().gk_apply_adv(A, float(alpha), _ptr(b), float(beta), _ptr(x), _stream(stream))


def make_opts(method="cg", precond=None, tol=1e-10, max_iters=1000, krylov_dim=30, mixed=0,
              inner_tol=0.0, max_outer=0, engine=0, block_size=0, wait_budget_ns=0):
    """precond: None / "none" / 0, "jacobi" / 1 / True, "block_jacobi" / 2
    (with block_size rows per diagonal block) or "ilu" / 3 (ILU(0))."""
    m = METHODS[method] if isinstance(method, str) else int(method)
    p = _precond(precond)
    return gk_solve_opts(m, p, tol, max_iters, krylov_dim, mixed, inner_tol, max_outer, None,
                         engine, block_size, int(wait_budget_ns))


def _precond(precond):
    if precond in (None, "none", 0, False):
        return GK_PRECOND_NONE
    if isinstance(precond, str):
        return PRECONDS[precond]
    if precond is True:
        return GK_PRECOND_JACOBI
    return int(precond)


def gk_precond_apply(A, kind, block_size, r, z, wait_budget_ns=0, stream=None):
    return lib().gk_precond_apply(A, _precond(kind), int(block_size), _ptr(r), _ptr(z),
                                  int(wait_budget_ns), _stream(stream))


def gk_solve(A, b, x, opts, stream=None):
    info = gk_solve_info()
    st = lib().gk_solve(A, _ptr(b), _ptr(x), ctypes.byref(opts), ctypes.byref(info),
                        _stream(stream))
    d = info.as_dict()
    d["return"] = st
    return d


def gk_solve_async(A, b, x, opts, info_dev, stream=None):
    """Enqueues the solve; info_dev: a device buffer of
    ctypes.sizeof(gk_solve_info) bytes (e.g. a CUDA uint8 tensor) that
    receives the outcome.  Returns the enqueue status."""
    return lib().gk_solve_async(A, _ptr(b), _ptr(x), ctypes.byref(opts), _ptr(info_dev),
                                _stream(stream))


def solve_info_from_bytes(buf):
    """A gk_solve_info (dict) from its bytes (e.g. a device info buffer
    copied to the host)."""
    raw = bytes(np.asarray(buf, dtype=np.uint8).tobytes())
    return gk_solve_info.from_buffer_copy(raw[:ctypes.sizeof(gk_solve_info)]).as_dict()


def gk_solve_batched(As, bs, xs, opts, stream=None, tols=None):
    """Solves len(As) systems in one launch; tols: optional per-system
    tolerances (overrides opts.tol)."""
    n = len(As)
    keep = None
    if tols is not None:
        keep = np.ascontiguousarray(tols, dtype=np.float64)
        opts.batch_tols = keep.ctypes.data
    arrA = (ctypes.c_void_p * n)(*As)
    arrB = (ctypes.c_void_p * n)(*[_ptr(b) for b in bs])
    arrX = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    infos = (gk_solve_info * n)()
    st = lib().gk_solve_batched(n, arrA, arrB, arrX, ctypes.byref(opts), infos, _stream(stream))
    if keep is not None:
        opts.batch_tols = None
    return st, [i.as_dict() for i in infos]


def gk_spmv_csr_f64_noalloc(n, ncols, nnz, row_ptr, col_idx, values, alpha, b, beta, x,
                            stream=None):
    """x = alpha A b + beta x from raw device CSR arrays, with no device
    allocation (scratch in a fixed device array; see include/gk.h)."""
    return lib().gk_spmv_csr_f64_noalloc(n, ncols, nnz, _ptr(row_ptr), _ptr(col_idx),
                                         _ptr(values), float(alpha), _ptr(b), float(beta),
                                         _ptr(x), _stream(stream))


def gk_status_string(s):
    return lib().gk_status_string(int(s)).decode()


def gk_version():
    return lib().gk_version()


# ------------------------------------------------------------------ convenience

class Matrix:
    """Owning wrapper of a gk_matrix handle."""

    def __init__(self, handle):
        self.handle = handle
        self.desc = gk_matrix_describe(handle)

    @classmethod
    def from_csr(cls, m, dtype="f64", device=None):
        """From a workloads.CSR (host arrays) or any object with n, ncols,
        row_ptr, col_idx, values.  Values wider than dtype (float64 for
        F32/BF16/F16, float32 for BF16/F16) are uploaded in their own type
        and rounded on the device (gk_matrix_convert); BF16 values may also
        be given as uint16 bit patterns."""
        src = np.asarray(m.values).dtype
        if _dt(dtype) != GK_F64 and src == np.float64:
            A = cls.from_csr(m, "f64", device)
            B = A.convert("csr", dtype)
            A.close()
            return B
        if _dt(dtype) in (GK_BF16, GK_F16) and src == np.float32:
            A = cls.from_csr(m, "f32", device)
            B = A.convert("csr", dtype)
            A.close()
            return B
        vals = host_values(m.values, dtype)
        rp = np.ascontiguousarray(m.row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(m.col_idx, dtype=np.int32)
        if device is not None:
            import torch
            rp, ci, vals = (torch.from_numpy(a).to(device) for a in (rp, ci, vals))
        return cls(gk_matrix_create_csr(m.n, m.ncols, int(m.col_idx.shape[0]), rp, ci, vals,
                                        dtype))

    @classmethod
    def from_coo(cls, n, ncols, row, col, val, dtype="f64"):
        row = np.ascontiguousarray(row, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        vals = host_values(val, dtype)
        return cls(gk_matrix_create_coo(n, ncols, row.shape[0], row, col, vals, dtype))

    def convert(self, fmt, dtype=None, slice_size=0, stride_factor=0):
        dt = self.desc["dtype"] if dtype is None else _dt(dtype)
        return Matrix(gk_matrix_convert(self.handle, fmt, dt, slice_size, stride_factor))

    @property
    def n(self):
        return self.desc["n"]

    @property
    def nnz(self):
        return self.desc["nnz"]

    def export(self):
        """Host copies of the format arrays (dict)."""
        d = self.desc
        vdt = {GK_F64: np.float64, GK_F32: np.float32, GK_BF16: np.uint16,
               GK_F16: np.float16}[d["dtype"]]
        out = {}
        if d["format"] == GK_COO:
            nz = max(d["nnz"], 1)
            out["row"] = np.zeros(nz, np.int32)
            out["col_idx"] = np.zeros(nz, np.int32)
            out["values"] = np.zeros(nz, vdt)
            gk_matrix_export(self.handle, out["row"], None, out["col_idx"], out["values"])
            for k in ("row", "col_idx", "values"):
                out[k] = out[k][:d["nnz"]]
        elif d["format"] == GK_CSR:
            out["row_ptr"] = np.zeros(d["n"] + 1, np.int32)
            out["col_idx"] = np.zeros(max(d["nnz"], 1), np.int32)
            out["values"] = np.zeros(max(d["nnz"], 1), vdt)
            gk_matrix_export(self.handle, out["row_ptr"], None, out["col_idx"], out["values"])
            out["col_idx"] = out["col_idx"][:d["nnz"]]
            out["values"] = out["values"][:d["nnz"]]
        else:
            st = d["stored"]
            out["col"] = np.zeros(max(st, 1), np.int32)
            out["values"] = np.zeros(max(st, 1), vdt)
            sl = ss = None
            if d["format"] == GK_SELLP:
                sl = np.zeros(max(d["num_slices"], 1), np.int32)
                ss = np.zeros(d["num_slices"] + 1, np.int64)
            gk_matrix_export(self.handle, sl, ss, out["col"], out["values"])
            out["col"] = out["col"][:st]
            out["values"] = out["values"][:st]
            if sl is not None:
                out["slice_lengths"] = sl[:d["num_slices"]]
                out["slice_sets"] = ss
        return out

    def apply(self, b, x, stream=None):
        _check(gk_apply(self.handle, b, x, stream), "gk_apply")

    def apply_adv(self, alpha, b, beta, x, stream=None):
        _check(gk_apply_adv(self.handle, alpha, b, beta, x, stream), "gk_apply_adv")

    def precond_apply(self, r, z, kind="ilu", block_size=0, stream=None, wait_budget_ns=0):
        """z = M^-1 r for the preconditioner `kind` (device vectors)."""
        _check(gk_precond_apply(self.handle, kind, block_size, r, z, wait_budget_ns, stream),
               "gk_precond_apply")

    def triangular_solve(self, b, x, upper=False, unit_diagonal=False, stream=None,
                         wait_budget_ns=0):
        """x with T x = b, T the lower (or upper) triangle of this matrix
        including its diagonal (unit_diagonal: taken as 1); device vectors."""
        _check(lib().gk_triangular_solve(self.handle, int(bool(upper)), int(bool(unit_diagonal)),
                                         _ptr(b), _ptr(x), int(wait_budget_ns), _stream(stream)),
               "gk_triangular_solve")

    def ilu_factors(self):
        """ILU(0) factors in the CSR order of the matrix (host array of the
        vector type): L left of the diagonal (unit diagonal implied), U on
        and right of it."""
        d = self.desc
        vdt = np.float64 if d["dtype"] == GK_F64 else np.float32
        out = np.zeros(max(d["nnz"], 1), vdt)
        _check(lib().gk_ilu_factors(self.handle, out.ctypes.data_as(ctypes.c_void_p), None),
               "gk_ilu_factors")
        return out[:d["nnz"]]

    def describe(self):
        """Fresh gk_matrix_describe (solve_format is set by the first solve)."""
        self.desc = gk_matrix_describe(self.handle)
        return self.desc

    def solve(self, b, x, stream=None, **kw):
        return gk_solve(self.handle, b, x, make_opts(**kw), stream)

    def close(self):
        if self.handle:
            gk_matrix_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def host_values(values, dtype):
    """Values in the ABI layout of dtype, unchanged: float64 for F64,
    float32 for F32, uint16 bfloat16 bit patterns for BF16, float16 for F16.
    Narrowing is never done here; wider values go through the device
    conversion (gk_matrix_convert)."""
    want = {GK_F64: np.float64, GK_F32: np.float32, GK_BF16: np.uint16,
            GK_F16: np.float16}[_dt(dtype)]
    v = np.asarray(values)
    if v.dtype != want:
        raise TypeError(f"dtype {dtype} takes {np.dtype(want).name} values, got {v.dtype}; "
                        "upload wider values in their own type and convert them on the "
                        "device with gk_matrix_convert")
    return np.ascontiguousarray(v)
