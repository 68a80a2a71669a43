"""CPU oracle for the sparse operator path (TEST INFRASTRUCTURE ONLY).

Plain FP64 C code (``gk_oracle.c``) behind a small ctypes wrapper.  Only
the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package; the library itself never does, and shares no code
with it.  See ``gk_oracle.c`` for what each routine follows.

FP32 inputs are handled as the FP32-rounded values promoted to FP64 (the
oracle always computes in double).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gk_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, NOT_CONVERGED, BREAKDOWN = 0, 1, 2
ERR_INVALID, ERR_ZERO_DIAG, ERR_NAN = -1, -5, -6
CG, BICGSTAB, GMRES, CGS = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE: no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _declare(_lib)
    return _lib


_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


class Opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("tol", ctypes.c_double), ("max_iters", ctypes.c_int32),
                ("krylov_dim", ctypes.c_int32), ("block_size", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("restarts", ctypes.c_int32), ("rel_res_rec", ctypes.c_double),
                ("rel_res_true", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _declare(L):
    i32, i64, f64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    L.or_spmv_csr.argtypes = [i32, _i32p, _i32p, _f64p, _f64p, f64, f64, _f64p, ctypes.c_int]
    L.or_spmv_csr.restype = None
    L.or_spmv_csr_omp.argtypes = [i32, _i32p, _i32p, _f64p, _f64p, f64, f64, _f64p, ctypes.c_int]
    L.or_spmv_csr_omp.restype = ctypes.c_int
    L.or_spmv_coo.argtypes = [i32, i32, i64, _i32p, _i32p, _f64p, _f64p, f64, f64, _f64p,
                              ctypes.c_int]
    L.or_spmv_coo.restype = ctypes.c_int
    L.or_coo_to_csr.argtypes = [i32, i32, i64, _i32p, _i32p, _f64p, ctypes.c_int, _i32p, _i32p, _f64p]
    L.or_coo_to_csr.restype = i64
    L.or_ell_width.argtypes = [i32, _i32p]
    L.or_ell_width.restype = i32
    L.or_csr_to_ell.argtypes = [i32, _i32p, _i32p, _f64p, i32, i64, _i32p, _f64p]
    L.or_csr_to_ell.restype = None
    L.or_ell_to_csr.argtypes = [i32, i32, i64, _i32p, _f64p, _i32p, _i32p, _f64p]
    L.or_ell_to_csr.restype = i64
    L.or_sellp_sizes.argtypes = [i32, _i32p, i32, i32, _i32p, _i64p]
    L.or_sellp_sizes.restype = None
    L.or_csr_to_sellp.argtypes = [i32, _i32p, _i32p, _f64p, i32, _i64p, _i32p, _f64p]
    L.or_csr_to_sellp.restype = None
    L.or_sellp_to_csr.argtypes = [i32, i32, _i32p, _i64p, _i32p, _f64p, _i32p, _i32p, _f64p]
    L.or_sellp_to_csr.restype = i64
    L.or_jacobi_gen.argtypes = [i32, _i32p, _i32p, _f64p, _f64p]
    L.or_jacobi_gen.restype = ctypes.c_int
    L.or_block_jacobi_gen.argtypes = [i32, _i32p, _i32p, _f64p, i32, _f64p]
    L.or_block_jacobi_gen.restype = ctypes.c_int
    L.or_block_jacobi_apply.argtypes = [i32, i32, _f64p, _f64p, _f64p]
    L.or_block_jacobi_apply.restype = None
    L.or_ilu0.argtypes = [i32, _i32p, _i32p, _f64p, _f64p]
    L.or_ilu0.restype = ctypes.c_int
    L.or_ilu0_apply.argtypes = [i32, _i32p, _i32p, _f64p, _f64p, _f64p]
    L.or_ilu0_apply.restype = None
    L.or_trsv.argtypes = [i32, _i32p, _i32p, _f64p, ctypes.c_int, ctypes.c_int, _f64p, _f64p]
    L.or_trsv.restype = ctypes.c_int
    for name in ("or_cg", "or_bicgstab", "or_gmres", "or_cgs"):
        f = getattr(L, name)
        f.argtypes = [i32, _i32p, _i32p, _f64p, _f64p, _f64p, ctypes.POINTER(Opts),
                      ctypes.POINTER(Info), vp]
        f.restype = ctypes.c_int


def _f64(a):
    return np.ascontiguousarray(np.asarray(a).astype(np.float64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def spmv(m, x, alpha=1.0, beta=0.0, y=None, compensated=True):
    """y = alpha * A x + beta * y for a CSR matrix ``m`` (workloads.CSR or
    any object with n, row_ptr, col_idx, values).  Returns a new array."""
    out = np.zeros(m.n) if y is None else _f64(y).copy()
    lib().or_spmv_csr(m.n, _i32(m.row_ptr), _i32(m.col_idx), _f64(m.values), _f64(x),
                      float(alpha), float(beta), out, 1 if compensated else 0)
    return out


def spmv_coo(n, ncols, row, col, val, x, alpha=1.0, beta=0.0, y=None, compensated=True):
    """y = alpha * A x + beta * y with A given as COO triplets (visited in
    storage order).  Returns a new array."""
    out = np.zeros(n) if y is None else _f64(y).copy()
    row, col = _i32(row), _i32(col)
    st = lib().or_spmv_coo(n, ncols, row.shape[0], row, col, _f64(val), _f64(x), float(alpha),
                           float(beta), out, 1 if compensated else 0)
    if st != 0:
        raise ValueError("COO index out of range")
    return out


def spmv_omp(m, x, threads=0, alpha=1.0, beta=0.0, y=None, arrays=None):
    """Row-parallel plain-sum SpMV (the timing mode).  Returns (y, threads)."""
    rp, ci, va = arrays if arrays is not None else (_i32(m.row_ptr), _i32(m.col_idx), _f64(m.values))
    out = np.zeros(m.n) if y is None else y
    used = lib().or_spmv_csr_omp(m.n, rp, ci, va, x, float(alpha), float(beta), out, int(threads))
    return out, used


def coo_to_csr(n, ncols, row, col, val, sum_f32=False):
    """COO triplets -> (row_ptr, col_idx, values); duplicates summed in
    input order."""
    row, col = _i32(row), _i32(col)
    nnz = row.shape[0]
    rp = np.zeros(n + 1, dtype=np.int32)
    oc = np.zeros(max(nnz, 1), dtype=np.int32)
    ov = np.zeros(max(nnz, 1), dtype=np.float64)
    out = lib().or_coo_to_csr(n, ncols, nnz, row, col, _f64(val), 1 if sum_f32 else 0, rp, oc, ov)
    if out < 0:
        raise ValueError("COO index out of range")
    return rp, oc[:out].copy(), ov[:out].copy()


def ell_stride(n):
    """ELL stride: n rounded up to a multiple of 32."""
    return ((n + 31) // 32) * 32


def csr_to_ell(m, stride=None):
    """Returns (K, stride, col[K*stride], val[K*stride])."""
    rp = _i32(m.row_ptr)
    K = lib().or_ell_width(m.n, rp)
    stride = ell_stride(m.n) if stride is None else stride
    ecol = np.zeros(max(K * stride, 1), dtype=np.int32)
    ev = np.zeros(max(K * stride, 1), dtype=np.float64)
    lib().or_csr_to_ell(m.n, rp, _i32(m.col_idx), _f64(m.values), K, stride, ecol, ev)
    return K, stride, ecol[:K * stride], ev[:K * stride]


def ell_to_csr(n, K, stride, ecol, ev):
    nnz_max = max(int((np.asarray(ecol) >= 0).sum()), 1)
    rp = np.zeros(n + 1, dtype=np.int32)
    ci = np.zeros(nnz_max, dtype=np.int32)
    va = np.zeros(nnz_max, dtype=np.float64)
    ec = np.ascontiguousarray(ecol, dtype=np.int32) if K * stride else np.zeros(1, np.int32)
    evv = _f64(ev) if K * stride else np.zeros(1)
    out = lib().or_ell_to_csr(n, K, stride, ec, evv, rp, ci, va)
    return rp, ci[:out].copy(), va[:out].copy()


def csr_to_sellp(m, S=32, f=1):
    """Returns (slice_lengths, slice_sets, col, val)."""
    rp = _i32(m.row_ptr)
    ns = (m.n + S - 1) // S
    sl = np.zeros(max(ns, 1), dtype=np.int32)
    ss = np.zeros(ns + 1, dtype=np.int64)
    lib().or_sellp_sizes(m.n, rp, S, f, sl, ss)
    total = int(ss[ns]) * S
    sc = np.zeros(max(total, 1), dtype=np.int32)
    sv = np.zeros(max(total, 1), dtype=np.float64)
    lib().or_csr_to_sellp(m.n, rp, _i32(m.col_idx), _f64(m.values), S, ss, sc, sv)
    return sl[:ns], ss, sc[:total], sv[:total]


def sellp_to_csr(n, S, slice_lengths, slice_sets, scol, sval):
    nnz_max = max(int((np.asarray(scol) >= 0).sum()), 1)
    rp = np.zeros(n + 1, dtype=np.int32)
    ci = np.zeros(nnz_max, dtype=np.int32)
    va = np.zeros(nnz_max, dtype=np.float64)
    sl = np.ascontiguousarray(slice_lengths, dtype=np.int32)
    if sl.size == 0:
        sl = np.zeros(1, np.int32)
    sc = np.ascontiguousarray(scol, dtype=np.int32)
    if sc.size == 0:
        sc = np.zeros(1, np.int32)
    sv = _f64(sval) if np.asarray(sval).size else np.zeros(1)
    out = lib().or_sellp_to_csr(n, S, sl, np.ascontiguousarray(slice_sets, dtype=np.int64),
                                sc, sv, rp, ci, va)
    return rp, ci[:out].copy(), va[:out].copy()


def jacobi(m):
    """Inverse diagonal; raises ZeroDivisionError on a zero/missing diagonal."""
    d = np.zeros(max(m.n, 1))
    st = lib().or_jacobi_gen(m.n, _i32(m.row_ptr), _i32(m.col_idx), _f64(m.values), d)
    if st != OK:
        raise ZeroDivisionError("zero or missing diagonal")
    return d[:m.n]


def block_jacobi(m, bs):
    """Inverted diagonal blocks of bs rows, shape (nblocks, bs, bs); raises
    ZeroDivisionError on a singular block."""
    nb = (m.n + bs - 1) // bs
    out = np.zeros(max(nb, 1) * bs * bs)
    st = lib().or_block_jacobi_gen(m.n, _i32(m.row_ptr), _i32(m.col_idx), _f64(m.values), bs, out)
    if st != OK:
        raise ZeroDivisionError("singular diagonal block")
    return out[:nb * bs * bs].reshape(nb, bs, bs)


def block_jacobi_apply(n, bs, binv, r):
    z = np.zeros(n)
    lib().or_block_jacobi_apply(n, bs, _f64(binv).reshape(-1), _f64(r), z)
    return z


def ilu0(m):
    """ILU(0) factors in A's CSR pattern (L strictly lower with unit
    diagonal implied, U on and above the diagonal).  Raises ValueError for
    rows whose columns are not strictly ascending and ZeroDivisionError for
    a missing diagonal or a zero pivot."""
    lu = np.zeros(max(int(m.nnz), 1))
    st = lib().or_ilu0(m.n, _i32(m.row_ptr), _i32(m.col_idx), _f64(m.values), lu)
    if st == ERR_INVALID:
        raise ValueError("ILU(0) needs strictly ascending columns in every row")
    if st != OK:
        raise ZeroDivisionError("missing diagonal or zero pivot")
    return lu[:m.nnz]


def ilu0_apply(m, lu, r):
    """z = U^-1 L^-1 r with the factors of ilu0(m)."""
    z = np.zeros(max(m.n, 1))
    lib().or_ilu0_apply(m.n, _i32(m.row_ptr), _i32(m.col_idx),
                        _f64(lu) if np.asarray(lu).size else np.zeros(1), _f64(r), z)
    return z[:m.n]


def trsv(m, b, upper=False, unit=False):
    """x with T x = b for the lower (or upper) triangle of m including its
    diagonal (unit: diagonal taken as 1).  Raises ValueError for unsorted
    columns or a missing diagonal, ZeroDivisionError for a zero diagonal."""
    x = np.zeros(max(m.n, 1))
    st = lib().or_trsv(m.n, _i32(m.row_ptr), _i32(m.col_idx),
                       _f64(m.values) if m.nnz else np.zeros(1), int(upper), int(unit),
                       _f64(b) if m.n else np.zeros(1), x)
    if st == ERR_INVALID:
        raise ValueError("triangular solve needs ascending columns and a stored diagonal")
    if st != OK:
        raise ZeroDivisionError("zero diagonal")
    return x[:m.n]


def solve(m, b, x0=None, method=CG, precond=0, tol=1e-10, max_iters=1000,
          krylov_dim=30, history=False, block_size=0):
    """Runs CG / BiCGSTAB / GMRES(m) / CGS; precond 0 none, 1 Jacobi,
    2 block-Jacobi with `block_size` rows per block, 3 ILU(0).  Returns (x, info
    dict[, history])."""
    x = np.zeros(m.n) if x0 is None else _f64(x0).copy()
    o = Opts(method, precond, tol, max_iters, krylov_dim, block_size)
    info = Info()
    hist = np.full(max_iters + 2, np.nan) if history else None
    f = {CG: lib().or_cg, BICGSTAB: lib().or_bicgstab, GMRES: lib().or_gmres,
         CGS: lib().or_cgs}[method]
    if m.n == 0:
        x = np.zeros(0)
        info.status = OK
        return (x, info.as_dict(), hist) if history else (x, info.as_dict())
    f(m.n, _i32(m.row_ptr), _i32(m.col_idx), _f64(m.values), _f64(b), x,
      ctypes.byref(o), ctypes.byref(info),
      hist.ctypes.data_as(ctypes.c_void_p) if history else None)
    d = info.as_dict()
    if history:
        return x, d, hist[:d["iters"] + 1]
    return x, d


def true_rel_residual(m, b, x):
    """||b - A x|| / ||b|| with the compensated oracle SpMV."""
    r = spmv(m, x, alpha=-1.0, beta=1.0, y=b)
    bn = np.linalg.norm(_f64(b))
    return float(np.linalg.norm(r) / bn) if bn > 0 else float(np.linalg.norm(r))
