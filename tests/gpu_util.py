"""Helpers shared by the GPU parity tests: building the library, moving
arrays to the device, and the per-row SpMV tolerance against the oracle.

Tolerance (per row i): |y_i - y_oracle_i| <= tol * (|alpha| sum_j |a_ij x_j|
+ |beta| |y_i|), tol = 1e-13 for FP64 and 1e-5 for FP32 / BF16- / FP16-
stored values (the oracle then uses the rounded A and FP32 x in FP64).
It is scaled by the absolute row sum because stencil rows cancel to ~0.
"""
import numpy as np

import oracle
import paper_2510_08230_gb300 as gk
from paper_2510_08230_gb300 import workloads as W

TOL = {"f64": 1e-13, "f32": 1e-5, "bf16": 1e-5, "f16": 1e-5}


def ensure_built():
    import __graft_entry__
    __graft_entry__.build()


def torch_dev():
    import torch
    return torch.device("cuda:0")


def vec_dtype(dtype):
    import torch
    return torch.float64 if dtype == "f64" else torch.float32


def bf16_round_f64(v):
    """float64 -> nearest bfloat16 (ties to even) in one rounding step, as a
    float64 (finite values inside the float32 exponent range)."""
    b = np.ascontiguousarray(v, dtype=np.float64).view(np.uint64)
    q = b >> np.uint64(45)
    rem = b & np.uint64((1 << 45) - 1)
    half = np.uint64(1 << 44)
    up = (rem > half) | ((rem == half) & ((q & np.uint64(1)) == np.uint64(1)))
    return ((q + up.astype(np.uint64)) << np.uint64(45)).view(np.float64)


def f32_to_bf16_bits(a):
    """bfloat16 bit patterns (uint16) of float32 values, rounded to nearest
    even (finite inputs), written from the bfloat16 definition: the upper 16
    bits of the float32 encoding after rounding away the lower 16."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    low = u & np.uint64(0xFFFF)
    hi = u >> np.uint64(16)
    up = (low > 0x8000) | ((low == 0x8000) & ((hi & np.uint64(1)) == np.uint64(1)))
    return (hi + up.astype(np.uint64)).astype(np.uint16)


def bf16_bits_to_f64(bits):
    """The float64 value of bfloat16 bit patterns (exact)."""
    u = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << np.uint32(16)
    return u.view(np.float32).astype(np.float64)


def rounded_values(m, dtype):
    """Matrix values as the GPU stores them, promoted to float64."""
    v = np.asarray(m.values)
    if dtype == "f64":
        return v.astype(np.float64)
    if v.dtype == np.float64 and dtype == "bf16":
        return bf16_round_f64(v)
    if dtype == "f16":  # IEEE half, one rounding to nearest even from the input type
        return v.astype(np.float16).astype(np.float64)
    f = v.astype(np.float32)
    if dtype == "f32":
        return f.astype(np.float64)
    return bf16_bits_to_f64(f32_to_bf16_bits(f))


def rounded_vector(x, dtype):
    x = np.asarray(x)
    return x.astype(np.float64) if dtype == "f64" else x.astype(np.float32).astype(np.float64)


def oracle_apply(m, x, alpha, beta, y0, dtype):
    """Oracle result and the per-row error scale for a device SpMV in dtype."""
    mv = W.CSR(m.n, m.ncols, m.row_ptr, m.col_idx, rounded_values(m, dtype))
    xv = rounded_vector(x, dtype)
    y0v = rounded_vector(y0, dtype) if y0 is not None else np.zeros(m.n)
    ref = oracle.spmv(mv, xv, alpha, beta, y0v)
    absm = W.CSR(m.n, m.ncols, m.row_ptr, m.col_idx, np.abs(mv.values))
    scale = abs(alpha) * oracle.spmv(absm, np.abs(xv)) + abs(beta) * np.abs(y0v)
    return ref, scale


def assert_rows_close(y, ref, scale, tol, what=""):
    y = np.asarray(y, dtype=np.float64)
    err = np.abs(y - ref)
    bad = err > tol * scale + 1e-300
    if bad.any():
        i = int(np.argmax(err - tol * scale))
        raise AssertionError(f"{what}: {bad.sum()} rows off; row {i}: got {y[i]!r} want "
                             f"{ref[i]!r} (scale {scale[i]:.3e}, tol {tol})")


def sub_rows(m, rows):
    """The CSR made of the given rows of m (for sampling huge matrices)."""
    rows = np.asarray(rows, dtype=np.int64)
    lens = m.row_ptr[rows + 1].astype(np.int64) - m.row_ptr[rows]
    rp = np.zeros(rows.size + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    idx = np.concatenate([np.arange(m.row_ptr[r], m.row_ptr[r + 1]) for r in rows]) \
        if rows.size else np.zeros(0, np.int64)
    return W.CSR(rows.size, m.ncols, rp.astype(np.int32), m.col_idx[idx], m.values[idx])
