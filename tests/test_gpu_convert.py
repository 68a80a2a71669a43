"""Bit-exact GPU parity of the format conversions against the CPU oracle,
through the C ABI: COO -> CSR on the device (every row sorter, duplicate
summation in each value type, host and device triplets, the full 2^22-row
power-law matrix permuted), CSR -> ELL and CSR -> SELL-P for every slice
size and stride factor (including the padding and the virtual rows of the
last slice), and the padded formats back to CSR.

The conversions do no arithmetic except the duplicate sums of COO -> CSR
(summed in input order: double for FP64 input, float for FP32, BF16 and
FP16 input, the last two rounded once at the end), so every integer array
and every stored value must match the oracle bit for bit.
"""
import numpy as np
import pytest

import oracle
import paper_2510_08230_gb300 as gk
from paper_2510_08230_gb300 import workloads as W
from gpu_util import (bf16_bits_to_f64, bf16_round_f64, ensure_built, f32_to_bf16_bits,
                      torch_dev)

pytestmark = pytest.mark.gpu

DTYPES = ["f64", "f32", "bf16", "f16"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


# ------------------------------------------------------------------ helpers

def _bits(a):
    """Integer view of a value array (bit-exact comparison, signed zeros
    and NaN payloads included)."""
    a = np.ascontiguousarray(a)
    return a.view({8: np.uint64, 4: np.uint32, 2: np.uint16}[a.dtype.itemsize])


def _abi_values(v64, dtype):
    """float64 test values -> the ABI array of dtype (each value rounded to
    nearest even once: numpy for F32/F16, the bfloat16 definition for BF16)."""
    if dtype == "f64":
        return np.ascontiguousarray(v64, dtype=np.float64)
    if dtype == "f32":
        return np.ascontiguousarray(v64, dtype=np.float32)
    if dtype == "f16":
        return np.ascontiguousarray(np.asarray(v64, dtype=np.float64).astype(np.float16))
    return f32_to_bf16_bits(np.asarray(v64, dtype=np.float32))


def _as_f64(abi, dtype):
    return bf16_bits_to_f64(abi) if dtype == "bf16" else np.asarray(abi, dtype=np.float64)


def _from_oracle_sum(v, dtype):
    """The oracle's duplicate sums (FP64, or the float sum promoted to FP64)
    stored in dtype: F32 exact, BF16/F16 the one final rounding."""
    if dtype == "f64":
        return np.asarray(v, dtype=np.float64)
    f = np.asarray(v, dtype=np.float32)
    if dtype == "f32":
        return f
    if dtype == "f16":
        return f.astype(np.float16)
    return f32_to_bf16_bits(f)


def _coo_on_gpu(n, ncols, row, col, vals, dtype, mem):
    row = np.ascontiguousarray(row, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if mem == "device":
        import torch
        dev = torch_dev()
        up = vals.view(np.int16) if vals.dtype == np.uint16 else vals  # raw bits
        r, c, v = (torch.from_numpy(a.copy()).to(dev) for a in (row, col, up))
        h = gk.gk_matrix_create_coo(n, ncols, row.shape[0], r, c, v, dtype)
        torch.cuda.synchronize()
    else:
        h = gk.gk_matrix_create_coo(n, ncols, row.shape[0], row, col, vals, dtype)
    return gk.Matrix(h)


def _check_coo(n, ncols, row, col, v64, dtype, mem="host"):
    vals = _abi_values(v64, dtype)
    A = _coo_on_gpu(n, ncols, row, col, vals, dtype, mem)
    got = A.export()
    A.close()
    rp, ci, va = oracle.coo_to_csr(n, ncols, row, col, _as_f64(vals, dtype),
                                   sum_f32=dtype != "f64")
    want = _from_oracle_sum(va, dtype)
    assert np.array_equal(got["row_ptr"], rp), "row_ptr"
    assert np.array_equal(got["col_idx"], ci), "col_idx"
    assert got["values"].dtype == want.dtype
    assert np.array_equal(_bits(got["values"]), _bits(want)), "value bits"
    return rp, ci


# ------------------------------------------------------------------ COO -> CSR

@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mem", ["host", "device"])
def test_coo_to_csr_duplicates_unsorted(dtype, mem):
    """Unsorted triplets, ~30 % repeated positions (some repeated many
    times, so the input-order summation is visible in float), rows of up to
    ~60 entries (the 2..32-lane and block sorters)."""
    n, ncols = 1500, 900
    row, col, v = W.random_coo(n, ncols, 30000, seed=5, dup_frac=0.3)
    # one position repeated 40 times with values of mixed magnitude: the
    # float sum depends on the order
    rng = np.random.default_rng(9)
    k = rng.integers(0, row.size, 40)
    row[k], col[k] = 17, 23
    v = v.copy()
    v[k] = rng.standard_normal(40) * 10.0 ** rng.integers(-4, 4, 40)  # finite in FP16
    _check_coo(n, ncols, row, col, v, dtype, mem)
    assert np.bincount(row, minlength=n).max() > 32  # the block sorter ran


@pytest.mark.parametrize("dtype", DTYPES)
def test_coo_to_csr_zeros_and_empty_rows(dtype):
    """Explicit zeros (+0 and -0) are kept, duplicate zeros summed; rows
    without entries give equal row_ptr entries; the last rows are empty."""
    n, ncols = 400, 300
    rng = np.random.default_rng(3)
    used = rng.choice(n - 20, size=150, replace=False)
    row = rng.choice(used, size=2500).astype(np.int32)
    col = rng.integers(0, ncols, 2500).astype(np.int32)
    v = rng.standard_normal(2500)
    v[rng.random(2500) < 0.2] = 0.0
    v[rng.random(2500) < 0.1] = -0.0
    rp, _ = _check_coo(n, ncols, row, col, v, dtype)
    lens = np.diff(rp)
    assert (lens == 0).sum() >= n - 150 and np.all(lens[-20:] == 0)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_coo_to_csr_long_rows_all_sorters(dtype):
    """Rows of length 1..32 (shuffle sorters), 33..16384 (one block per row
    in shared memory) and > 16384 (the global-memory sorter), with
    duplicates inside the long rows."""
    n, ncols = 3000, 40000
    rng = np.random.default_rng(21)
    parts_r, parts_c = [], []
    lens = rng.integers(0, 33, n)
    lens[5], lens[77], lens[1234] = 20000, 3000, 16385
    lens[2999] = 16384
    for i, L in enumerate(lens):
        parts_r.append(np.full(L, i, np.int32))
        parts_c.append(rng.integers(0, ncols, L).astype(np.int32))
    row = np.concatenate(parts_r)
    col = np.concatenate(parts_c)
    perm = rng.permutation(row.size)
    row, col = row[perm], col[perm]
    v = rng.standard_normal(row.size)
    _check_coo(n, ncols, row, col, v, dtype, "device")


def test_coo_to_csr_degenerate():
    """nnz = 0, a single entry, n = 0 and a 1 x 1 matrix with duplicates."""
    for n, ncols, row, col in [(5, 5, [], []), (1, 1, [0], [0]), (0, 0, [], []),
                               (1, 1, [0, 0, 0], [0, 0, 0]), (3, 7, [2], [6])]:
        row = np.asarray(row, np.int32)
        col = np.asarray(col, np.int32)
        v = np.arange(1, row.size + 1, dtype=np.float64) * 0.1
        _check_coo(n, ncols, row, col, v, "f64")


def test_coo_to_csr_rejects_out_of_range():
    for row, col in [([0, 3], [0, 0]), ([0, -1], [0, 0]), ([0, 0], [0, 4])]:
        with pytest.raises(gk.GkError) as e:
            gk.gk_matrix_create_coo(3, 4, 2, np.asarray(row, np.int32),
                                    np.asarray(col, np.int32), np.ones(2), "f64")
        assert e.value.status == gk.GK_ERR_INVALID


def test_coo_to_csr_powerlaw_full_permuted():
    """The full 2^22-row power-law matrix (67M entries, rows up to 4096)
    given as randomly permuted triplets: the device result equals the
    oracle's COO -> CSR and the original CSR arrays, bit for bit."""
    m = W.power_law()
    rows = np.repeat(np.arange(m.n, dtype=np.int32), m.row_lengths())
    perm = np.random.default_rng(2512).permutation(m.nnz)
    row, col, v = rows[perm], m.col_idx[perm], m.values[perm]
    del rows, perm
    A = _coo_on_gpu(m.n, m.ncols, row, col, v, "f64", "device")
    got = A.export()
    A.close()
    assert np.array_equal(got["row_ptr"], m.row_ptr)
    assert np.array_equal(got["col_idx"], m.col_idx)
    assert np.array_equal(_bits(got["values"]), _bits(m.values))
    rp, ci, va = oracle.coo_to_csr(m.n, m.ncols, row, col, v)
    assert np.array_equal(rp, m.row_ptr) and np.array_equal(ci, m.col_idx)
    assert np.array_equal(_bits(va), _bits(m.values))


# ------------------------------------------------------------------ CSR -> ELL / SELL-P

def _shuffled_rows(m, seed):
    """m with the entries of every row in a random order (the padded
    layouts keep CSR order, which sorted columns would not reveal)."""
    rng = np.random.default_rng(seed)
    ci, va = m.col_idx.copy(), m.values.copy()
    for i in range(m.n):
        a, b = m.row_ptr[i], m.row_ptr[i + 1]
        p = rng.permutation(b - a) + a
        ci[a:b], va[a:b] = m.col_idx[p], m.values[p]
    return W.CSR(m.n, m.ncols, m.row_ptr, ci, va)


PAD_MATS = {
    "rand_33x40": lambda: W.random_csr(33, 40, 0.2, 3, empty_rows=5, full_rows=1),
    "rand_1x1": lambda: W.random_csr(1, 1, 1.0, 1),
    "rand_301x50": lambda: _shuffled_rows(W.random_csr(301, 50, 0.15, 8, empty_rows=40), 1),
    "lap3d_17": lambda: W.laplacian_3d(17),
    "powerlaw_5k": lambda: W.power_law(5003, max_len=300, seed=4),
    "empty_rows_only": lambda: W.CSR(45, 45, np.zeros(46, np.int32), np.zeros(0, np.int32),
                                     np.zeros(0)),
}


def _device_csr(m, dtype):
    """A CSR handle whose stored values are m's values in dtype; returns
    (handle, those stored values as float64)."""
    A = gk.Matrix.from_csr(m, dtype)
    got = A.export()
    return A, _as_f64(got["values"], dtype)


def _same_values(got, want64, dtype):
    """got (dtype array) equals want64 exactly, padding +0.0 included."""
    want = _abi_values(want64, dtype)
    assert np.array_equal(_bits(got), _bits(want))


@pytest.mark.parametrize("name", list(PAD_MATS))
@pytest.mark.parametrize("dtype", DTYPES)
def test_csr_to_ell_bit_exact(name, dtype):
    m = PAD_MATS[name]()
    A, v = _device_csr(m, dtype)
    mr = W.CSR(m.n, m.ncols, m.row_ptr, m.col_idx, v)
    K, stride, ecol, ev = oracle.csr_to_ell(mr)
    E = A.convert("ell")
    d = E.desc
    assert (d["ell_width"], d["ell_stride"], d["stored"]) == (K, stride, K * stride)
    got = E.export()
    assert np.array_equal(got["col"], ecol)
    _same_values(got["values"], ev, dtype)
    # padding is col -1 with +0.0, including rows n..stride-1
    pad = ecol < 0
    assert np.all(_bits(got["values"])[pad] == 0)
    # back to CSR: the original arrays
    C = E.convert("csr")
    back = C.export()
    assert np.array_equal(back["row_ptr"], m.row_ptr)
    assert np.array_equal(back["col_idx"], m.col_idx)
    _same_values(back["values"], v, dtype)
    orp, oci, ova = oracle.ell_to_csr(m.n, K, stride, ecol, ev)
    assert np.array_equal(orp, m.row_ptr) and np.array_equal(oci, m.col_idx)
    for H in (C, E, A):
        H.close()


@pytest.mark.parametrize("name", list(PAD_MATS))
@pytest.mark.parametrize("S", [8, 16, 32, 64])
@pytest.mark.parametrize("f", [1, 2, 4])
def test_csr_to_sellp_bit_exact(name, S, f):
    m = PAD_MATS[name]()
    dtype = "f64"
    A, v = _device_csr(m, dtype)
    mr = W.CSR(m.n, m.ncols, m.row_ptr, m.col_idx, v)
    sl, ss, scol, sv = oracle.csr_to_sellp(mr, S, f)
    P = A.convert("sellp", None, S, f)
    d = P.desc
    assert (d["slice_size"], d["stride_factor"], d["num_slices"]) == (S, f, sl.size)
    assert d["stored"] == int(ss[-1]) * S
    got = P.export()
    if sl.size:
        assert np.array_equal(got["slice_lengths"], sl)
    assert np.array_equal(got["slice_sets"], ss)
    assert np.array_equal(got["col"], scol)
    _same_values(got["values"], sv, dtype)
    assert np.all(_bits(got["values"])[scol < 0] == 0)
    # the virtual rows of the last partial slice are all padding
    if m.n % S and sl.size:
        s = sl.size - 1
        block = got["col"][int(ss[s]) * S:int(ss[s + 1]) * S].reshape(-1, S)
        assert np.all(block[:, m.n - s * S:] == -1)
    C = P.convert("csr")
    back = C.export()
    assert np.array_equal(back["row_ptr"], m.row_ptr)
    assert np.array_equal(back["col_idx"], m.col_idx)
    _same_values(back["values"], v, dtype)
    orp, oci, _ = oracle.sellp_to_csr(m.n, S, sl, ss, scol, sv)
    assert np.array_equal(orp, m.row_ptr) and np.array_equal(oci, m.col_idx)
    for H in (C, P, A):
        H.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("S,f", [(32, 1), (8, 4), (64, 2)])
def test_csr_to_sellp_value_types(dtype, S, f):
    """SELL-P of the narrow value types: the same layout, values stored in
    the type bit for bit (the conversion only moves them)."""
    m = PAD_MATS["rand_301x50"]()
    A, v = _device_csr(m, dtype)
    mr = W.CSR(m.n, m.ncols, m.row_ptr, m.col_idx, v)
    sl, ss, scol, sv = oracle.csr_to_sellp(mr, S, f)
    P = A.convert("sellp", None, S, f)
    got = P.export()
    assert np.array_equal(got["col"], scol) and np.array_equal(got["slice_sets"], ss)
    _same_values(got["values"], sv, dtype)
    P.close()
    A.close()


def test_ell_to_sellp_and_narrowing_conversions():
    """Padded -> padded goes through the CSR view (ELL -> SELL-P equals
    CSR -> SELL-P), and a narrowing conversion rounds each value once
    (F64 -> BF16 equals the bfloat16 rounding of the FP64 value)."""
    m = PAD_MATS["powerlaw_5k"]()
    A = gk.Matrix.from_csr(m, "f64")
    E = A.convert("ell")
    P1 = E.convert("sellp", None, 16, 2)
    P2 = A.convert("sellp", None, 16, 2)
    g1, g2 = P1.export(), P2.export()
    assert np.array_equal(g1["col"], g2["col"]) and np.array_equal(_bits(g1["values"]),
                                                                  _bits(g2["values"]))
    B = A.convert("csr", "bf16")
    gb = B.export()
    assert np.array_equal(bf16_bits_to_f64(gb["values"]), bf16_round_f64(m.values))
    for H in (B, P2, P1, E, A):
        H.close()
