"""C-ABI library: loads without a GPU, exports every symbol gk.h declares,
and rejects malformed arguments before touching the device.  CPU only."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2510_08230_gb300 as gk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gk_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return gk.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "gk_apply" in names and "gk_solve" in names
    for n in names:
        assert hasattr(lib, n), n
    # the binding wraps exactly the declared entry points
    assert set(gk.EXPORTED) <= set(names)
    for n in names:
        assert n in gk.EXPORTED or hasattr(lib, n), n


def test_status_strings(lib):
    for s in (0, 1, 2, -1, -2, -3, -4, -5, -6, -7):
        assert gk.gk_status_string(s) and gk.gk_status_string(s) != "unknown status"
    assert gk.gk_status_string(99) == "unknown status"
    assert gk.gk_version() == 1


def test_invalid_arguments_rejected_on_host(lib):
    h = ctypes.c_void_p()
    rp = np.zeros(3, np.int32)
    assert lib.gk_matrix_create_csr(-1, 2, 0, rp.ctypes.data, None, None, 0, 0, None,
                                    ctypes.byref(h)) == gk.GK_ERR_INVALID
    assert lib.gk_matrix_create_csr(2, 2, 0, rp.ctypes.data, None, None, 7, 0, None,
                                    ctypes.byref(h)) == gk.GK_ERR_INVALID
    assert lib.gk_matrix_create_csr(2, 2, 5, rp.ctypes.data, None, None, 0, 0, None,
                                    ctypes.byref(h)) == gk.GK_ERR_INVALID
    assert lib.gk_matrix_create_csr(2, 2, 0, rp.ctypes.data, None, None, 0, 0, None,
                                    None) == gk.GK_ERR_INVALID
    assert lib.gk_matrix_create_coo(2, 2, 1, None, None, None, 0, 0, None,
                                    ctypes.byref(h)) == gk.GK_ERR_INVALID
    assert lib.gk_apply(None, None, None, None) == gk.GK_ERR_INVALID
    assert lib.gk_matrix_destroy(None) == gk.GK_ERR_INVALID
    assert lib.gk_matrix_describe(None, None) == gk.GK_ERR_INVALID
    assert lib.gk_solve(None, None, None, None, None, None) == gk.GK_ERR_INVALID
    assert lib.gk_precond_apply(None, gk.GK_PRECOND_ILU, 0, None, None, 0,
                                None) == gk.GK_ERR_INVALID
    assert lib.gk_ilu_factors(None, None, None) == gk.GK_ERR_INVALID
    assert lib.gk_triangular_solve(None, 0, 0, None, None, 0, None) == gk.GK_ERR_INVALID


def test_struct_layouts_match_header(lib, tmp_path):
    """ctypes mirrors of the ABI structs have the sizes and field offsets the
    C compiler gives them for gk.h."""
    import subprocess
    structs = {"gk_solve_info": gk.gk_solve_info, "gk_solve_opts": gk.gk_solve_opts,
               "gk_matrix_desc": gk.gk_matrix_desc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gk.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("%zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({name}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    expect = []
    for name, cls in structs.items():
        expect.append(ctypes.sizeof(cls))
        expect += [getattr(cls, f).offset for f, _ in cls._fields_]
    assert vals == expect


def test_product_path_does_not_import_the_oracle():
    import subprocess
    import sys
    code = ("import sys; import paper_2510_08230_gb300, paper_2510_08230_gb300.workloads; "
            "assert 'oracle' not in sys.modules, 'oracle imported by the product path'")
    subprocess.check_call([sys.executable, "-c", code], cwd=ROOT)
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2510_08230_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "gk_oracle" not in txt, f


def test_native_overhead_driver_builds_and_checks_arguments():
    """The native side of the binding-overhead measurement compiles against
    include/gk.h and libgk.so, and rejects bad arguments before any CUDA
    call (no GPU needed)."""
    import subprocess
    from paper_2510_08230_gb300 import _build
    exe = _build.build_native()
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 1 and "usage" in r.stderr
    r = subprocess.run([exe, "/nonexistent.csr", "csr", "5"], capture_output=True, text=True)
    assert r.returncode == 1 and "cannot open" in r.stderr
