"""The C ABI: the library loads and exports every function include/spmvc.h
declares (no GPU needed), and host-side argument checks return statuses."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1612_00530_gb300 as P
from paper_1612_00530_gb300 import build as lib_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    lib_build.build()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "spmvc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|const char \*)\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for must in ("spmv_build", "spmv_compress", "spmv_decompress", "spmv_apply", "spmm_apply", "cg_solve"):
        assert must in names


def test_every_declared_symbol_is_exported():
    lib = ctypes.CDLL(P.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_strerror_and_version():
    lib = P.library()
    for code in range(9):
        assert lib.spmv_strerror(code)
    assert b"sm_103a" in lib.spmv_version()


def test_invalid_arguments_rejected_before_device_work():
    lib = P.library()
    assert lib.spmv_apply(None, None, None, None) == P.SPMV_EINVAL
    assert lib.spmv_build(None, None) == P.SPMV_EINVAL
    assert lib.spmv_batch_autotune(None, 1, None) == P.SPMV_EINVAL
    assert lib.spmv_batch_launch(None, None) == P.SPMV_EINVAL
    assert lib.spmv_batch_create(0, None, None, None, None) == P.SPMV_EINVAL
    # columns out of order
    with pytest.raises(P.SpmvError) as e:
        P.spmv_build_csr(np.array([0, 2]), np.array([0, 0]), np.array([1.0, 2.0]))
    assert e.value.status == P.SPMV_EINVAL
    with pytest.raises(P.SpmvError):
        P.spmv_build("hpcg", 0, 3, 3)


def test_fast_order_refused_for_unsuitable_tables():
    A = P.spmv_build_csr(np.array([0, 1, 2]), np.array([0, 1]), np.array([0.1, 3.0]))
    C = P.spmv_compress(A, format="pattern")
    assert P.spmv_info(C)["fast_eligible"] == 0
    with pytest.raises(P.SpmvError) as e:
        P.spmv_set_order(C, "fast")
    assert e.value.status == P.SPMV_EUNSUPPORTED


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Every struct the binding mirrors has the C compiler's size and field
    offsets (host-only: compiles a tiny C program against include/spmvc.h)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [P.spmv_gen_desc, P.spmv_opts, P.spmv_info_t, P.spmv_cg_opts, P.spmv_cg_result]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "spmvc.h"', "int main(void) {"]
    for s in structs:
        lines.append(f'    printf("{s.__name__} size %zu\\n", sizeof({s.__name__}));')
        for name, _ in s._fields_:
            lines.append(f'    printf("{s.__name__} {name} %zu\\n", offsetof({s.__name__}, {name}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for s in structs:
        assert got[(s.__name__, "size")] == ctypes.sizeof(s), s.__name__
        for name, _ in s._fields_:
            assert got[(s.__name__, name)] == getattr(s, name).offset, (s.__name__, name)
