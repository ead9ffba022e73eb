"""The C ABI library builds, loads and exports every symbol include/psi.h declares; the
binding's argument lists and the ctypes structs match the header; host-side argument
checks need no GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "psi.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(psi_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2206_09960_gb300 import _binding

    return _binding.load(build_if_missing=True)


def test_every_declared_symbol_is_exported(lib):
    from paper_2206_09960_gb300 import _binding

    names = _declared_functions()
    assert set(names) == set(_binding.EXPORTS), names
    so = os.path.join(ROOT, "paper_2206_09960_gb300", "libpsi_gb300.so")
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(psi_\w+)", out))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)


def _declarations():
    """(name, [parameter text]) of every function include/psi.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    out = []
    for name, params in re.findall(r"\b(psi_[a-z_]+)\s*\(([^;{}]*?)\)\s*;", text, flags=re.S):
        p = params.strip()
        out.append((name, [] if p in ("", "void") else [x.strip() for x in p.split(",")]))
    return out


def _kind_of_c(param):
    if "*" in param:
        return "ptr"
    base = param.split()[-2] if len(param.split()) > 1 else param
    return {"int64_t": "i64", "uint64_t": "u64", "int32_t": "i32", "psi_status": "i32", "int": "i32",
            "double": "f64", "float": "f32"}[base]


def _kind_of_ctypes(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return "ptr"
    return {ctypes.c_int64: "i64", ctypes.c_uint64: "u64", ctypes.c_int32: "i32", ctypes.c_double: "f64",
            ctypes.c_float: "f32"}[t]


def test_binding_signatures_match_header(lib):
    """Every declared function has the binding's argument list: the same number of
    parameters, each of the same kind (64- or 32-bit integer, double, float, pointer)."""
    decls = _declarations()
    assert sorted(n for n, _ in decls) == _declared_functions()
    for name, params in decls:
        at = getattr(lib, name).argtypes
        assert at is not None, name
        assert [_kind_of_c(p) for p in params] == [_kind_of_ctypes(t) for t in at], name


def test_struct_layout_matches_header(tmp_path):
    from paper_2206_09960_gb300 import _binding as B

    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "psi.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(psi_options), sizeof(psi_solve_info),"
        " sizeof(psi_graph_stats), sizeof(psi_allocator), offsetof(psi_options, stream),"
        " offsetof(psi_solve_info, spmv_ms)); return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(B.psi_options), ctypes.sizeof(B.psi_solve_info), ctypes.sizeof(B.psi_graph_stats),
            ctypes.sizeof(B.psi_allocator), B.psi_options.stream.offset, B.psi_solve_info.spmv_ms.offset]
    assert got == want


def test_host_side_calls(lib):
    from paper_2206_09960_gb300 import _binding as B

    o = B.psi_options_default()
    assert (o.precision, o.tol_mode, o.bnorm_mode, o.self_loops, o.reorder) == (
        B.PSI_FP32_REFINE, B.PSI_TOL_PSI, B.PSI_BNORM_NONE, B.PSI_REJECT, 1)
    assert B.status_name(B.PSI_ERR_NOT_CONVERGED) == "PSI_ERR_NOT_CONVERGED"
    assert B.psi_version() >= 100
    # argument checks happen before any CUDA call
    h = ctypes.c_void_p()
    st = lib.psi_graph_create(0, 0, None, None, None, None, None, ctypes.byref(h))
    assert st == B.PSI_ERR_INVALID_ARG and not h.value
    assert "n must be" in B.last_error()
    st = lib.psi_graph_create(10, 5, None, None, None, None, None, ctypes.byref(h))
    assert st == B.PSI_ERR_INVALID_ARG
    bad = B.psi_options_default()
    bad.precision = 9
    lam = (ctypes.c_double * 10)()
    st = lib.psi_graph_create(10, 0, None, None, lam, lam, ctypes.byref(bad), ctypes.byref(h))
    assert st == B.PSI_ERR_INVALID_ARG
    assert lib.psi_solve(None, 1e-8, 10, None, None) == B.PSI_ERR_INVALID_ARG
    assert lib.psi_scores(None, None) == B.PSI_ERR_INVALID_ARG
    assert lib.psi_topk(None, 5, None, None) == B.PSI_ERR_INVALID_ARG
    lib.psi_graph_destroy(None)


def test_product_path_does_not_import_the_oracle():
    """The CUDA path and the oracle share no code and neither imports the other."""
    pkg = os.path.join(ROOT, "paper_2206_09960_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", text).replace("oracle/", ""), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2206_09960_gb300" not in text, f
