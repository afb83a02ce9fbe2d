"""The C ABI library builds, loads without a GPU, and exports every entry point femasm.h declares.
Also host-side argument checks that return before any device work."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "femasm.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fem_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    import paper_1804_05156_gb300 as fa
    return fa.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["fem_mesh_build_pattern", "fem_assemble_stiffness", "fem_assemble_rhs", "fem_apply_dirichlet",
                 "fem_assemble_backward", "fem_batch_plan", "fem_batch_assemble", "fem_get_error"]:
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    L = C.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(L, s)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(fem_[a-z0-9_]+)\b", out))
    assert set(declared_symbols()) <= exported


def test_binding_names_match_header(libpath):
    import paper_1804_05156_gb300 as fa
    for s in declared_symbols():
        assert hasattr(fa.lib(), s)


def test_host_side_argument_checks(libpath):
    """These checks return before touching the device, so they run without a GPU."""
    import paper_1804_05156_gb300 as fa
    L = fa.lib()
    h = C.c_void_p()
    assert L.fem_mesh_build_pattern(4, 10, 10, None, C.byref(h), None) == fa.FEM_ERR_ARG
    assert b"d must be" in L.fem_last_error_string()
    assert L.fem_mesh_build_pattern(2, -1, 10, None, C.byref(h), None) == fa.FEM_ERR_ARG
    assert L.fem_mesh_build_pattern(3, 10, 1 << 28, None, C.byref(h), None) == fa.FEM_ERR_ARG
    assert L.fem_mesh_build_pattern(2, 10, 5, None, C.byref(h), None) == fa.FEM_ERR_ARG  # null elem
    assert L.fem_mesh_build_pattern(2, 10, 5, C.c_void_p(2), C.byref(h), None) == fa.FEM_ERR_ARG  # misaligned
    assert L.fem_mesh_build_pattern(2, 10, 5, C.c_void_p(16), None, None) == fa.FEM_ERR_ARG  # null out
    assert L.fem_assemble(None, None, None, 0, None, None, None, 0, None) == fa.FEM_ERR_ARG
    assert L.fem_batch_plan(2, 0, None, None, None, C.byref(h), None) == fa.FEM_ERR_ARG
    assert L.fem_pattern_barrier_fault(None, 1, 16) == fa.FEM_ERR_ARG
    assert L.fem_csr_spmv(None, None, None, None, None, None) == fa.FEM_ERR_ARG
    assert L.fem_cg_solve_csr(None, None, None, None, None, None, 10, C.c_double(1e-8), None, None, None) == fa.FEM_ERR_ARG
    assert L.fem_cg_solve(None, None, None, None, None, None, None, 10, C.c_double(1e-8), None, None, None) == fa.FEM_ERR_ARG
    assert L.fem_launch_count() >= 0


def test_oracle_and_product_share_no_code():
    """The oracle and the CUDA library are independent: neither includes, imports or loads the other."""
    pkg = os.path.join(ROOT, "paper_1804_05156_gb300")
    bad_pkg = re.compile(r"^\s*(import\s+oracle|from\s+oracle|#include\s+\S*oracle)|liboracle", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                assert not bad_pkg.search(open(os.path.join(dirpath, f)).read()), f
    bad_ora = re.compile(r"^\s*(import\s+paper_1804_05156_gb300|from\s+paper_1804_05156_gb300|#include\s+\S*femasm)"
                         r"|libfemasm", re.M)
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            assert not bad_ora.search(open(os.path.join(ROOT, "oracle", f)).read()), f


def test_library_rules_match_the_oracle_rules(libpath):
    """The library builds its quadrature rules on the host (Newton on the Jacobi recurrence); the oracle
    by the eigenvalues of the Jacobi matrix. Same rules to rounding, without a GPU."""
    import numpy as np

    import oracle
    import paper_1804_05156_gb300 as fa
    for d in (2, 3):
        for n in range(1, 9):
            b1, w1 = fa.fem_quad_rule(d, n)
            b2, w2 = oracle.quad_rule(d, n)
            # both orderings are (u, v[, w]) lexicographic with nodes ascending or descending per direction
            k1 = np.lexsort(b1.T[::-1])
            k2 = np.lexsort(b2.T[::-1])
            assert np.allclose(b1[k1], b2[k2], rtol=0, atol=2e-15), (d, n)
            assert np.allclose(w1[k1], w2[k2], rtol=1e-13, atol=0), (d, n)
    L = fa.lib()
    assert L.fem_quad_rule(4, 2, None, None, None) == fa.FEM_ERR_ARG
    assert L.fem_quad_rule(2, 0, None, None, None) == fa.FEM_ERR_ARG
    assert L.fem_quad_rule(2, 9, None, None, None) == fa.FEM_ERR_ARG
