"""The allocation-free entry point, fem_assemble_noalloc, against the regular fem_assemble.

fem_assemble_noalloc serves callers that cannot allocate device memory while they assemble, for
example an application that gives all device memory to its own pool at start-up, or a loop with a
fixed latency budget. Its per-element scratch is a fixed 16 MiB device array inside the library.
These tests call it through the C ABI, twice in a row on meshes of different dimension and size (the
shared array keeps the previous call's contents), and compare each result with the deterministic
fem_assemble on the same inputs, within the parity tolerance used by the other GPU tests. They also
check that a mesh beyond the array's capacity is refused before any work is launched.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import meshgen
import oracle
from tests._common import TOL, assert_close_scaled, dev, host

pytestmark = pytest.mark.gpu

fa = pytest.importorskip("paper_1804_05156_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fa.build()
    oracle.build()


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _noalloc(p, node, k, f_kind, val, b):
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fa.lib().fem_assemble_noalloc(p.handle, _ptr(node), _ptr(k), f_kind, None, _ptr(val), _ptr(b), s)


def _case(d, n, seed):
    m = meshgen.square_mesh(n, 0.2, seed, permute=True) if d == 2 else meshgen.kuhn_mesh(n, 0.1, seed)
    k = meshgen.lognormal(seed, meshgen.TAG_COEF, m["elem"].shape[0])
    return m["node"], m["elem"], k


def test_noalloc_matches_fem_assemble_on_two_calls_in_a_row():
    # first call: a 3-D mesh; second call: a larger 2-D mesh close to the 2-D limit
    for d, n, seed, f_kind in ((3, 20, 31, fa.FEM_F_SINPROD), (2, 330, 32, fa.FEM_F_SINPROD)):
        node, elem, k = _case(d, n, seed)
        assert elem.shape[0] * (9 if d == 2 else 14) <= (1 << 21)
        p = fa.Pattern(dev(elem), node.shape[0])
        nd, kd = dev(node), dev(k)
        val = torch.full((p.nnz,), np.nan, dtype=torch.float64, device="cuda")
        b = torch.full((p.N,), np.nan, dtype=torch.float64, device="cuda")
        rc = _noalloc(p, nd, kd, f_kind, val, b)
        assert rc == fa.FEM_OK, fa.lib().fem_last_error_string()
        fa.get_error()
        v_ref, b_ref = fa.assemble(p, nd, kd, f_kind, None, fa.FEM_DETERMINISTIC)
        fa.get_error()
        _, _, _, scale = oracle.assemble(d, node, elem, k)
        assert_close_scaled(host(val), host(v_ref), scale, tol=TOL, what="noalloc stiffness")
        assert_close_scaled(host(b), host(b_ref), np.abs(host(b_ref)), tol=TOL, what="noalloc rhs")


def test_noalloc_refuses_meshes_beyond_its_scratch():
    node, elem, k = _case(2, 342, 33)  # 233,928 triangles > 2^21 / 9
    p = fa.Pattern(dev(elem), node.shape[0])
    val = torch.full((p.nnz,), 7.0, dtype=torch.float64, device="cuda")
    b = torch.full((p.N,), 7.0, dtype=torch.float64, device="cuda")
    rc = _noalloc(p, dev(node), dev(k), fa.FEM_F_CONST, val, b)
    assert rc == fa.FEM_ERR_ARG
    assert b"too large" in fa.lib().fem_last_error_string()
    torch.cuda.synchronize()
    assert bool((val == 7.0).all()) and bool((b == 7.0).all())
