"""The allocation-free entry point, fem_assemble_noalloc, against the regular fem_assemble and the oracle.

fem_assemble_noalloc serves callers that cannot allocate device memory while they assemble, for
example an application that gives all device memory to its own pool at start-up, or a loop with a
fixed latency budget. Its per-element scratch is a fixed 16 MiB device array inside the library, shared
by every call. These tests call it through the C ABI, twice in a row on meshes of different dimension
and size (the shared array keeps the previous call's contents), and check each result three ways: bit
for bit against fem_assemble on the same pattern forced to the FP64 two-pass path (the kernels the entry
point runs), within the parity tolerance of the regular float-float fem_assemble, and within that
tolerance of the oracle. A repeat call after a call on another mesh must give the same bits (no stale
scratch leaks into a result). A mesh beyond the array's capacity is refused before any work is launched.
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


def _run_noalloc(p, nd, kd, f_kind):
    val = torch.full((p.nnz,), np.nan, dtype=torch.float64, device="cuda")
    b = torch.full((p.N,), np.nan, dtype=torch.float64, device="cuda")
    rc = _noalloc(p, nd, kd, f_kind, val, b)
    assert rc == fa.FEM_OK, fa.lib().fem_last_error_string()
    fa.get_error()
    return val, b


def test_noalloc_matches_two_pass_tiles_and_oracle_on_calls_in_a_row():
    # a 3-D mesh, then a larger 2-D mesh close to the 2-D limit, then the 3-D mesh again
    cases = [(3, 20, 31, fa.FEM_F_SINPROD), (2, 330, 32, fa.FEM_F_SINPROD)]
    first = {}
    for it, (d, n, seed, f_kind) in enumerate(cases + [cases[0]]):
        node, elem, k = _case(d, n, seed)
        assert elem.shape[0] * (9 if d == 2 else 14) <= (1 << 21)
        p = fa.Pattern(dev(elem), node.shape[0])
        nd, kd = dev(node), dev(k)
        val, b = _run_noalloc(p, nd, kd, f_kind)
        # the regular (float-float) deterministic path: within tolerance
        v_df, b_df = fa.assemble(p, nd, kd, f_kind, None, fa.FEM_DETERMINISTIC)
        fa.get_error()
        # the oracle: within tolerance
        _, _, vo, scale = oracle.assemble(d, node, elem, k)
        bo = oracle.rhs(d, node, elem, oracle.F_SINPROD)
        assert_close_scaled(host(val), vo, scale, tol=TOL, what="noalloc stiffness vs oracle")
        assert_close_scaled(host(b), bo, np.abs(bo), tol=TOL, what="noalloc rhs vs oracle")
        assert_close_scaled(host(val), host(v_df), scale, tol=TOL, what="noalloc stiffness vs fem_assemble")
        assert_close_scaled(host(b), host(b_df), np.abs(bo), tol=TOL, what="noalloc rhs vs fem_assemble")
        # the FP64 two-pass path the entry point runs: the same bits
        fa.fem_pattern_force_path(p, fa.FEM_PATH_TWO_PASS)
        v_tp, b_tp = fa.assemble(p, nd, kd, f_kind, None, fa.FEM_DETERMINISTIC)
        fa.get_error()
        assert torch.equal(val, v_tp) and torch.equal(b, b_tp), "noalloc differs from the two-pass path"
        key = (d, n, seed)
        if key in first:  # the same inputs after a call on another mesh: the same bits
            assert torch.equal(val, first[key][0]) and torch.equal(b, first[key][1]), "repeat call differs"
        else:
            first[key] = (val.clone(), b.clone())
    assert len(first) == 2


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
