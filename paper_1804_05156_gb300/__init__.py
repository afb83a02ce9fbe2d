"""GB300-native P1 finite-element assembly (Poisson), after L. Chen, "Programming of Finite Element
Methods in MATLAB" (arXiv:1804.05156).

This module is a thin ctypes binding of the C ABI in ``include/femasm.h`` (same names, argument
marshalling only): every step of the assembly runs in the CUDA kernels of ``libfemasm.so``.
PyTorch provides device memory, streams and autograd plumbing. There is no CPU fallback: if the
library has not been built, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfemasm.so")

FEM_OK = 0
FEM_ERR_ARG, FEM_ERR_INDEX, FEM_ERR_DEGENERATE, FEM_ERR_CUDA, FEM_ERR_OOM, FEM_ERR_TIMEOUT, FEM_ERR_STATE = (
    -1, -2, -3, -4, -5, -6, -7)
FEM_ERR_RANGE = -8
FEM_DETERMINISTIC, FEM_ATOMIC = 0, 1
FEM_F_CONST, FEM_F_SINPROD, FEM_F_QPVALUES = 0, 1, 2
FEM_PATH_TWO_PASS, FEM_PATH_BLOCKED, FEM_PATH_TILES, FEM_PATH_TILES_FUSED = 0, 1, 2, 3
FEM_OP_STIFFNESS, FEM_OP_MASS, FEM_OP_ANISO = 0, 1, 2

_lib = None


class FemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("femasm error %d: %s" % (code, msg))
        self.code = code


def build(force: bool = False) -> str:
    """Compile libfemasm.so in-tree for sm_103a (see buildlib.py)."""
    from . import buildlib
    return buildlib.build(force=force)


def lib():
    """The loaded C library (raises if it was not built: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FemError(FEM_ERR_STATE, "libfemasm.so is not built; run paper_1804_05156_gb300.build()")
        L = C.CDLL(LIB_PATH)
        P, I32, I64 = C.c_void_p, C.c_int, C.c_int64
        sig = {
            "fem_mesh_build_pattern": (I32, [I32, I64, I64, P, P, P]),
            "fem_pattern_info": (I32, [P, P, P, P, P, P, P, P]),
            "fem_pattern_set_locality": (I32, [P, P, P, P]),
            "fem_pattern_launch_shape": (I32, [P, P, P, P, P, P]),
            "fem_pattern_force_launch": (I32, [P, I32, I32, I32]),
            "fem_pattern_value_path": (I32, [P, P, P, P]),
            "fem_pattern_force_path": (I32, [P, I32, I32, P]),
            "fem_pattern_barrier_fault": (I32, [P, I32, I32]),
            "fem_pattern_destroy": (None, [P]),
            "fem_assemble": (I32, [P, P, P, I32, P, P, P, I32, P]),
            "fem_assemble_stiffness": (I32, [P, P, P, P, I32, P]),
            "fem_assemble_rhs": (I32, [P, P, I32, P, P, I32, P]),
            "fem_boundary_nodes": (I32, [P, P, P, P]),
            "fem_apply_dirichlet": (I32, [P, P, P, P, P, P, P, P]),
            "fem_assemble_backward": (I32, [P, P, P, I32, P, P, P, P, P, P]),
            "fem_boundary_terms": (I32, [P, P, P, P, C.c_double, C.c_double, P, P, P]),
            "fem_assemble_operator": (I32, [P, P, I32, P, P, P]),
            "fem_quad_rule": (I32, [I32, I32, P, P, P]),
            "fem_apply_stiffness": (I32, [P, P, P, P, P, P, P]),
            "fem_cg_solve": (I32, [P, P, P, P, P, P, P, I32, C.c_double, P, P, P]),
            "fem_csr_spmv": (I32, [P, P, P, P, P, P]),
            "fem_cg_solve_csr": (I32, [P, P, P, P, P, P, I32, C.c_double, P, P, P]),
            "fem_rule_points": (I32, [P, P, I32, P, P]),
            "fem_assemble_rhs_rule": (I32, [P, P, I32, I32, P, P, P]),
            "fem_side_points": (I32, [P, P, P, P]),
            "fem_mean_shift": (I32, [P, C.c_int64, P]),
            "fem_zero_average": (I32, [P, P, P, P, P]),
            "fem_batch_plan": (I32, [I32, I32, P, P, P, P, P]),
            "fem_batch_info": (I32, [P, P, P, P, P, P]),
            "fem_batch_set_locality": (I32, [P, P, P]),
            "fem_batch_assemble": (I32, [P, P, P, I32, P, P, P, I32, P]),
            "fem_batch_assemble_graph": (I32, [P, P, P, I32, P, P, P, I32, P]),
            "fem_batch_destroy": (None, [P]),
            "fem_get_error": (I32, [P]),
            "fem_last_error_string": (C.c_char_p, []),
            "fem_launch_count": (I64, []),
            "fem_assemble_noalloc": (I32, [P, P, P, I32, P, P, P, P]),
            "fem_assemble_host": (I32, [P, I32, P, P, I32, P, P, P, P]),
            "fem_timing_enable": (I32, [I32]),
            "fem_timing_report": (I32, [C.c_char_p, I64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int) -> int:
    if rc != FEM_OK:
        raise FemError(rc, lib().fem_last_error_string().decode())
    return rc


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise FemError(FEM_ERR_ARG, "expected a CUDA tensor")
    if not t.is_contiguous():
        raise FemError(FEM_ERR_ARG, "expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def launch_count() -> int:
    return int(lib().fem_launch_count())


def fem_timing_enable(on: bool) -> None:
    _check(lib().fem_timing_enable(1 if on else 0))


def fem_timing_report() -> dict:
    """{kernel name: (launches, total ms)} since the last report; synchronises the recorded events."""
    buf = C.create_string_buffer(1 << 16)
    _check(lib().fem_timing_report(buf, len(buf)))
    out = {}
    for line in buf.value.decode().splitlines():
        name, n, ms = line.rsplit(" ", 2)
        out[name] = (int(n), float(ms))
    return out


def get_error(stream=None) -> None:
    """Raise if a kernel recorded an error (synchronises the stream)."""
    _check(lib().fem_get_error(_stream(stream)))


class _DevArray:
    """Zero-copy view of a library-owned device array (kept alive by its owner)."""

    def __init__(self, ptr: int, n: int, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr or 0, False),
                                         "version": 3, "strides": None}
        self._owner = owner


class Pattern:
    """Structural CSR pattern + slot map of a mesh (``fem_mesh_build_pattern``)."""

    def __init__(self, elem: torch.Tensor, N: int, stream=None, _handle=None):
        self._h = C.c_void_p()
        if _handle is not None:
            self._h = _handle
        else:
            if elem.dtype != torch.int32 or elem.dim() != 2:
                raise FemError(FEM_ERR_ARG, "elem must be an int32 [NT, d+1] CUDA tensor")
            d = elem.shape[1] - 1
            _check(lib().fem_mesh_build_pattern(d, int(N), int(elem.shape[0]), _ptr(elem), C.byref(self._h),
                                                _stream(stream)))
        d, n, nt, nnz = C.c_int(), C.c_int64(), C.c_int64(), C.c_int64()
        rp, ci, sl = C.c_void_p(), C.c_void_p(), C.c_void_p()
        _check(lib().fem_pattern_info(self._h, C.byref(d), C.byref(n), C.byref(nt), C.byref(nnz), C.byref(rp),
                                      C.byref(ci), C.byref(sl)))
        self.d, self.N, self.NT, self.nnz = d.value, n.value, nt.value, nnz.value
        dev = torch.device("cuda", torch.cuda.current_device())
        self.row_ptr = torch.as_tensor(_DevArray(rp.value, self.N + 1, "<i4", self), device=dev)
        self.col_idx = torch.as_tensor(_DevArray(ci.value, self.nnz, "<i4", self), device=dev)
        self.slot = torch.as_tensor(_DevArray(sl.value, (self.d + 1) ** 2 * self.NT, "<i4", self), device=dev)

    @property
    def handle(self):
        return self._h

    def destroy(self):
        if self._h and self._h.value:
            lib().fem_pattern_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            if getattr(self, "_owned", True):
                self.destroy()
        except Exception:
            pass


def fem_pattern_set_locality(p: Pattern, node, group=None, stream=None):
    _check(lib().fem_pattern_set_locality(p.handle, _ptr(node), _ptr(group), _stream(stream)))


def fem_pattern_launch_shape(p: Pattern) -> dict:
    v, t, c, pe, ms = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_float()
    _check(lib().fem_pattern_launch_shape(p.handle, C.byref(v), C.byref(t), C.byref(c), C.byref(pe), C.byref(ms)))
    return {"rows_per_block": v.value, "threads": t.value, "ctas_per_sm": c.value, "persistent": bool(pe.value),
            "tuned_ms": ms.value}


def fem_pattern_force_launch(p: Pattern, threads: int, ctas_per_sm: int, persistent: bool):
    _check(lib().fem_pattern_force_launch(p.handle, threads, ctas_per_sm, 1 if persistent else 0))


def fem_pattern_value_path(p: Pattern) -> dict:
    """The deterministic value path: {"path": "tiles"|"tiles_fused"|"blocked"|"two_pass", "tile_elems", "tuned_ms"}."""
    pa, te, ms = C.c_int(), C.c_int(), C.c_float()
    _check(lib().fem_pattern_value_path(p.handle, C.byref(pa), C.byref(te), C.byref(ms)))
    names = {FEM_PATH_TWO_PASS: "two_pass", FEM_PATH_BLOCKED: "blocked", FEM_PATH_TILES: "tiles",
             FEM_PATH_TILES_FUSED: "tiles_fused"}
    return {"path": names[pa.value], "tile_elems": te.value, "tuned_ms": ms.value}


def fem_pattern_force_path(p: Pattern, path: int, tile_elems: int = 256, stream=None):
    _check(lib().fem_pattern_force_path(p.handle, path, tile_elems, _stream(stream)))


def fem_pattern_barrier_fault(p: Pattern, extra_arrivals: int, max_polls: int):
    """Fault injection for the fused launch's bounded grid barrier (see include/femasm.h)."""
    _check(lib().fem_pattern_barrier_fault(p.handle, int(extra_arrivals), int(max_polls)))


def fem_assemble_operator(p: Pattern, node, op: int, coef=None, val=None, stream=None):
    """Values [nnz] of the mass matrix (FEM_OP_MASS, coef c [NT] or None), of -div(K grad) (FEM_OP_ANISO,
    coef [NT, d(d+1)/2] upper triangles) or of the stiffness matrix (FEM_OP_STIFFNESS, coef k [NT])."""
    if val is None:
        val = torch.empty(p.nnz, dtype=torch.float64, device=node.device)
    _check(lib().fem_assemble_operator(p.handle, _ptr(node), op, _ptr(coef), _ptr(val), _stream(stream)))
    return val


def fem_apply_stiffness(p: Pattern, node, k, u, is_bd=None, y=None, stream=None):
    """y = A u, matrix-free (the Dirichlet-eliminated operator when is_bd is given)."""
    if y is None:
        y = torch.empty_like(u)
    _check(lib().fem_apply_stiffness(p.handle, _ptr(node), _ptr(k), _ptr(u), _ptr(is_bd), _ptr(y), _stream(stream)))
    return y


def fem_cg_solve(p: Pattern, node, k, is_bd, b, gD=None, u=None, max_iter=10000, rtol=1e-10, stream=None):
    """Reduced Dirichlet solve by matrix-free conjugate gradients: returns (u [N], iterations, relres)."""
    if u is None:
        u = torch.empty(p.N, dtype=torch.float64, device=node.device)
    it, rr = C.c_int(), C.c_double()
    _check(lib().fem_cg_solve(p.handle, _ptr(node), _ptr(k), _ptr(is_bd), _ptr(b), _ptr(gD), _ptr(u), int(max_iter),
                              float(rtol), C.byref(it), C.byref(rr), _stream(stream)))
    return u, it.value, rr.value


def fem_csr_spmv(p: Pattern, val, x, is_bd=None, y=None, stream=None):
    """y = A x with the pattern's CSR structure and the values val (is_bd: the eliminated operator)."""
    if y is None:
        y = torch.empty_like(x)
    _check(lib().fem_csr_spmv(p.handle, _ptr(val), _ptr(x), _ptr(is_bd), _ptr(y), _stream(stream)))
    return y


def fem_cg_solve_csr(p: Pattern, val, is_bd, b, gD=None, u=None, max_iter=10000, rtol=1e-10, stream=None):
    """Reduced Dirichlet solve by conjugate gradients on the assembled matrix val: (u [N], iterations, relres)."""
    if u is None:
        u = torch.empty(p.N, dtype=torch.float64, device=b.device)
    it, rr = C.c_int(), C.c_double()
    _check(lib().fem_cg_solve_csr(p.handle, _ptr(val), _ptr(is_bd), _ptr(b), _ptr(gD), _ptr(u), int(max_iter),
                                  float(rtol), C.byref(it), C.byref(rr), _stream(stream)))
    return u, it.value, rr.value


def fem_quad_rule(d: int, n: int):
    """(bary [n^d, d+1], w [n^d]) of the library's conical-product Gauss rule (host; no GPU needed)."""
    import numpy as np
    nq = n ** d
    bary = np.zeros((nq, d + 1), np.float64)
    w = np.zeros(nq, np.float64)
    m = C.c_int()
    _check(lib().fem_quad_rule(d, n, bary.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p), C.byref(m)))
    return bary, w


def fem_rule_points(p: Pattern, node, n: int, pts=None, stream=None):
    if pts is None:
        pts = torch.empty((p.NT, n ** p.d, p.d), dtype=torch.float64, device=node.device)
    _check(lib().fem_rule_points(p.handle, _ptr(node), n, _ptr(pts), _stream(stream)))
    return pts


def fem_assemble_rhs_rule(p: Pattern, node, n: int, f_kind=FEM_F_CONST, f_arg=None, b=None, stream=None):
    if b is None:
        b = torch.empty(p.N, dtype=torch.float64, device=node.device)
    _check(lib().fem_assemble_rhs_rule(p.handle, _ptr(node), n, f_kind, _ptr(f_arg), _ptr(b), _stream(stream)))
    return b


def fem_boundary_terms(p: Pattern, node, bdflag, g_side=None, g_const=0.0, alpha=0.0, val=None, b=None, stream=None):
    """Neumann (bdflag 2) and Robin (bdflag 3) side terms added to val and b in place."""
    _check(lib().fem_boundary_terms(p.handle, _ptr(node), _ptr(bdflag), _ptr(g_side), float(g_const), float(alpha),
                                    _ptr(val), _ptr(b), _stream(stream)))


def fem_side_points(p: Pattern, node, pts, stream=None):
    _check(lib().fem_side_points(p.handle, _ptr(node), _ptr(pts), _stream(stream)))


def fem_mean_shift(x, stream=None):
    _check(lib().fem_mean_shift(_ptr(x), x.numel(), _stream(stream)))


def fem_zero_average(p: Pattern, node, u, c_out=None, stream=None):
    _check(lib().fem_zero_average(p.handle, _ptr(node), _ptr(u), _ptr(c_out), _stream(stream)))


def fem_mesh_build_pattern(elem: torch.Tensor, N: int, stream=None) -> Pattern:
    return Pattern(elem, N, stream)


def fem_assemble(p: Pattern, node, k=None, f_kind=FEM_F_CONST, f_arg=None, val=None, b=None,
                 variant=FEM_DETERMINISTIC, stream=None):
    _check(lib().fem_assemble(p.handle, _ptr(node), _ptr(k), f_kind, _ptr(f_arg), _ptr(val), _ptr(b), variant,
                              _stream(stream)))


def fem_assemble_noalloc(p: Pattern, node, k=None, f_kind=FEM_F_CONST, f_arg=None, val=None, b=None, stream=None):
    """Deterministic assembly that allocates nothing (scratch in a fixed device array; see femasm.h)."""
    _check(lib().fem_assemble_noalloc(p.handle, _ptr(node), _ptr(k), f_kind, _ptr(f_arg), _ptr(val), _ptr(b),
                                      _stream(stream)))


def _host_ptrs(ts, steps, what):
    """ctypes array of the data pointers of `steps` contiguous float64 host tensors (None entries: NULL)."""
    if ts is None:
        return None
    if len(ts) != steps:
        raise FemError(FEM_ERR_ARG, "%s: expected %d entries" % (what, steps))
    out = (C.c_void_p * steps)()
    for i, t in enumerate(ts):
        if t is None:
            continue
        if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
            raise FemError(FEM_ERR_ARG, "%s[%d]: expected a contiguous float64 host tensor" % (what, i))
        out[i] = t.data_ptr()
    return out


def fem_assemble_host(p: Pattern, nodes, ks=None, f_kind=FEM_F_CONST, f_arg=None, vals=None, bs=None, stream=None):
    """len(nodes) assemblies from and to host memory, pipelined (see femasm.h): nodes[i] [N, d], ks[i] [NT]
    (None: k = 1) in, vals[i] [nnz] and bs[i] [N] out, all float64 host tensors (page-locked for overlap);
    f_arg a CUDA tensor or None. Returns when every output is written."""
    steps = len(nodes)
    for what, ts, n in (("nodes", nodes, p.N * p.d), ("ks", ks, p.NT), ("vals", vals, p.nnz), ("bs", bs, p.N)):
        for t in (ts or []):
            if t is not None and t.numel() != n:
                raise FemError(FEM_ERR_ARG, "%s: expected %d values per step" % (what, n))
    _check(lib().fem_assemble_host(p.handle, steps, _host_ptrs(nodes, steps, "nodes"), _host_ptrs(ks, steps, "ks"),
                                   f_kind, _ptr(f_arg), _host_ptrs(vals, steps, "vals"), _host_ptrs(bs, steps, "bs"),
                                   _stream(stream)))


def fem_assemble_stiffness(p: Pattern, node, k, val, variant=FEM_DETERMINISTIC, stream=None):
    _check(lib().fem_assemble_stiffness(p.handle, _ptr(node), _ptr(k), _ptr(val), variant, _stream(stream)))


def fem_assemble_rhs(p: Pattern, node, f_kind, f_arg, b, variant=FEM_DETERMINISTIC, stream=None):
    _check(lib().fem_assemble_rhs(p.handle, _ptr(node), f_kind, _ptr(f_arg), _ptr(b), variant, _stream(stream)))


def fem_boundary_nodes(p: Pattern, bdflag, is_bd, stream=None):
    _check(lib().fem_boundary_nodes(p.handle, _ptr(bdflag), _ptr(is_bd), _stream(stream)))


def fem_apply_dirichlet(p: Pattern, is_bd, gD, val, b, free_node=None, want_count=True, stream=None):
    nf = C.c_int64(-1)
    _check(lib().fem_apply_dirichlet(p.handle, _ptr(is_bd), _ptr(gD), _ptr(val), _ptr(b), _ptr(free_node),
                                     C.byref(nf) if want_count else None, _stream(stream)))
    return nf.value if want_count else None


def fem_assemble_backward(p: Pattern, node, k, f_kind, f_arg, w, r, gnode, gk, stream=None):
    _check(lib().fem_assemble_backward(p.handle, _ptr(node), _ptr(k), f_kind, _ptr(f_arg), _ptr(w), _ptr(r),
                                       _ptr(gnode), _ptr(gk), _stream(stream)))


class Batch:
    """Block-diagonal assembly of many meshes (``fem_batch_plan``)."""

    def __init__(self, d: int, Ns, NTs, elem_cat: torch.Tensor, stream=None):
        B = len(Ns)
        self._h = C.c_void_p()
        n_arr = (C.c_int64 * B)(*[int(x) for x in Ns])
        t_arr = (C.c_int64 * B)(*[int(x) for x in NTs])
        _check(lib().fem_batch_plan(d, B, n_arr, t_arr, _ptr(elem_cat), C.byref(self._h), _stream(stream)))
        bb = C.c_int()
        no, eo, zo = C.POINTER(C.c_int64)(), C.POINTER(C.c_int64)(), C.POINTER(C.c_int64)()
        ph = C.c_void_p()
        _check(lib().fem_batch_info(self._h, C.byref(bb), C.byref(no), C.byref(eo), C.byref(zo), C.byref(ph)))
        self.B = bb.value
        self.node_off = [no[i] for i in range(B + 1)]
        self.elem_off = [eo[i] for i in range(B + 1)]
        self.nnz_off = [zo[i] for i in range(B + 1)]
        self.pattern = Pattern(None, 0, _handle=ph)
        self.pattern._owned = False  # owned by the batch

    def set_locality(self, node_cat, stream=None):
        _check(lib().fem_batch_set_locality(self._h, _ptr(node_cat), _stream(stream)))

    def assemble(self, node_cat, k_cat, f_kind, f_arg, val_cat, b_cat, variant=FEM_DETERMINISTIC, graph=False,
                 stream=None):
        f = lib().fem_batch_assemble_graph if graph else lib().fem_batch_assemble
        _check(f(self._h, _ptr(node_cat), _ptr(k_cat), f_kind, _ptr(f_arg), _ptr(val_cat), _ptr(b_cat), variant,
                 _stream(stream)))

    def destroy(self):
        if self._h and self._h.value:
            lib().fem_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def assemble(p: Pattern, node, k=None, f_kind=FEM_F_CONST, f_arg=None, variant=FEM_DETERMINISTIC):
    """Convenience: returns (val [nnz], b [N]) as new CUDA tensors."""
    val = torch.empty(p.nnz, dtype=torch.float64, device=node.device)
    b = torch.empty(p.N, dtype=torch.float64, device=node.device)
    fem_assemble(p, node, k, f_kind, f_arg, val, b, variant)
    return val, b


def assemble_system(node, elem, k=None, f_kind=FEM_F_CONST, f_arg=None, dirichlet=None, gD=None,
                    variant=FEM_DETERMINISTIC, pattern=None, sparse=False):
    """The P1 system of the Poisson problem in one call (CUDA tensors in and out): builds the pattern of
    ``elem`` [NT, d+1] (or reuses ``pattern``) with locality plans from ``node`` [N, d], assembles the
    stiffness matrix and the load vector, and with ``dirichlet`` eliminates the Dirichlet rows:
    True for the whole boundary, or an int8 tensor [NT, d+1] whose 1 entries mark Dirichlet sides; gD
    [N] gives the boundary values (None: 0). Returns (row_ptr, col_idx, val, b), or (A, b) with A a
    torch.sparse_csr_tensor when ``sparse``."""
    if pattern is None:
        pattern = Pattern(elem.to(torch.int32).contiguous(), node.shape[0])
        fem_pattern_set_locality(pattern, node)
    val, b = assemble(pattern, node, k, f_kind, f_arg, variant)
    if dirichlet is not None and dirichlet is not False:
        is_bd = torch.empty(pattern.N, dtype=torch.uint8, device=node.device)
        fem_boundary_nodes(pattern, None if dirichlet is True else dirichlet, is_bd)
        fem_apply_dirichlet(pattern, is_bd, gD, val, b, want_count=False)
    if sparse:
        import warnings
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")  # torch marks its CSR layout as beta
            A = torch.sparse_csr_tensor(pattern.row_ptr.long(), pattern.col_idx.long(), val,
                                        size=(pattern.N, pattern.N))
        return A, b
    return pattern.row_ptr, pattern.col_idx, val, b


class FemAssemble(torch.autograd.Function):
    """(node [N, d], k [NT]) -> (val [nnz], b [N]); backward recomputes the basis gradients."""

    @staticmethod
    def forward(ctx, node, k, p: Pattern, f_kind: int = FEM_F_CONST, f_arg=None):
        node_c, k_c = node.detach().contiguous(), k.detach().contiguous()
        val, b = assemble(p, node_c, k_c, f_kind, f_arg)
        ctx.save_for_backward(node_c, k_c)
        ctx.p, ctx.f_kind, ctx.f_arg = p, f_kind, f_arg
        return val, b

    @staticmethod
    def backward(ctx, gval, gb):
        node, k = ctx.saved_tensors
        gnode = torch.empty_like(node) if ctx.needs_input_grad[0] else None
        gk = torch.empty_like(k) if ctx.needs_input_grad[1] else None
        w = None if gval is None else gval.contiguous()
        r = None if gb is None else gb.contiguous()
        fem_assemble_backward(ctx.p, node, k, ctx.f_kind, ctx.f_arg, w, r, gnode, gk)
        return gnode, gk, None, None, None
