"""ctypes binding of the CPU oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY: the plain FP64 reference the CUDA library is checked against. Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this package.
It shares no code with ``paper_1804_05156_gb300``; both are fed by ``meshgen``.

All functions take and return numpy arrays; indices are 0-based; pattern arrays are int64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ORA_ERRORS = {-1: "bad argument", -2: "index out of range", -3: "degenerate or inverted element",
              -5: "out of memory"}


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C99, -O2, no floating-point contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               "-D_DEFAULT_SOURCE", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        I64, I32 = C.c_int64, C.c_int
        lib.ora_sparse.restype = I64
        lib.ora_sparse.argtypes = [I64, I64, I64, P, P, P, P, P, P, P, P]
        lib.ora_triples.restype = I64
        lib.ora_triples.argtypes = [I32, I64, I64, P, P, P, P, P, P, P, P]
        lib.ora_slots.restype = I32
        lib.ora_slots.argtypes = [I32, I64, I64, P, P, P, P]
        lib.ora_measure.restype = I32
        lib.ora_measure.argtypes = [I32, I64, I64, P, P, P]
        lib.ora_rhs.restype = I32
        lib.ora_rhs.argtypes = [I32, I64, I64, P, P, I32, P, P, P]
        lib.ora_boundary.restype = I32
        lib.ora_boundary.argtypes = [I32, I64, I64, P, P, P]
        lib.ora_dirichlet.restype = I32
        lib.ora_dirichlet.argtypes = [I64, P, P, P, P, P, P, P, P]
        lib.ora_backward.restype = I32
        lib.ora_backward.argtypes = [I32, I64, I64, P, P, P, I32, P, P, P, P, P, P, P, P]
        lib.ora_local_affine.restype = I32
        lib.ora_local_affine.argtypes = [P, P]
        lib.ora_boundary_terms.restype = I32
        lib.ora_boundary_terms.argtypes = [I32, I64, I64, P, P, P, P, C.c_double, C.c_double, P, P, P, P]
        lib.ora_side_points.restype = I32
        lib.ora_side_points.argtypes = [I32, I64, P, P, P]
        lib.ora_mean_shift.restype = I32
        lib.ora_mean_shift.argtypes = [I64, P]
        lib.ora_zero_average.restype = I32
        lib.ora_zero_average.argtypes = [I32, I64, I64, P, P, P, P]
        lib.ora_rhs_rule.restype = I32
        lib.ora_rhs_rule.argtypes = [I32, I64, I64, P, P, I32, P, P, I32, P, P]
        lib.ora_operator_triples.restype = I64
        lib.ora_operator_triples.argtypes = [I32, I64, I64, P, P, I32, P, P, P, P, P]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(rc):
    if rc < 0:
        raise RuntimeError("oracle error %d (%s)" % (rc, ORA_ERRORS.get(int(rc), "?")))
    return rc


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


F_CONST, F_SINPROD, F_QP = 0, 1, 2


def sparse(m, n, I, J, S, S2=None):
    """``sparse(i, j, s, m, n)``: duplicates summed, CSR out (row_ptr, col, val[, val2])."""
    I, J, S, S2 = _c(I, np.int64), _c(J, np.int64), _c(S, np.float64), _c(S2, np.float64)
    nt = I.size
    row_ptr = np.zeros(m + 1, np.int64)
    col = np.zeros(max(nt, 1), np.int64)
    val = np.zeros(max(nt, 1), np.float64)
    val2 = np.zeros(max(nt, 1), np.float64) if S2 is not None else None
    nnz = _check(_load().ora_sparse(m, n, nt, _p(I), _p(J), _p(S), _p(S2), _p(row_ptr), _p(col), _p(val), _p(val2)))
    out = (row_ptr, col[:nnz].copy(), val[:nnz].copy())
    if val2 is not None:
        out = out + (val2[:nnz].copy(),)
    return out


def triples(d, node, elem, k=None, rows=None):
    """COO triples (I, J, S, Sscale) of the stiffness matrix in element order."""
    node, elem, k = _c(node, np.float64), _c(elem, np.int32), _c(k, np.float64)
    N, NT = node.shape[0], elem.shape[0]
    mask = None
    if rows is not None:
        mask = np.zeros(N, np.uint8)
        mask[np.asarray(rows)] = 1
        cnt = int(mask[elem].sum()) * (d + 1)
    else:
        cnt = NT * (d + 1) ** 2
    I = np.zeros(max(cnt, 1), np.int64)
    J = np.zeros(max(cnt, 1), np.int64)
    S = np.zeros(max(cnt, 1), np.float64)
    Ss = np.zeros(max(cnt, 1), np.float64)
    q = _check(_load().ora_triples(d, N, NT, _p(node), _p(elem), _p(k), _p(mask), _p(I), _p(J), _p(S), _p(Ss)))
    return I[:q], J[:q], S[:q], Ss[:q]


def assemble(d, node, elem, k=None, rows=None):
    """Stiffness matrix as CSR: (row_ptr, col, val, scale). With ``rows``, only those rows are filled
    (the others are empty); this is ``sparse`` applied to the triples whose row is selected."""
    N = np.asarray(node).shape[0]
    I, J, S, Ss = triples(d, node, elem, k, rows)
    return sparse(N, N, I, J, S, Ss)


def pattern(d, N, elem):
    """Structural CSR pattern (row_ptr, col) of the P1 matrix: the pairs (elem[t,i], elem[t,j])."""
    elem = _c(elem, np.int32)
    d1 = d + 1
    I = np.repeat(elem, d1, axis=1).ravel()
    J = np.tile(elem, (1, d1)).ravel()
    rp, col, _ = sparse(N, N, I, J, np.zeros(I.size))
    return rp, col


def slots(d, N, elem, row_ptr, col):
    """slot[t, i, j]: CSR position of (elem[t,i], elem[t,j])."""
    elem = _c(elem, np.int32)
    NT = elem.shape[0]
    out = np.zeros((NT, d + 1, d + 1), np.int64)
    _check(_load().ora_slots(d, N, NT, _p(elem), _p(_c(row_ptr, np.int64)), _p(_c(col, np.int64)), _p(out)))
    return out


def measure(d, node, elem):
    """Signed area/volume of each element."""
    node, elem = _c(node, np.float64), _c(elem, np.int32)
    out = np.zeros(elem.shape[0], np.float64)
    _check(_load().ora_measure(d, node.shape[0], elem.shape[0], _p(node), _p(elem), _p(out)))
    return out


def rhs(d, node, elem, fkind=F_CONST, farg=None, rows=None):
    """Load vector b (length N). With ``rows``, only elements touching those rows contribute."""
    node, elem, farg = _c(node, np.float64), _c(elem, np.int32), _c(farg, np.float64)
    N = node.shape[0]
    mask = None
    if rows is not None:
        mask = np.zeros(N, np.uint8)
        mask[np.asarray(rows)] = 1
    b = np.zeros(N, np.float64)
    _check(_load().ora_rhs(d, N, elem.shape[0], _p(node), _p(elem), fkind, _p(farg), _p(mask), _p(b)))
    return b


def boundary(d, N, elem, bdflag=None):
    """Dirichlet node mask (uint8, length N)."""
    elem, bdflag = _c(elem, np.int32), _c(bdflag, np.int8)
    out = np.zeros(N, np.uint8)
    _check(_load().ora_boundary(d, N, elem.shape[0], _p(elem), _p(bdflag), _p(out)))
    return out


def dirichlet(row_ptr, col, val, b, is_bd, gD=None):
    """Returns (val', b', freeNode) of the eliminated system (inputs are not modified)."""
    row_ptr, col = _c(row_ptr, np.int64), _c(col, np.int64)
    val, b = np.array(val, np.float64, copy=True), np.array(b, np.float64, copy=True)
    is_bd, gD = _c(is_bd, np.uint8), _c(gD, np.float64)
    N = row_ptr.size - 1
    fn = np.zeros(max(N, 1), np.int64)
    nf = np.zeros(1, np.int64)
    _check(_load().ora_dirichlet(N, _p(row_ptr), _p(col), _p(is_bd), _p(gD), _p(val), _p(b), _p(fn), _p(nf)))
    return val, b, fn[: int(nf[0])].copy()


def solve_reduced(row_ptr, col, val, b, is_bd, gD=None):
    r"""Sec. 3.3: u = g_D on the boundary, u(freeNode) = A(freeNode, freeNode) \ (b - A u_D)(freeNode), with A
    the assembled CSR matrix (before elimination) and a direct sparse solve (scipy.sparse.linalg.spsolve)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    N = len(row_ptr) - 1
    A = sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col), np.asarray(row_ptr)), shape=(N, N))
    bd = np.asarray(is_bd).astype(bool)
    uD = np.where(bd, 0.0 if gD is None else np.asarray(gD, np.float64), 0.0)
    free = np.nonzero(~bd)[0]
    rhs = np.asarray(b, np.float64) - A @ uD
    u = uD.copy()
    if free.size:
        u[free] = spla.spsolve(A[free][:, free].tocsc(), rhs[free])
    return u


def backward(d, node, elem, k, fkind, farg, slot, w, r, with_scale=False):
    """(gnode [N, d], gk [NT]) of L = w . A + r . b; with_scale=True also returns the per-entry magnitudes
    (gnode_mag, gk_mag): the same sums with every term replaced by its absolute value, the scale the
    parity tolerance of each gradient entry is relative to."""
    node, elem, k = _c(node, np.float64), _c(elem, np.int32), _c(k, np.float64)
    farg, slot, w, r = _c(farg, np.float64), _c(slot, np.int64), _c(w, np.float64), _c(r, np.float64)
    N, NT = node.shape[0], elem.shape[0]
    gn = np.zeros((N, d), np.float64)
    gk = np.zeros(NT, np.float64)
    gnm = np.zeros((N, d), np.float64) if with_scale else None
    gkm = np.zeros(NT, np.float64) if with_scale else None
    _check(_load().ora_backward(d, N, NT, _p(node), _p(elem), _p(k), fkind, _p(farg), _p(slot), _p(w), _p(r),
                                _p(gn), _p(gk), _p(gnm), _p(gkm)))
    return (gn, gk, gnm, gkm) if with_scale else (gn, gk)


def local_affine(p):
    """3x3 local stiffness of one triangle (3x2 vertex array) by the reference-element map."""
    p = _c(p, np.float64)
    At = np.zeros((3, 3), np.float64)
    _check(_load().ora_local_affine(_p(p), _p(At)))
    return At


def boundary_terms(d, node, elem, bdflag, row_ptr, col, val, b, g_side=None, g_const=0.0, alpha=0.0):
    """(val', b') after the Neumann (bdflag 2) and Robin (bdflag 3) side terms (inputs not modified)."""
    node, elem, bdflag = _c(node, np.float64), _c(elem, np.int32), _c(bdflag, np.int8)
    row_ptr, col, g_side = _c(row_ptr, np.int64), _c(col, np.int64), _c(g_side, np.float64)
    val, b = np.array(val, np.float64, copy=True), np.array(b, np.float64, copy=True)
    _check(_load().ora_boundary_terms(d, node.shape[0], elem.shape[0], _p(node), _p(elem), _p(bdflag), _p(g_side),
                                      float(g_const), float(alpha), _p(row_ptr), _p(col), _p(val), _p(b)))
    return val, b


def side_points(d, node, elem):
    """Quadrature point of every side (midpoint 2-D, centroid 3-D): [NT, d+1, d]."""
    node, elem = _c(node, np.float64), _c(elem, np.int32)
    out = np.zeros((elem.shape[0], d + 1, d), np.float64)
    _check(_load().ora_side_points(d, elem.shape[0], _p(node), _p(elem), _p(out)))
    return out


def mean_shift(b):
    """b - mean(b)."""
    out = np.array(b, np.float64, copy=True)
    _check(_load().ora_mean_shift(out.size, _p(out)))
    return out


def zero_average(d, node, elem, u):
    """(u - c, c) with c the area-weighted mean of the P1 function u."""
    node, elem = _c(node, np.float64), _c(elem, np.int32)
    out = np.array(u, np.float64, copy=True)
    c = np.zeros(1, np.float64)
    _check(_load().ora_zero_average(d, node.shape[0], elem.shape[0], _p(node), _p(elem), _p(out), _p(c)))
    return out, float(c[0])


OP_MASS, OP_ANISO = 1, 2


def operator(d, node, elem, op, coef=None):
    """CSR (row_ptr, col, val, scale) of the mass matrix (op 1, coefficient per element) or of the
    anisotropic operator (op 2, symmetric tensor per element, upper triangle)."""
    node, elem, coef = _c(node, np.float64), _c(elem, np.int32), _c(coef, np.float64)
    N, NT = node.shape[0], elem.shape[0]
    cnt = max(NT * (d + 1) ** 2, 1)
    I, J = np.zeros(cnt, np.int64), np.zeros(cnt, np.int64)
    S, Ss = np.zeros(cnt, np.float64), np.zeros(cnt, np.float64)
    q = _check(_load().ora_operator_triples(d, N, NT, _p(node), _p(elem), op, _p(coef), _p(I), _p(J), _p(S), _p(Ss)))
    return sparse(N, N, I[:q], J[:q], S[:q], Ss[:q])


def _gauss_jacobi01(n, a):
    """Gauss rule on [0, 1] for the weight (1 - v)^a, by the eigenvalues of the Jacobi matrix of the
    orthogonal polynomials (Golub-Welsch); weights sum to 1 / (a + 1)."""
    # monic recurrence of the Jacobi polynomials P_k^{(a, 0)} on [-1, 1]
    k = np.arange(n, dtype=np.float64)
    al = np.where(2 * k + a == 0, 0.0, -(a * a) / np.maximum((2 * k + a) * (2 * k + a + 2), 1e-300))
    if n > 0 and a == 0:
        al[:] = 0.0
    kk = np.arange(1, n, dtype=np.float64)
    be = 4 * kk * (kk + a) * kk * (kk + a) / ((2 * kk + a) ** 2 * (2 * kk + a + 1) * (2 * kk + a - 1))
    J = np.diag(al) + np.diag(np.sqrt(be), 1) + np.diag(np.sqrt(be), -1)
    t, vec = np.linalg.eigh(J)
    mu0 = 2.0 ** (a + 1) / (a + 1)
    w = mu0 * vec[0, :] ** 2
    return 0.5 * (1.0 + t), w * 0.5 ** (a + 1)


def quad_rule(d, n):
    """Conical-product Gauss rule on the reference simplex: (bary [n^d, d+1], weights [n^d]) summing to 1,
    exact for total degree 2n - 1."""
    xu, wu = _gauss_jacobi01(n, 0)
    xv, wv = _gauss_jacobi01(n, 1)
    pts, ws = [], []
    if d == 2:
        for a in range(n):
            for b in range(n):
                x, y = xu[a] * (1 - xv[b]), xv[b]
                pts.append([1 - x - y, x, y])
                ws.append(2 * wu[a] * wv[b])
    else:
        xw, ww = _gauss_jacobi01(n, 2)
        for a in range(n):
            for b in range(n):
                for c in range(n):
                    x, y, z = xu[a] * (1 - xv[b]) * (1 - xw[c]), xv[b] * (1 - xw[c]), xw[c]
                    pts.append([1 - x - y - z, x, y, z])
                    ws.append(6 * wu[a] * wv[b] * ww[c])
    return np.array(pts), np.array(ws)


def rhs_rule(d, node, elem, bary, w, fkind=F_CONST, farg=None):
    """Load vector with a given rule: b_i = sum_tau |tau| sum_q w_q f(p_q) lambda_i(p_q)."""
    node, elem = _c(node, np.float64), _c(elem, np.int32)
    bary, w, farg = _c(bary, np.float64), _c(w, np.float64), _c(farg, np.float64)
    N = node.shape[0]
    b = np.zeros(N, np.float64)
    _check(_load().ora_rhs_rule(d, N, elem.shape[0], _p(node), _p(elem), w.size, _p(bary), _p(w), fkind, _p(farg),
                                _p(b)))
    return b
