"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test pins one oracle function to something other than itself: the paper's worked example,
closed forms, an independent formula, brute force on tiny meshes, or an invariant.
"""
import json
import math
import os

import numpy as np
import pytest

import meshgen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_from_csr(rp, col, val, n):
    A = np.zeros((rp.size - 1, n))
    for r in range(rp.size - 1):
        A[r, col[rp[r]:rp[r + 1]]] = val[rp[r]:rp[r + 1]]
    return A


def brute_local(p, k=1.0):
    """Local stiffness by inverting [x_i 1]: column i of the inverse holds lambda_i's coefficients."""
    d = p.shape[1]
    M = np.hstack([p, np.ones((d + 1, 1))])
    Minv = np.linalg.inv(M)
    G = Minv[:d, :].T  # rows: grad lambda_i
    vol = abs(np.linalg.det(M)) / math.factorial(d)
    return k * vol * G @ G.T, G, vol


def random_simplex(rng, d):
    while True:
        p = rng.uniform(-1, 1, size=(d + 1, d))
        det = np.linalg.det(p[1:] - p[0])  # d! times the signed measure
        if abs(det) > 0.05:
            if det < 0:  # positive orientation (Sec. 1.1): swap two vertices
                p[[0, 1]] = p[[1, 0]]
            return p


# --- Sec. 2.1 / 2.2: sparse -----------------------------------------------------------------------

def test_sparse_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "sparse_worked_example.json")))
    I = np.array(g["i_1based"]) - 1
    J = np.array(g["j_1based"]) - 1
    rp, col, val = oracle.sparse(g["m"], g["n"], I, J, np.array(g["s"], float))
    assert rp.tolist() == g["csr_row_ptr_0based"]
    assert col.tolist() == g["csr_col_0based"]
    assert val.tolist() == g["csr_val"]
    A = dense_from_csr(rp, col, val, g["n"])
    assert A.tolist() == g["dense"]
    # CSC of the same matrix = CSR of its transpose: the column pointer printed in the paper
    rpt, _, _ = oracle.sparse(g["n"], g["m"], J, I, np.array(g["s"], float))
    assert (rpt + 1).tolist() == g["csc_colptr_1based"]


def test_sparse_sums_duplicates_in_given_order():
    I = np.array([2, 0, 2, 2, 1])
    J = np.array([1, 0, 1, 1, 2])
    S = np.array([1e16, 3.0, 1.0, -1e16, 5.0])
    rp, col, val = oracle.sparse(3, 3, I, J, S)
    assert rp.tolist() == [0, 1, 2, 3]
    assert col.tolist() == [0, 2, 1]
    # ((1e16 + 1) - 1e16) in the given order is 0 in double; any reordering that adds 1 last gives 1
    assert val.tolist() == [3.0, 5.0, (1e16 + 1.0) - 1e16]


def test_sparse_keeps_exact_zero_sums():
    rp, col, val = oracle.sparse(2, 2, np.array([0, 0, 1]), np.array([1, 1, 1]), np.array([2.0, -2.0, 1.0]))
    assert col.tolist() == [1, 1] and val.tolist() == [0.0, 1.0]


# --- Sec. 3.1: local stiffness by three independent formulas --------------------------------------

@pytest.mark.parametrize("d", [2, 3])
def test_local_stiffness_three_formulas(d):
    rng = np.random.default_rng(7 + d)
    for _ in range(200):
        p = random_simplex(rng, d)
        k = float(np.exp(rng.normal()))
        elem = np.arange(d + 1, dtype=np.int32)[None, :]
        rp, col, val, scale = oracle.assemble(d, p, elem, np.array([k]))
        A = dense_from_csr(rp, col, val, d + 1)
        B, _, _ = brute_local(p, k)
        assert np.all(np.abs(A - B) <= 1e-13 * dense_from_csr(rp, col, scale, d + 1) + 1e-300)
        if d == 2:
            Aff = oracle.local_affine(p) * k
            assert np.allclose(A, Aff, rtol=0, atol=1e-13 * np.abs(B).max())


def test_local_affine_reference_triangle():
    # reference triangle (1,0), (0,1), (0,0): At = 1/2 * [[1,0,-1],[0,1,-1],[-1,-1,2]]
    At = oracle.local_affine(np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]]))
    assert At.tolist() == [[0.5, 0.0, -0.5], [0.0, 0.5, -0.5], [-0.5, -0.5, 1.0]]


@pytest.mark.parametrize("d,n", [(2, 3), (3, 2)])
def test_dense_elementwise_assembly(d, n):
    """Sec. 3.1.1 element loop into a dense matrix, with brute-force local matrices."""
    mesh = meshgen.square_mesh(n, 0.2, 11) if d == 2 else meshgen.kuhn_mesh(n, 0.1, 11)
    node, elem = mesh["node"], mesh["elem"]
    k = meshgen.lognormal(5, 3, elem.shape[0])
    N = node.shape[0]
    D = np.zeros((N, N))
    for t, e in enumerate(elem):
        At, _, _ = brute_local(node[e], k[t])
        D[np.ix_(e, e)] += At
    rp, col, val, scale = oracle.assemble(d, node, elem, k)
    A = dense_from_csr(rp, col, val, N)
    S = dense_from_csr(rp, col, scale, N)
    assert np.all(np.abs(A - D) <= 1e-13 * S + 1e-300)
    # pattern: structural pairs; the dense nonzero set lies inside it
    P = dense_from_csr(rp, col, np.ones_like(val), N) > 0
    assert not np.any((np.abs(D) > 1e-14) & ~P)
    # the pattern is exactly the set of vertex pairs sharing an element
    Q = np.zeros((N, N), bool)
    for e in elem:
        Q[np.ix_(e, e)] = True
    assert np.array_equal(P, Q)


# --- closed forms on uniform meshes ---------------------------------------------------------------

def test_five_point_stencil_exact():
    m = meshgen.make_config("c1")
    n = m["n"]
    rp, col, val, _ = oracle.assemble(2, m["node"], m["elem"])
    assert rp[-1] == 29057
    for j in range(1, n):
        for i in range(1, n):
            r = j * (n + 1) + i
            c = col[rp[r]:rp[r + 1]] - r
            v = val[rp[r]:rp[r + 1]]
            assert c.tolist() == [-(n + 2), -(n + 1), -1, 0, 1, n + 1, n + 2]
            assert v.tolist() == [0.0, -1.0, -1.0, 4.0, -1.0, -1.0, 0.0]


def test_kuhn_stencil():
    n = 4
    m = meshgen.kuhn_mesh(n)
    h = 1.0 / n
    rp, col, val, scale = oracle.assemble(3, m["node"], m["elem"])
    n1 = n + 1
    for c3 in range(1, n):
        for b3 in range(1, n):
            for a3 in range(1, n):
                r = a3 + n1 * (b3 + n1 * c3)
                cols = col[rp[r]:rp[r + 1]] - r
                v = val[rp[r]:rp[r + 1]]
                assert cols.size == 15
                exp = {0: 6 * h, 1: -h, -1: -h, n1: -h, -n1: -h, n1 * n1: -h, -n1 * n1: -h}
                for cc, vv in zip(cols.tolist(), v.tolist()):
                    assert abs(vv - exp.get(cc, 0.0)) <= 1e-15
    # 24 incident tetrahedra per interior vertex
    cnt = np.bincount(m["elem"].ravel(), minlength=n1 ** 3)
    assert cnt[1 + n1 * (1 + n1 * 1)] == 24


@pytest.mark.parametrize("d,n", [(2, 1), (2, 2), (2, 5), (2, 16), (3, 1), (3, 2), (3, 3), (3, 6)])
def test_nnz_closed_form(d, n):
    m = meshgen.square_mesh(n) if d == 2 else meshgen.kuhn_mesh(n)
    N = m["node"].shape[0]
    rp, col = oracle.pattern(d, N, m["elem"])
    if d == 2:
        exp = N + 2 * (3 * n * n + 2 * n)
    else:
        exp = N + 2 * (3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3)
    assert rp[-1] == exp


# --- invariants -------------------------------------------------------------------------------------

@pytest.mark.parametrize("d", [2, 3])
def test_symmetry_rowsum_measure(d):
    m = meshgen.square_mesh(12, 0.2, 3) if d == 2 else meshgen.kuhn_mesh(5, 0.1, 3)
    node, elem = m["node"], m["elem"]
    k = meshgen.lognormal(4, 3, elem.shape[0])
    N = node.shape[0]
    rp, col, val, scale = oracle.assemble(d, node, elem, k)
    A = dense_from_csr(rp, col, val, N)
    S = dense_from_csr(rp, col, scale, N)
    assert np.all(np.abs(A - A.T) <= 1e-14 * S)
    assert np.all(np.abs(A.sum(axis=1)) <= 1e-13 * S.sum(axis=1))
    meas = oracle.measure(d, node, elem)
    assert np.all(meas > 0)
    assert abs(meas.sum() - 1.0) <= 1e-13
    # positive semidefinite with the constants as kernel (Sec. 3.3, pure Neumann): rank N-1
    w = np.linalg.eigvalsh(A)
    assert w[0] > -1e-12 * w[-1] and w[1] > 1e-10 * w[-1]


@pytest.mark.parametrize("d", [2, 3])
def test_linear_annihilation(d):
    """Interior rows of A kill linear functions when the coefficient is constant."""
    m = meshgen.square_mesh(10, 0.2, 5) if d == 2 else meshgen.kuhn_mesh(4, 0.1, 5)
    node, elem, isbd = m["node"], m["elem"], m["is_bd"]
    rp, col, val, _ = oracle.assemble(d, node, elem)
    N = node.shape[0]
    A = dense_from_csr(rp, col, val, N)
    g = np.array([0.3, -1.7, 0.9][:d])
    ell = 2.0 + node @ g
    res = A @ ell
    mag = np.abs(A) @ np.abs(ell)
    assert np.all(np.abs(res[isbd == 0]) <= 1e-13 * mag[isbd == 0])
    # and not for a boundary row in general
    assert np.max(np.abs(res[isbd == 1])) > 1e-6


def test_variable_k_does_not_annihilate():
    m = meshgen.square_mesh(6, 0.2, 5)
    k = meshgen.lognormal(1, 3, m["elem"].shape[0])
    rp, col, val, _ = oracle.assemble(2, m["node"], m["elem"], k)
    A = dense_from_csr(rp, col, val, m["node"].shape[0])
    res = A @ (m["node"] @ np.array([1.0, 0.0]))
    assert np.max(np.abs(res[m["is_bd"] == 0])) > 1e-3


@pytest.mark.parametrize("d", [2, 3])
def test_mesh_relabelling_invariance(d):
    """Sec. 1.1: any row permutation of elem and any even vertex permutation is the same mesh."""
    m = meshgen.square_mesh(7, 0.2, 9) if d == 2 else meshgen.kuhn_mesh(3, 0.1, 9)
    node, elem = m["node"], m["elem"]
    k = meshgen.lognormal(2, 3, elem.shape[0])
    rng = np.random.default_rng(0)
    perm = rng.permutation(elem.shape[0])
    even = [[0, 1, 2], [1, 2, 0], [2, 0, 1]] if d == 2 else [[0, 1, 2, 3], [1, 2, 0, 3], [0, 2, 3, 1], [1, 0, 3, 2]]
    e2 = np.stack([elem[perm[t]][even[t % len(even)]] for t in range(elem.shape[0])])
    rp1, c1, v1, s1 = oracle.assemble(d, node, elem, k)
    rp2, c2, v2, _ = oracle.assemble(d, node, e2, k[perm])
    assert np.array_equal(rp1, rp2) and np.array_equal(c1, c2)
    assert np.all(np.abs(v1 - v2) <= 1e-13 * s1)


def test_orientation_is_enforced():
    m = meshgen.square_mesh(3)
    e = m["elem"].copy()
    e[4] = e[4][[1, 0, 2]]
    with pytest.raises(RuntimeError):  # 2-D takes abs() of the area, so only zero area is rejected
        oracle.assemble(2, np.zeros_like(m["node"]), e)
    k3 = meshgen.kuhn_mesh(2)
    e3 = k3["elem"].copy()
    e3[5] = e3[5][[1, 0, 2, 3]]
    with pytest.raises(RuntimeError):  # 3-D uses the signed volume
        oracle.assemble(3, k3["node"], e3)
    with pytest.raises(RuntimeError):
        oracle.assemble(2, m["node"], np.array([[0, 1, 99]], np.int32))


# --- Sec. 3.2 and Sec. 4: load vector --------------------------------------------------------------

def quad_points_by_rule(d, p):
    """Points of the rule (2-D: edge midpoints, point q opposite vertex q; 3-D: (a,b,b,b) rule)."""
    if d == 2:
        return np.stack([(p[(q + 1) % 3] + p[(q + 2) % 3]) / 2 for q in range(3)])
    s5 = math.sqrt(5.0)
    a, b = (5 + 3 * s5) / 20, (5 - s5) / 20
    L = np.full((4, 4), b) + np.eye(4) * (a - b)
    return L @ p


@pytest.mark.parametrize("d", [2, 3])
def test_rhs_f1_closed_form(d):
    m = meshgen.square_mesh(9, 0.2, 1) if d == 2 else meshgen.kuhn_mesh(4, 0.1, 1)
    node, elem = m["node"], m["elem"]
    b = oracle.rhs(d, node, elem)
    meas = np.array([brute_local(node[e])[2] for e in elem])
    exp = np.zeros(node.shape[0])
    np.add.at(exp, elem.ravel(), np.repeat(meas / (d + 1), d + 1))
    assert np.allclose(b, exp, rtol=1e-13, atol=0)
    assert abs(b.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("d", [2, 3])
def test_rhs_linear_f_closed_form(d):
    """int_tau f lambda_i = |tau|/((d+1)(d+2)) (sum_m f(x_m) + f(x_i)) for linear f."""
    m = meshgen.square_mesh(6, 0.2, 2) if d == 2 else meshgen.kuhn_mesh(3, 0.1, 2)
    node, elem = m["node"], m["elem"]
    g, c = np.array([0.7, -0.4, 1.1][:d]), 0.35
    fq = np.stack([quad_points_by_rule(d, node[e]) @ g + c for e in elem])
    b = oracle.rhs(d, node, elem, oracle.F_QP, fq.ravel())
    exp = np.zeros(node.shape[0])
    for e in elem:
        vol = brute_local(node[e])[2]
        fv = node[e] @ g + c
        exp[e] += vol / ((d + 1) * (d + 2)) * (fv.sum() + fv)
    assert np.allclose(b, exp, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("d", [2, 3])
def test_rule_exact_for_quadratics(d):
    """Sec. 4: sum_i b_i = int_tau f exactly for quadratic f = (g.x + c)^2, by the barycentric formula
    int lambda_i lambda_j = d! |tau| (1 + delta_ij) / (d+2)!."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        p = random_simplex(rng, d)
        g, c = rng.normal(size=d), rng.normal()
        a = p @ g + c
        vol = brute_local(p)[2]
        exact = math.factorial(d) * vol / math.factorial(d + 2) * (a.sum() ** 2 + (a ** 2).sum())
        fq = (quad_points_by_rule(d, p) @ g + c) ** 2
        b = oracle.rhs(d, p, np.arange(d + 1, dtype=np.int32)[None, :], oracle.F_QP, fq)
        assert abs(b.sum() - exact) <= 1e-13 * max(1.0, abs(exact))
    # a first-order rule would fail: the centroid value times |tau| misses the quadratic part
    assert abs(vol * ((p.mean(axis=0) @ g + c) ** 2) - exact) > 1e-6


@pytest.mark.parametrize("d", [2, 3])
def test_rhs_sinprod_matches_point_values(d):
    m = meshgen.square_mesh(5, 0.2, 8) if d == 2 else meshgen.kuhn_mesh(3, 0.1, 8)
    node, elem = m["node"], m["elem"]
    fq = np.stack([np.prod(np.sin(np.pi * quad_points_by_rule(d, node[e])), axis=1) for e in elem])
    b1 = oracle.rhs(d, node, elem, oracle.F_SINPROD)
    b2 = oracle.rhs(d, node, elem, oracle.F_QP, fq.ravel())
    assert np.allclose(b1, b2, rtol=1e-13, atol=1e-18)


def test_sinpi_special_values():
    # f = sin(pi x) sin(pi y) at (1/2, 1/6) is 1 * 1/2; at integers it is exactly 0
    node = np.array([[0.5, 1.0 / 6.0], [0.5, 1.0 / 6.0], [0.5, 1.0 / 6.0]])
    # a degenerate "element" is rejected, so probe f through a real one whose midpoints are known
    p = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    fq = np.stack([np.prod(np.sin(np.pi * quad_points_by_rule(2, p)), axis=1)])
    b = oracle.rhs(2, p, np.array([[0, 1, 2]], np.int32), oracle.F_SINPROD)
    # midpoints (0.5,0.5), (0,0.5), (0.5,0): f = 1, 0, 0 exactly
    assert fq[0, 0] == 1.0
    assert b.tolist() == [0.5 * (0.0 + 0.0) / 6, 0.5 * (0.0 + 1.0) / 6, 0.5 * (1.0 + 0.0) / 6]
    del node


# --- Sec. 1.2 and 3.3: boundary and Dirichlet ------------------------------------------------------

@pytest.mark.parametrize("d", [2, 3])
def test_boundary_whole_and_bdflag(d):
    m = meshgen.square_mesh(7, 0.2, 4, permute=True) if d == 2 else meshgen.kuhn_mesh(3, 0.1, 4)
    N = m["node"].shape[0]
    assert np.array_equal(oracle.boundary(d, N, m["elem"]), m["is_bd"])
    assert np.array_equal(oracle.boundary(d, N, m["elem"], m["bdflag"]), m["is_bd"])
    # a partial flag marks only that side's vertices
    bf = np.zeros_like(m["bdflag"])
    t, i = np.argwhere(m["bdflag"] == 1)[0]
    bf[t, i] = 1
    mask = oracle.boundary(d, N, m["elem"], bf)
    assert mask.sum() == d


@pytest.mark.parametrize("d", [2, 3])
def test_dirichlet_reproduces_linear_solution(d):
    """Sec. 3.3: with f = 0, k = 1 and linear g_D, the reduced solve returns the linear function."""
    m = meshgen.square_mesh(8, 0.2, 6) if d == 2 else meshgen.kuhn_mesh(4, 0.1, 6)
    node, elem = m["node"], m["elem"]
    N = node.shape[0]
    rp, col, val, _ = oracle.assemble(d, node, elem)
    b = oracle.rhs(d, node, elem, oracle.F_CONST, np.array([0.0]))
    isbd = oracle.boundary(d, N, elem)
    gD = 0.5 - 1.3 * node[:, 0] + 0.8 * node[:, 1]
    val2, b2, free = oracle.dirichlet(rp, col, val, b, isbd, gD)
    assert np.array_equal(free, np.flatnonzero(isbd == 0))
    A = dense_from_csr(rp, col, val, N)
    u_free = np.linalg.solve(A[np.ix_(free, free)], b2[free])
    assert np.allclose(u_free, gD[free], rtol=0, atol=1e-12)
    # the eliminated square system gives the same solution everywhere
    A2 = dense_from_csr(rp, col, val2, N)
    assert np.allclose(np.linalg.solve(A2, b2), gD, rtol=0, atol=1e-12)
    assert np.array_equal(A2, A2.T)
    bd = np.flatnonzero(isbd)
    assert np.array_equal(A2[bd], np.eye(N)[bd])
    assert np.array_equal(b2[bd], gD[bd])


def test_dirichlet_lift_is_b_minus_Au():
    m = meshgen.square_mesh(5, 0.2, 2)
    node, elem = m["node"], m["elem"]
    N = node.shape[0]
    k = meshgen.lognormal(3, 3, elem.shape[0])
    rp, col, val, _ = oracle.assemble(2, node, elem, k)
    b = oracle.rhs(2, node, elem, oracle.F_SINPROD)
    isbd = m["is_bd"]
    gD = np.cos(node[:, 0] * 3) + node[:, 1]
    _, b2, _ = oracle.dirichlet(rp, col, val, b, isbd, gD)
    u = np.where(isbd == 1, gD, 0.0)
    exp = b - dense_from_csr(rp, col, val, N) @ u
    free = isbd == 0
    assert np.allclose(b2[free], exp[free], rtol=1e-14, atol=1e-15)


# --- backward: closed-form adjoint vs finite differences and invariants ----------------------------

def loss(d, node, elem, k, rp, col, fkind, w, r):
    I, J, S, _ = oracle.triples(d, node, elem, k)
    rp2, col2, val = oracle.sparse(node.shape[0], node.shape[0], I, J, S)
    assert np.array_equal(rp2, rp) and np.array_equal(col2, col)
    b = oracle.rhs(d, node, elem, fkind)
    return float(w @ val + r @ b)


@pytest.mark.parametrize("part", ["both", "r_only"])
@pytest.mark.parametrize("d", [2, 3])
def test_backward_central_fd(d, part):
    """The adjoint against central differences of the assembled loss; r_only (w = 0) checks the
    load-vector part on its own scale."""
    m = meshgen.square_mesh(3, 0.2, 12) if d == 2 else meshgen.kuhn_mesh(2, 0.1, 12)
    node, elem = m["node"], m["elem"]
    N, NT = node.shape[0], elem.shape[0]
    k = meshgen.lognormal(12, 3, NT)
    rp, col = oracle.pattern(d, N, elem)
    slot = oracle.slots(d, N, elem, rp, col)
    w = meshgen.normal(13, 4, rp[-1]) if part == "both" else np.zeros(rp[-1])
    r = meshgen.normal(13, 5, N)
    gn, gk = oracle.backward(d, node, elem, k, oracle.F_SINPROD, None, slot, w, r)
    eps = 1e-6
    for v in range(N):
        for c in range(d):
            xp, xm = node.copy(), node.copy()
            xp[v, c] += eps
            xm[v, c] -= eps
            fd = (loss(d, xp, elem, k, rp, col, oracle.F_SINPROD, w, r)
                  - loss(d, xm, elem, k, rp, col, oracle.F_SINPROD, w, r)) / (2 * eps)
            tol = 1e-6 * max(1.0, abs(gn[v, c])) if part == "both" else 1e-8 * max(1e-2, abs(gn[v, c]))
            assert abs(fd - gn[v, c]) <= tol, (v, c, fd, gn[v, c])
    for t in range(NT):
        kp, km = k.copy(), k.copy()
        kp[t] += eps
        km[t] -= eps
        fd = (loss(d, node, elem, kp, rp, col, oracle.F_SINPROD, w, r)
              - loss(d, node, elem, km, rp, col, oracle.F_SINPROD, w, r)) / (2 * eps)
        assert abs(fd - gk[t]) <= 1e-6 * max(1.0, abs(gk[t]))


@pytest.mark.parametrize("d", [2, 3])
def test_backward_invariants(d):
    """Stiffness part only (r = 0): translation invariance, homogeneity of degree d-2, and
    k dL/dk = L element by element (a^tau is linear in k)."""
    m = meshgen.square_mesh(6, 0.2, 14) if d == 2 else meshgen.kuhn_mesh(3, 0.1, 14)
    node, elem = m["node"], m["elem"]
    N, NT = node.shape[0], elem.shape[0]
    k = meshgen.lognormal(14, 3, NT)
    rp, col = oracle.pattern(d, N, elem)
    slot = oracle.slots(d, N, elem, rp, col)
    w = meshgen.normal(15, 4, rp[-1])
    gn, gk = oracle.backward(d, node, elem, k, oracle.F_CONST, None, slot, w, np.zeros(N))
    I, J, S, _ = oracle.triples(d, node, elem, k)
    _, _, val = oracle.sparse(N, N, I, J, S)
    L = float(w @ val)
    scale = float(np.abs(gn).sum() + abs(L))
    assert np.all(np.abs(gn.sum(axis=0)) <= 1e-12 * scale)
    homog = float((node * gn).sum())
    assert abs(homog - (d - 2) * L) <= 1e-12 * scale
    assert abs(float(k @ gk) - L) <= 1e-12 * (abs(L) + float(np.abs(k * gk).sum()))


@pytest.mark.parametrize("d", [2, 3])
def test_backward_magnitudes(d):
    """The per-entry magnitudes the gradient tolerance is relative to: never below the gradient itself,
    and equal to it where every term is nonnegative (2-D, w = 1 on the diagonal slots only, r = 0:
    dL/dk_t = |tau| sum_i |grad lambda_i|^2, a sum of squares)."""
    m = meshgen.square_mesh(5, 0.2, 16) if d == 2 else meshgen.kuhn_mesh(3, 0.1, 16)
    node, elem = m["node"], m["elem"]
    N, NT = node.shape[0], elem.shape[0]
    k = meshgen.lognormal(16, 3, NT)
    rp, col = oracle.pattern(d, N, elem)
    slot = oracle.slots(d, N, elem, rp, col)
    w, r = meshgen.normal(17, 4, rp[-1]), meshgen.normal(17, 5, N)
    gn, gk, gnm, gkm = oracle.backward(d, node, elem, k, oracle.F_SINPROD, None, slot, w, r, with_scale=True)
    assert np.all(gnm >= np.abs(gn)) and np.all(gkm >= np.abs(gk))
    assert np.all(gnm > 0) and np.all(gkm > 0)
    if d == 2:
        wd = np.zeros(rp[-1])
        for row in range(N):
            wd[rp[row] + np.searchsorted(col[rp[row]:rp[row + 1]], row)] = 1.0
        _, gk1, _, gkm1 = oracle.backward(d, node, elem, k, oracle.F_CONST, None, slot, wd, None, with_scale=True)
        assert np.all(gk1 > 0)
        assert np.allclose(gkm1, gk1, rtol=1e-14, atol=0)


# --- Neumann / Robin sides and the pure-Neumann fixes (Sec. 3.3 and "Boundary conditions") --------

def _geometry(d, n, jitter, seed):
    return meshgen.square_mesh(n, jitter, seed) if d == 2 else meshgen.kuhn_mesh(n, jitter, seed)


@pytest.mark.parametrize("d", [2, 3])
def test_neumann_constant_g_integrates_the_side_measure(d):
    """Constant g: the side rule is exact, so the Neumann load sums to g |Gamma_N| and each vertex gets
    g times a d-th of its incident Neumann sides' measure."""
    m = _geometry(d, 5, 0.2, 31)
    node, elem = m["node"], m["elem"]
    N = node.shape[0]
    flags = meshgen.side_flags(m, {"x0": 2, "x1": 2})  # two opposite faces of measure 1 each
    rp, col = oracle.pattern(d, N, elem)
    z = np.zeros(rp[-1])
    _, b = oracle.boundary_terms(d, node, elem, flags, rp, col, z, np.zeros(N), g_const=2.5)
    assert abs(b.sum() - 2.5 * 2.0) <= 1e-14
    # only vertices on the two faces receive load; on x = 0 (2-D) each vertex gets g times half the
    # lengths of its two boundary edges
    x0 = np.isclose(node[:, 0], 0.0)
    assert np.all(b[~(x0 | np.isclose(node[:, 0], 1.0))] == 0.0)
    if d == 2:
        ys = np.sort(node[x0, 1])
        h = np.diff(ys)
        exp = np.zeros(ys.size)
        exp[:-1] += h / 2
        exp[1:] += h / 2
        order = np.argsort(node[x0, 1])
        assert np.allclose(b[x0][order], 2.5 * exp, rtol=1e-14, atol=0)


@pytest.mark.parametrize("d", [2, 3])
def test_robin_side_mass_matrix(d):
    """The Robin matrix is alpha times the side mass matrix: u^T M u = alpha int u^2 over Gamma_R, exact for
    linear u (u = 1 gives alpha |Gamma_R|; u = x on the face y = 1 (2-D) or z = 1 (3-D) gives alpha/3)."""
    m = _geometry(d, 4, 0.2, 32)
    node, elem = m["node"], m["elem"]
    N = node.shape[0]
    face = "y1" if d == 2 else "z1"
    flags = meshgen.side_flags(m, {face: 3})
    rp, col = oracle.pattern(d, N, elem)
    val, _ = oracle.boundary_terms(d, node, elem, flags, rp, col, np.zeros(rp[-1]), np.zeros(N), alpha=1.7)
    M = dense_from_csr(rp, col, val, N)
    assert np.array_equal(M, M.T)
    one = np.ones(N)
    assert abs(one @ M @ one - 1.7) <= 1e-14
    x = node[:, 0]
    assert abs(x @ M @ x - 1.7 / 3.0) <= 1e-14
    # Robin sides add no load when g = 0, and the load matches the Neumann rule when g != 0
    _, b = oracle.boundary_terms(d, node, elem, flags, rp, col, np.zeros(rp[-1]), np.zeros(N), g_const=1.0, alpha=1.7)
    assert abs(b.sum() - 1.0) <= 1e-14


def test_side_points_are_midpoints_and_centroids():
    m = meshgen.square_mesh(3, 0.2, 33)
    p = oracle.side_points(2, m["node"], m["elem"])
    e = m["elem"]
    for t in range(e.shape[0]):
        for j in range(3):
            a, b = [e[t, k] for k in range(3) if k != j]
            assert np.array_equal(p[t, j], (m["node"][a] + m["node"][b]) / 2)
    m3 = meshgen.kuhn_mesh(2, 0.1, 33)
    p3 = oracle.side_points(3, m3["node"], m3["elem"])
    e3 = m3["elem"]
    assert np.allclose(p3[:, 0], m3["node"][e3[:, 1:]].mean(axis=1), rtol=1e-15, atol=1e-16)


@pytest.mark.parametrize("d", [2, 3])
def test_pure_neumann_reproduces_linear_solution(d):
    """-Laplace u = 0 with du/dn = g on the whole boundary, u = c + x - 2y (+ 0.5 z): g is constant on each
    face, so the side rule is exact, mean(b) = 0 up to rounding, and the solve with freeNode = 2:N followed by
    the zero-average shift returns the zero-average linear function."""
    m = _geometry(d, 6, 0.2, 34)
    node, elem = m["node"], m["elem"]
    N = node.shape[0]
    grad = np.array([1.0, -2.0, 0.5])[:d]
    faces = {"x0": 10, "x1": 11, "y0": 20, "y1": 21, "z0": 30, "z1": 31}
    flags = meshgen.side_flags(m, faces)
    g_side = np.zeros(flags.shape)
    for nm, code in faces.items():
        ax, sgn = "xyz".index(nm[0]), (1.0 if nm[1] == "1" else -1.0)
        if ax < d:
            g_side[flags == code] = sgn * grad[ax]
    neu = np.where(flags > 1, 2, flags).astype(np.int8)
    rp, col, val, _ = oracle.assemble(d, node, elem)
    _, b = oracle.boundary_terms(d, node, elem, neu, rp, col, val, np.zeros(N), g_side=g_side)
    assert abs(b.mean()) <= 1e-15
    b = oracle.mean_shift(b)
    assert abs(b.sum()) <= 1e-14
    A = dense_from_csr(rp, col, val, N)
    u = np.zeros(N)
    u[1:] = np.linalg.solve(A[1:, 1:], b[1:])
    u0, _ = oracle.zero_average(d, node, elem, u)
    exact, _ = oracle.zero_average(d, node, elem, node @ grad)
    assert np.allclose(u0, exact, rtol=0, atol=1e-11)


@pytest.mark.parametrize("d", [2, 3])
def test_robin_and_dirichlet_reproduce_linear_solution(d):
    """u = 1 + x: Dirichlet u = 1 on x = 0, Robin du/dn + alpha u = 1 + 2 alpha on x = 1 (u = 2 there),
    zero Neumann elsewhere. The Robin matrix is exact for the linear u and the load for the constant g, so
    the solution is u at every node."""
    m = _geometry(d, 5, 0.2, 35)
    node, elem = m["node"], m["elem"]
    N = node.shape[0]
    alpha = 0.7
    faces = {"x0": 1, "x1": 3, "y0": 2, "y1": 2, "z0": 2, "z1": 2}
    flags = meshgen.side_flags(m, faces)
    g_side = np.where(flags == 3, 1.0 + 2.0 * alpha, 0.0)
    rp, col, val, _ = oracle.assemble(d, node, elem)
    val, b = oracle.boundary_terms(d, node, elem, flags, rp, col, val, np.zeros(N), g_side=g_side, alpha=alpha)
    isbd = oracle.boundary(d, N, elem, flags)
    gD = 1.0 + node[:, 0]
    val2, b2, free = oracle.dirichlet(rp, col, val, b, isbd, gD)
    A2 = dense_from_csr(rp, col, val2, N)
    assert np.allclose(np.linalg.solve(A2, b2), gD, rtol=0, atol=1e-12)


def test_mean_shift_and_zero_average():
    m = meshgen.square_mesh(7, 0.2, 36)
    rng = np.random.default_rng(36)
    b = rng.normal(size=m["node"].shape[0]) + 3.0
    s = oracle.mean_shift(b)
    assert abs(s.mean()) <= 1e-14 * np.abs(b).max() and np.allclose(s - b, -b.mean(), rtol=0, atol=1e-14)
    u = rng.normal(size=b.size)
    u0, c = oracle.zero_average(2, m["node"], m["elem"], u)
    meas = np.abs(oracle.measure(2, m["node"], m["elem"]))
    assert abs((u0[m["elem"]].mean(axis=1) * meas).sum()) <= 1e-14 * np.abs(u).max()
    # a constant function's average is the constant
    _, c1 = oracle.zero_average(2, m["node"], m["elem"], np.full(b.size, 4.25))
    assert abs(c1 - 4.25) <= 1e-15


# --- other second-order operators on the same element loop: mass, anisotropic div(K grad u) ------------

@pytest.mark.parametrize("d", [2, 3])
def test_mass_matrix_integrates_products_exactly(d):
    """M_ij = int lambda_i lambda_j: 1^T M 1 = |Omega|, x^T M x = int x^2 = 1/3 on the unit square/cube
    (P1 products are exact), symmetric positive definite; the local matrix equals the degree-2 rule's
    (the 2-D edge midpoints, the 3-D four points) applied to lambda_i lambda_j."""
    m = _geometry(d, 4, 0.2, 61)
    node, elem = m["node"], m["elem"]
    N = node.shape[0]
    c = meshgen.lognormal(61, 3, elem.shape[0])
    rp, col, val, _ = oracle.operator(d, node, elem, oracle.OP_MASS)
    M = dense_from_csr(rp, col, val, N)
    assert np.array_equal(M, M.T)
    one = np.ones(N)
    assert abs(one @ M @ one - 1.0) <= 1e-14
    x = node[:, 0]
    assert abs(x @ M @ x - 1.0 / 3.0) <= 1e-14
    assert np.linalg.eigvalsh(M).min() > 0
    # coefficient: c-weighted, element by element
    rpc, colc, valc, _ = oracle.operator(d, node, elem, oracle.OP_MASS, c)
    meas = np.abs(oracle.measure(d, node, elem))
    assert abs(valc.sum() - (c * meas).sum()) <= 1e-14 * (c * meas).sum()
    # the local matrix by the degree-2 rule on one element
    e = elem[3]
    p = node[e]
    if d == 2:
        lam = np.array([[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
        w = np.full(3, 1.0 / 3.0)
    else:
        a, b = (5 + 3 * math.sqrt(5)) / 20, (5 - math.sqrt(5)) / 20
        lam = np.full((4, 4), b) + np.eye(4) * (a - b)
        w = np.full(4, 0.25)
    loc = meas[3] * np.einsum("q,qi,qj->ij", w, lam, lam)
    one_el, _ = np.zeros(elem.shape[0]), None
    one_el[3] = 1.0
    rp1, col1, val1, _ = oracle.operator(d, node, elem, oracle.OP_MASS, one_el)
    M1 = dense_from_csr(rp1, col1, val1, N)
    assert np.allclose(M1[np.ix_(e, e)], loc, rtol=1e-14, atol=0)


@pytest.mark.parametrize("d", [2, 3])
def test_anisotropic_operator(d):
    """div(K grad u): K = I gives the stiffness matrix; zero row sums; for linear u = g.x the energy
    u^T A u = g^T K g |Omega| exactly (constant K); rotating the mesh by Q and K by Q K Q^T changes nothing."""
    m = _geometry(d, 4, 0.2, 62)
    node, elem = m["node"], m["elem"]
    N, NT = node.shape[0], elem.shape[0]
    nk = d * (d + 1) // 2
    eye = np.array([1.0, 0.0, 1.0]) if d == 2 else np.array([1.0, 0.0, 0.0, 1.0, 0.0, 1.0])
    rpI, colI, vI, _ = oracle.operator(d, node, elem, oracle.OP_ANISO, np.tile(eye, (NT, 1)))
    rpS, colS, vS, _ = oracle.assemble(d, node, elem)
    assert np.array_equal(colI, colS) and np.array_equal(vI, vS)
    if d == 2:
        Kf = np.array([2.0, 0.3, 0.7])
        Km = np.array([[2.0, 0.3], [0.3, 0.7]])
    else:
        Kf = np.array([2.0, 0.3, -0.2, 0.7, 0.1, 1.3])
        Km = np.array([[2.0, 0.3, -0.2], [0.3, 0.7, 0.1], [-0.2, 0.1, 1.3]])
    rp, col, v, sc = oracle.operator(d, node, elem, oracle.OP_ANISO, np.tile(Kf, (NT, 1)))
    A = dense_from_csr(rp, col, v, N)
    S = dense_from_csr(rp, col, sc, N)
    assert np.all(np.abs(A - A.T) <= 1e-15 * (S + S.T))  # symmetric up to the rounding of n_i^T K n_j
    assert np.all(np.abs(A.sum(axis=1)) <= 1e-13 * np.abs(A).sum(axis=1))
    g = np.array([0.4, -1.1, 0.6])[:d]
    u = node @ g
    assert abs(u @ A @ u - g @ Km @ g) <= 1e-13
    th = 0.37
    if d == 2:
        Q = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    else:
        Q = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    KQ = Q @ Km @ Q.T
    iu = np.triu_indices(d)
    rpq, colq, vq, _ = oracle.operator(d, node @ Q.T, elem, oracle.OP_ANISO, np.tile(KQ[iu], (NT, 1)))
    assert np.all(np.abs(vq - v) <= 1e-12 * sc)


# --- load vector with rules of any order ("Numerical Quadrature") -----------------------------------------

@pytest.mark.parametrize("d", [2, 3])
def test_conical_rules_are_exact_to_degree_2n_minus_1(d):
    """int over the simplex of prod lambda_i^a_i = d! prod a_i! / (|a| + d)! (relative to |tau|), for every
    |a| <= 2n - 1; positive weights summing to 1."""
    for n in range(1, 6):
        bary, w = oracle.quad_rule(d, n)
        assert bary.shape == (n ** d, d + 1) and np.all(w > 0) and abs(w.sum() - 1) <= 1e-14
        assert np.allclose(bary.sum(axis=1), 1.0, rtol=0, atol=1e-15) and np.all(bary >= 0)
        for a in np.ndindex(*([2 * n] * (d + 1))):
            if sum(a) > 2 * n - 1:
                continue
            val = float((w * np.prod(bary ** np.array(a), axis=1)).sum())
            exact = math.factorial(d) * np.prod([math.factorial(x) for x in a]) / math.factorial(sum(a) + d)
            assert abs(val - exact) <= 2e-15 * max(1, n), (d, n, a)


@pytest.mark.parametrize("d", [2, 3])
def test_rule_load_vector(d):
    """One point (the centroid) and f = 1 give |tau|/(d+1) per vertex, as the paper's rules do; for a
    polynomial f of degree p the load is the same for every rule with 2n - 1 >= p + 1; for the sine product
    the rules converge (n = 6 and n = 7 agree to 1e-8 on this coarse mesh)."""
    m = _geometry(d, 3, 0.2, 81)
    node, elem = m["node"], m["elem"]
    NT = elem.shape[0]
    bary1, w1 = oracle.quad_rule(d, 1)
    b1 = oracle.rhs_rule(d, node, elem, bary1, w1, oracle.F_CONST)
    b0 = oracle.rhs(d, node, elem, oracle.F_CONST)
    assert np.allclose(b1, b0, rtol=1e-14, atol=0)

    def poly(x):  # degree 3
        return 1.0 + x[..., 0] ** 2 * x[..., 1] - 0.5 * x[..., d - 1] ** 3

    loads = []
    for n in (3, 4, 5):
        bary, w = oracle.quad_rule(d, n)
        pts = np.einsum("qi,tim->tqm", bary, node[elem])
        loads.append(oracle.rhs_rule(d, node, elem, bary, w, oracle.F_QP, poly(pts).ravel()))
    assert np.allclose(loads[0], loads[1], rtol=1e-13, atol=0) and np.allclose(loads[1], loads[2], rtol=1e-13, atol=0)
    b6 = oracle.rhs_rule(d, node, elem, *oracle.quad_rule(d, 6), oracle.F_SINPROD)
    b7 = oracle.rhs_rule(d, node, elem, *oracle.quad_rule(d, 7), oracle.F_SINPROD)
    inner = np.abs(b7) > 1e-3 * np.abs(b7).max()
    assert np.allclose(b6[inner], b7[inner], rtol=1e-8, atol=0)


def _exact_sine_load(d, node, elem):
    """b_i = sum over elements of the integral of prod_m sin(pi x_m) lambda_i over the element, by an
    independent brute force: 2-D adaptive quadrature (scipy.integrate.dblquad) over the reference
    triangle, 3-D a 24^3-point tensor Gauss-Legendre rule (numpy.polynomial.legendre.leggauss) over the
    unit cube mapped onto the reference tetrahedron by the collapsed (Duffy) map with its Jacobian
    (1-v)(1-w)^2 written out. f is evaluated as numpy's sin of pi times the physical coordinate, with no
    integer shift and no sign flip."""
    from scipy.integrate import dblquad
    b = np.zeros(node.shape[0])
    if d == 3:
        g, gw = np.polynomial.legendre.leggauss(24)
        g, gw = 0.5 * (g + 1.0), 0.5 * gw
        U, V, W = np.meshgrid(g, g, g, indexing="ij")
        WT = (gw[:, None, None] * gw[None, :, None] * gw[None, None, :]) * (1 - V) * (1 - W) ** 2
        # (u, v, w) in the unit cube -> reference tetrahedron point (x, y, z), x + y + z <= 1
        X, Y, Z = U * (1 - V) * (1 - W), V * (1 - W), W
        lam = [1 - X - Y - Z, X, Y, Z]
    for e in elem:
        P = node[e]
        J = P[1:] - P[0]
        det = abs(np.linalg.det(J))
        for i in range(d + 1):
            if d == 2:
                def fl(y, x, i=i):
                    p = P[0] + x * J[0] + y * J[1]
                    li = (1 - x - y, x, y)[i]
                    return np.sin(np.pi * p[0]) * np.sin(np.pi * p[1]) * li
                val, _ = dblquad(fl, 0.0, 1.0, 0.0, lambda x: 1.0 - x, epsabs=1e-15, epsrel=1e-13)
            else:
                pts = P[0] + X[..., None] * J[0] + Y[..., None] * J[1] + Z[..., None] * J[2]
                f = np.prod(np.sin(np.pi * pts), axis=-1)
                val = float((WT * f * lam[i]).sum())
            b[e[i]] += det * val
    return b


@pytest.mark.parametrize("d", [2, 3])
def test_sine_load_next_to_the_integers_keeps_relative_accuracy(d):
    """The load vector of f = prod sin(pi x_m) (Sec. 3.2 midpoint rule; 3-D four-point rule) on one element
    whose vertices lie within 4e-4 of the corner (1, 1[, 1]), where f is about 1e-3 per coordinate: against
    the same rule evaluated in 40-digit arithmetic at the exact points, every entry within 2^-48 relative.
    Forming a point first and reducing it by the integer afterwards (the sum of coordinates near 2 rounds to
    2^-52) would be off by about 1e-12 here."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(7 + d)
    if d == 2:
        node = np.array([[1 - 3.7e-4, 1 - 1.1e-4], [1 - 0.9e-4, 1 - 3.3e-4], [1 - 1.3e-4, 1 - 0.7e-4]])
        node += rng.uniform(-1e-6, 1e-6, node.shape)
    else:
        node = np.array([[1 - 3.7e-4, 1 - 1.1e-4, 1 - 2.1e-4], [1 - 0.9e-4, 1 - 3.3e-4, 1 - 1.9e-4],
                         [1 - 1.3e-4, 1 - 0.7e-4, 1 - 3.9e-4], [1 - 2.2e-4, 1 - 2.6e-4, 1 - 0.6e-4]])
        node += rng.uniform(-1e-6, 1e-6, node.shape)
    elem = np.arange(d + 1, dtype=np.int32)[None, :]
    meas = oracle.measure(d, node, elem)[0]
    if meas < 0:  # positive orientation
        elem = elem[:, [1, 0] + list(range(2, d + 1))]
        meas = -meas
    b = oracle.rhs(d, node, elem, oracle.F_SINPROD)
    X = [[mpmath.mpf(float(v)) for v in node[i]] for i in elem[0]]
    if d == 2:
        mids = [[(X[(q + 1) % 3][m] + X[(q + 2) % 3][m]) / 2 for m in range(2)] for q in range(3)]
        f = [mpmath.sin(mpmath.pi * p[0]) * mpmath.sin(mpmath.pi * p[1]) for p in mids]
        exact = [mpmath.mpf(float(meas)) * (f[(i + 1) % 3] + f[(i + 2) % 3]) / 6 for i in range(3)]
    else:
        s5 = mpmath.sqrt(5)
        al, be = (5 + 3 * s5) / 20, (5 - s5) / 20
        pts = [[sum((al if i == q else be) * X[i][m] for i in range(4)) for m in range(3)] for q in range(4)]
        f = [mpmath.sin(mpmath.pi * p[0]) * mpmath.sin(mpmath.pi * p[1]) * mpmath.sin(mpmath.pi * p[2]) for p in pts]
        exact = [mpmath.mpf(float(meas)) / 4 * sum(f[q] * (al if i == q else be) for q in range(4)) for i in range(4)]
    for i in range(d + 1):
        v = int(elem[0][i])
        assert abs(mpmath.mpf(float(b[v])) - exact[i]) <= 2.0 ** -48 * abs(exact[i]), (i, float(b[v]), exact[i])


@pytest.mark.parametrize("d", [2, 3])
def test_rule_sine_product_branch(d):
    """The sine-product branch of the rule load vector (the points are shifted by an integer near the
    element and the sign follows its parity) pinned two ways that do not use that branch:
    (1) against the exact integrals by an independent brute force (adaptive 2-D quadrature, a tensor
    Gauss-Legendre rule in 3-D) on a mesh moved by an integer vector of odd sum, so that the branch's
    shift is nonzero and its sign flips: the 8-point conical rule (exact to degree 15, h = 1/4) agrees to
    1e-12; (2) the periodicity sin(pi (x + s)) = (-1)^s sin(pi x): moving the mesh by an integer vector s
    multiplies the load by (-1)^(sum s)."""
    m = _geometry(d, 4 if d == 2 else 2, 0.2 if d == 2 else 0.1, 83)
    node, elem = m["node"], m["elem"]
    if d == 3:
        node = node * 0.5  # h = 1/4
    shift = np.array([3.0, -2.0] if d == 2 else [3.0, -2.0, 2.0])  # odd sum: the load changes sign
    moved = node + shift
    bary, w = oracle.quad_rule(d, 8)
    b_rule = oracle.rhs_rule(d, moved, elem, bary, w, oracle.F_SINPROD)
    b_exact = _exact_sine_load(d, moved, elem)
    scale = _exact_sine_load(d, node, elem)  # the same integrals unmoved: b_exact = -scale up to rounding
    assert np.all(np.abs(b_exact + scale) <= 1e-12 * np.abs(scale).max())
    assert np.all(np.abs(b_rule - b_exact) <= 1e-12 * np.abs(b_exact).max()), np.abs(b_rule - b_exact).max()
    # periodicity with a rule of modest order, several shifts of both parities
    bary3, w3 = oracle.quad_rule(d, 3)
    b0 = oracle.rhs_rule(d, node, elem, bary3, w3, oracle.F_SINPROD)
    shifts = ([1, 0], [0, -3], [2, 2], [5, 1], [-4, 7]) if d == 2 else ([1, 0, 0], [0, 2, 1], [-3, 1, 1], [2, 2, -2])
    for s in shifts:
        bs = oracle.rhs_rule(d, node + np.array(s, float), elem, bary3, w3, oracle.F_SINPROD)
        sign = -1.0 if sum(s) % 2 else 1.0
        assert np.all(np.abs(bs - sign * b0) <= 1e-12 * np.abs(b0).max()), (s, np.abs(bs - sign * b0).max())


# --- the whole method: assemble, eliminate the Dirichlet rows, solve ---------------------------------

@pytest.mark.parametrize("d", [2, 3])
def test_reduced_solve_by_lift_equals_eliminated_solve_and_reproduces_linear_data(d):
    """Sec. 3.3 two ways: oracle.solve_reduced (lift b - A u_D, solve on freeNode) and the symmetric
    eliminated system of oracle.dirichlet solved whole give the same u; with f = 0, k = 1 and a linear g_D
    both reproduce the linear function (P1 contains it)."""
    sp = pytest.importorskip("scipy.sparse")
    spla = pytest.importorskip("scipy.sparse.linalg")
    m = meshgen.square_mesh(9, 0.2, 71, True) if d == 2 else meshgen.kuhn_mesh(4, 0.1, 71)
    node, elem = m["node"], m["elem"]
    N, NT = node.shape[0], elem.shape[0]
    k = meshgen.lognormal(71, 3, NT)
    isbd = oracle.boundary(d, N, elem)
    gD = 1.0 + node @ np.arange(1.0, d + 1.0)
    rp, col, val, _ = oracle.assemble(d, node, elem, k)
    b = oracle.rhs(d, node, elem, oracle.F_SINPROD)
    u1 = oracle.solve_reduced(rp, col, val, b, isbd, gD)
    v2, b2, _ = oracle.dirichlet(rp, col, val, b, isbd, gD)
    u2 = spla.spsolve(sp.csr_matrix((v2, col, rp), shape=(N, N)).tocsc(), b2)
    assert np.allclose(u1, u2, rtol=0, atol=1e-12 * np.abs(u2).max())
    assert np.array_equal(u1[isbd.astype(bool)], gD[isbd.astype(bool)])
    rp, col, val1, _ = oracle.assemble(d, node, elem, None)
    ul = oracle.solve_reduced(rp, col, val1, np.zeros(N), isbd, gD)
    assert np.allclose(ul, gD, rtol=0, atol=1e-12 * np.abs(gD).max())



@pytest.mark.parametrize("d", [2, 3])
def test_poisson_solution_converges_at_second_order(d):
    """-Laplace u = f on the unit square / cube with u = 0 on the boundary and f the sine product: the
    exact solution is f / (d pi^2). Solving the oracle's eliminated system on uniform meshes halving h,
    the nodal error falls by about 4 per halving (second order for P1 at the nodes), and on the finest
    mesh it is small in absolute terms. A wrong factor in the stiffness matrix or the load vector
    (|tau|, d!, the quadrature weights, a sign) leaves an O(1) error that does not fall."""
    sp = pytest.importorskip("scipy.sparse")
    spla = pytest.importorskip("scipy.sparse.linalg")
    ns = (8, 16, 32) if d == 2 else (4, 8, 16)
    errs = []
    for n in ns:
        m = meshgen.square_mesh(n) if d == 2 else meshgen.kuhn_mesh(n)
        node, elem = m["node"], m["elem"]
        N = node.shape[0]
        rp, col, val, _ = oracle.assemble(d, node, elem, None)
        b = oracle.rhs(d, node, elem, oracle.F_SINPROD)
        isbd = oracle.boundary(d, N, elem)
        v2, b2, free = oracle.dirichlet(rp, col, val, b, isbd)
        A = sp.csr_matrix((v2, col, rp), shape=(N, N))
        u = spla.spsolve(A.tocsc(), b2)
        exact = np.prod(np.sin(np.pi * node), axis=1) / (d * np.pi ** 2)
        errs.append(float(np.abs(u - exact).max()))
    rates = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.5 < r < 4.5 for r in rates), (errs, rates)
    umax = 1.0 / (d * np.pi ** 2)
    assert errs[-1] < (1e-3 if d == 2 else 1e-2) * umax, errs
