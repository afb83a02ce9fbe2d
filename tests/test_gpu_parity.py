"""GPU path (through the C ABI) against the CPU oracle, element by element.

Pattern, slot map, boundary mask, freeNode and the Dirichlet rows: bit-exact. FP64 values:
|gpu - oracle| <= 1e-12 * scale, scale = sum over the slot's contributions of their magnitude bound.
"""
import numpy as np
import pytest
import torch

import meshgen
import oracle
from tests._common import BWD_TOL, TOL, assert_close_scaled, dev, gpu_slot_to_tij, host, mesh_case, sample_rows

pytestmark = pytest.mark.gpu

fa = pytest.importorskip("paper_1804_05156_gb300")

CASES = ["c1", "sq2", "sq37p", "kuhn5", "kuhn7s", "delaunay2", "delaunay3"]
VARIANTS = [fa.FEM_DETERMINISTIC, fa.FEM_ATOMIC]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fa.build()
    oracle.build()


@pytest.mark.parametrize("case", CASES)
def test_pattern_bit_exact(case):
    d, node, elem, _, _ = mesh_case(case)
    N = node.shape[0]
    p = fa.Pattern(dev(elem), N)
    rp, col = oracle.pattern(d, N, elem)
    assert p.nnz == rp[-1]
    assert np.array_equal(host(p.row_ptr), rp)
    assert np.array_equal(host(p.col_idx), col)
    slot_o = oracle.slots(d, N, elem, rp, col)
    assert np.array_equal(gpu_slot_to_tij(host(p.slot), elem.shape[0], d + 1), slot_o)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("case", CASES)
def test_values_match_oracle(case, variant):
    d, node, elem, k, f_kind = mesh_case(case)
    N = node.shape[0]
    p = fa.Pattern(dev(elem), N)
    val, b = fa.assemble(p, dev(node), None if k is None else dev(k), f_kind, None, variant)
    fa.get_error()
    rp, col, vo, so = oracle.assemble(d, node, elem, k)
    assert_close_scaled(host(val), vo, so, what="stiffness")
    bo = oracle.rhs(d, node, elem, f_kind)
    # all meshes lie in the unit box, where f >= 0: every contribution to b_i has the sign of b_i
    assert_close_scaled(host(b), bo, np.abs(bo), what="rhs")
    if case == "c1":
        v = host(val)
        n = 64
        for j in range(1, n):
            for i in range(1, n):
                r = j * (n + 1) + i
                assert v[rp[r]:rp[r + 1]].tolist() == [0.0, -1.0, -1.0, 4.0, -1.0, -1.0, 0.0]


@pytest.mark.parametrize("case", ["c1", "sq37p", "kuhn5", "kuhn7s", "delaunay2", "delaunay3"])
def test_locality_plan_values_match_oracle(case):
    """The owner-computes kernel with the geometric (Morton) block plan, and with the default plan."""
    d, node, elem, k, f_kind = mesh_case(case)
    N = node.shape[0]
    p = fa.Pattern(dev(elem), N)
    rp, col, vo, so = oracle.assemble(d, node, elem, k)
    bo = oracle.rhs(d, node, elem, f_kind)
    kd = None if k is None else dev(k)
    v_default, b_default = fa.assemble(p, dev(node), kd, f_kind, None, fa.FEM_DETERMINISTIC)
    fa.fem_pattern_set_locality(p, dev(node))
    val, b = fa.assemble(p, dev(node), kd, f_kind, None, fa.FEM_DETERMINISTIC)
    fa.get_error()
    for v_, b_ in ((val, b), (v_default, b_default)):
        assert_close_scaled(host(v_), vo, so, what="stiffness")
        assert_close_scaled(host(b_), bo, np.abs(bo), what="rhs")
    # the geometric plan changes only which CTA owns a row, not the summation order of any entry
    assert torch.equal(val, v_default) and torch.equal(b, b_default)
    # and a plan built from other coordinates gives the same bits
    rng = np.random.default_rng(3)
    fa.fem_pattern_set_locality(p, dev(rng.normal(size=node.shape)))
    v3, b3 = fa.assemble(p, dev(node), kd, f_kind, None, fa.FEM_DETERMINISTIC)
    assert torch.equal(v3, val) and torch.equal(b3, b)


@pytest.mark.parametrize("case", ["sq37p", "kuhn7s", "delaunay3"])
def test_far_from_the_origin(case):
    """The same meshes moved far from the origin (coordinates ~1e4): edge vectors stay exact (the
    three-float split), so the stiffness values and the constant-f load still match the oracle within
    1e-12 of their scale (the oracle's FP64 differences of nearby coordinates are exact too). The
    sine-product load is left out here: the oracle rounds each midpoint (x_i + x_j)/2 to ~1e-12 in
    absolute terms at this magnitude, which the float-float path does not."""
    d, node, elem, k, _ = mesh_case(case)
    shift = np.array([12345.0, -6789.0, 31415.0][:d])
    far = node + shift
    p = fa.Pattern(dev(elem), far.shape[0])
    fa.fem_pattern_set_locality(p, dev(far))
    v, b = fa.assemble(p, dev(far), dev(k), fa.FEM_F_CONST, dev(np.array([2.5])))
    fa.get_error()
    _, _, vo, so = oracle.assemble(d, far, elem, k)
    assert_close_scaled(host(v), vo, so)
    bo = oracle.rhs(d, far, elem, oracle.F_CONST, np.array([2.5]))
    assert_close_scaled(host(b), bo, np.abs(bo) + 1e-300, what="rhs")


@pytest.mark.parametrize("case", ["sq37p", "kuhn5", "delaunay2"])
def test_every_launch_shape_gives_the_same_bits(case):
    """Deterministic means independent of the launch: all shapes, one CTA per block or persistent."""
    d, node, elem, k, f_kind = mesh_case(case)
    p = fa.Pattern(dev(elem), node.shape[0])
    fa.fem_pattern_set_locality(p, dev(node))
    ref = None
    shapes = [(512, 2), (256, 4), (256, 2)] if d == 2 else [(512, 1), (256, 2), (256, 1)]
    for thr, cta in shapes:
        for pers in (False, True):
            try:
                fa.fem_pattern_force_launch(p, thr, cta, pers)
            except fa.FemError as e:
                assert e.code == fa.FEM_ERR_ARG  # this plan does not fit the shape
                continue
            v, b = fa.assemble(p, dev(node), dev(k), f_kind, None, fa.FEM_DETERMINISTIC)
            if ref is None:
                ref = (v, b)
                _, _, vo, so = oracle.assemble(d, node, elem, k)
                assert_close_scaled(host(v), vo, so)
            else:
                assert torch.equal(v, ref[0]) and torch.equal(b, ref[1]), (thr, cta, pers)


def _fan(m_ring, seed=0):
    """A disc of m_ring triangles around one centre vertex: the centre's row has m_ring + 1 entries."""
    rng = np.random.default_rng(seed)
    ang = np.sort(rng.uniform(0, 2 * np.pi, m_ring))
    node = np.vstack([[0.0, 0.0], np.stack([np.cos(ang), np.sin(ang)], 1) * rng.uniform(0.8, 1.2, (m_ring, 1))])
    elem = np.array([[0, 1 + i, 1 + (i + 1) % m_ring] for i in range(m_ring)], np.int32)
    return node, elem


@pytest.mark.parametrize("case", ["sq37p", "kuhn5", "kuhn7s", "delaunay2", "delaunay3"])
def test_all_value_paths_give_the_same_bits(case):
    """Tiles (both sizes) and owner-computes blocks sum every entry in the same order: identical bits,
    for every load kind and for stiffness-only / load-only calls; the FP64 two-pass path agrees with
    the oracle."""
    d, node, elem, k, _ = mesh_case(case)
    N, NT = node.shape[0], elem.shape[0]
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    kd = None if k is None else dev(k)
    fq = np.random.default_rng(8).normal(size=NT * (d + 1))
    loads = [(fa.FEM_F_SINPROD, None), (fa.FEM_F_CONST, dev(np.array([2.5]))), (fa.FEM_F_QPVALUES, dev(fq))]
    paths = [(fa.FEM_PATH_TILES, 256), (fa.FEM_PATH_TILES, 128), (fa.FEM_PATH_TILES_FUSED, 128),
             (fa.FEM_PATH_TILES_FUSED, 256), (fa.FEM_PATH_BLOCKED, 0)]
    names = {fa.FEM_PATH_TILES: "tiles", fa.FEM_PATH_TILES_FUSED: "tiles_fused", fa.FEM_PATH_BLOCKED: "blocked"}
    for fk, farg in loads:
        ref = None
        for path, te in paths:
            fa.fem_pattern_force_path(p, path, te or 256)
            assert fa.fem_pattern_value_path(p)["path"] == names[path]
            v, b = fa.assemble(p, dev(node), kd, fk, farg, fa.FEM_DETERMINISTIC)
            vs = torch.empty_like(v)
            fa.fem_assemble(p, dev(node), kd, fk, farg, vs, None, fa.FEM_DETERMINISTIC)
            bs = torch.empty_like(b)
            fa.fem_assemble(p, dev(node), kd, fk, farg, None, bs, fa.FEM_DETERMINISTIC)
            fa.get_error()
            assert torch.equal(vs, v) and torch.equal(bs, b), (path, te, fk)
            if ref is None:
                ref = (v, b)
                _, _, vo, so = oracle.assemble(d, node, elem, k)
                assert_close_scaled(host(v), vo, so)
                ok = {fa.FEM_F_SINPROD: oracle.F_SINPROD, fa.FEM_F_CONST: oracle.F_CONST,
                      fa.FEM_F_QPVALUES: oracle.F_QP}[fk]
                oarg = {fa.FEM_F_SINPROD: None, fa.FEM_F_CONST: np.array([2.5]), fa.FEM_F_QPVALUES: fq}[fk]
                sarg = np.abs(oarg) if oarg is not None else None
                bo = oracle.rhs(d, node, elem, ok, oarg)
                bsc = oracle.rhs(d, node, elem, ok, sarg) if fk == fa.FEM_F_QPVALUES else np.abs(bo)
                assert_close_scaled(host(b), bo, bsc + 1e-300, what="rhs")
            else:
                assert torch.equal(v, ref[0]) and torch.equal(b, ref[1]), (path, te, fk)
    fa.fem_pattern_force_path(p, fa.FEM_PATH_TWO_PASS)
    assert fa.fem_pattern_value_path(p)["path"] == "two_pass"
    v2, _ = fa.assemble(p, dev(node), kd, fa.FEM_F_SINPROD, None, fa.FEM_DETERMINISTIC)
    _, _, vo, so = oracle.assemble(d, node, elem, k)
    assert_close_scaled(host(v2), vo, so)


@pytest.mark.parametrize("d", [2, 3])
def test_fused_grid_barrier_gives_up_with_a_timeout(d):
    """The fused launch's grid barrier waits for one CTA more than the launch has (an arrival that never
    comes, set by fem_pattern_barrier_fault) and a short poll limit: every CTA gives up, the device error
    word reads FEM_ERR_TIMEOUT, and the context stays usable: with the defaults restored the next launch
    on the same pattern gives the oracle's values."""
    d_, node, elem, k, _ = mesh_case("sq37p" if d == 2 else "kuhn7s")
    N = node.shape[0]
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    fa.fem_pattern_force_path(p, fa.FEM_PATH_TILES_FUSED, 128)
    fa.fem_pattern_barrier_fault(p, 1, 4096)
    val, b = fa.assemble(p, dev(node), dev(k), fa.FEM_F_SINPROD, None, fa.FEM_DETERMINISTIC)
    with pytest.raises(fa.FemError) as e:
        fa.get_error()
    assert e.value.code == fa.FEM_ERR_TIMEOUT
    fa.get_error()  # the word was cleared by the read
    fa.fem_pattern_barrier_fault(p, 0, 0)
    val, b = fa.assemble(p, dev(node), dev(k), fa.FEM_F_SINPROD, None, fa.FEM_DETERMINISTIC)
    fa.get_error()
    _, _, vo, so = oracle.assemble(d, node, elem, k)
    assert_close_scaled(host(val), vo, so)
    bo = oracle.rhs(d, node, elem, oracle.F_SINPROD)
    assert_close_scaled(host(b), bo, np.abs(bo) + 1e-300, what="rhs")
    with pytest.raises(fa.FemError) as e:
        fa.fem_pattern_barrier_fault(p, -1, 0)
    assert e.value.code == fa.FEM_ERR_ARG


@pytest.mark.parametrize("d", [2, 3])
def test_row_shards_on_the_gpu_give_the_global_rows_bit_for_bit(d):
    """The row-ownership sharding of the multi-rank path, run through the CUDA library on one GPU: each
    shard's sub-mesh (every element touching the rank's vertex range, global order kept) gets its own
    pattern, locality plan and assembly, and its owned rows equal the whole-mesh GPU rows bit for bit
    (pattern, values, load vector) for 2 and 3 ranks: no exchange of data is needed."""
    from paper_1804_05156_gb300 import partition
    m = meshgen.square_mesh(48, 0.2, 61, permute=True) if d == 2 else meshgen.kuhn_mesh(9, 0.1, 62)
    node, elem = m["node"], m["elem"]
    N, NT = node.shape[0], elem.shape[0]
    k = meshgen.lognormal(63, meshgen.TAG_COEF, NT)
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    val, b = fa.assemble(p, dev(node), dev(k), fa.FEM_F_SINPROD, None, fa.FEM_DETERMINISTIC)
    fa.get_error()
    rp, col, val, b = host(p.row_ptr), host(p.col_idx), host(val), host(b)
    for P in (2, 3):
        got = []
        for lo, hi in partition.row_ranges(N, P, elem):
            sh = partition.shard_mesh(elem, lo, hi)
            sub_node = np.ascontiguousarray(node[sh["vert_ids"]])
            q = fa.Pattern(dev(sh["elem_local"]), sub_node.shape[0])
            fa.fem_pattern_set_locality(q, dev(sub_node))
            sv, sb = fa.assemble(q, dev(sub_node), dev(k[sh["elem_ids"]]), fa.FEM_F_SINPROD, None,
                                 fa.FEM_DETERMINISTIC)
            fa.get_error()
            got.append(partition.owned_rows(sh, host(q.row_ptr), host(q.col_idx), host(sv), host(sb)))
        assert np.array_equal(np.concatenate([g[0] for g in got]), np.arange(N))
        assert np.array_equal(np.concatenate([g[1] for g in got]), np.diff(rp))
        assert np.array_equal(np.concatenate([g[2] for g in got]), col)
        assert np.array_equal(np.concatenate([g[3] for g in got]).view(np.uint64), val.view(np.uint64))
        assert np.array_equal(np.concatenate([g[4] for g in got]).view(np.uint64), b.view(np.uint64))


def _expect_in_range(d, node, elem):
    """The documented range of the float-float path, predicted on the host from the FP64 oracle's
    measures: (stiffness in range, load of f = 1 in range). 2-D: the element's power-of-two frame keeps the
    stiffness (degree 0) in range at any scale; the load contribution |tau|/3 must lie in [2^-84, 2^120].
    3-D: 6|tau| must lie in [2^-72, 2^87] for anything at all."""
    meas = np.abs(oracle.measure(d, node, elem))
    if d == 2:
        c = meas / 3.0
        return True, bool(c.min() >= 2.0 ** -84 and c.max() <= 2.0 ** 120)
    v6 = 6.0 * meas
    ok = bool(v6.min() >= 2.0 ** -72 and v6.max() <= 2.0 ** 87)
    return ok, ok


def _expect_range_error(call):
    call()
    with pytest.raises(fa.FemError) as err:
        fa.get_error()
    assert err.value.code == fa.FEM_ERR_RANGE


@pytest.mark.parametrize("e", [-40, -27, -20, 0, 30, 40])
@pytest.mark.parametrize("case", ["sq37p", "kuhn7s", "delaunay3"])
def test_scaled_meshes_keep_the_parity_bar_or_report_the_range(case, e):
    """The mesh scaled by 2^e (coordinates exactly scaled, so the FP64 oracle's values scale exactly too):
    where the documented range holds (_expect_in_range), the stiffness (degree d - 2 in the coordinates),
    the load vector of f = 1 (degree d) and the adjoint stay within the parity bar on every value path;
    where it does not, the call reports FEM_ERR_RANGE. 2-D computes in the element's own power-of-two
    frame, so its stiffness is in range at every scale here while its load leaves the range below about
    2^-40 (|tau|/3 < 2^-84). 3-D computes at the element's own scale: kuhn7s at 2^-20 is a mesh of
    1e-7-sized tetrahedra (6|tau| near 2^-68) and still in range; at 2^-27 and 2^40 it is not. (A
    sine-product load is a different matter at these scales: at 2^-40 its values fall below the float
    range, which test_inputs_beyond_the_float_float_range_are_reported covers, and at 2^30 the FP64
    rounding of the quadrature points alone moves sin(pi x) by more than the bar.)"""
    d, node, elem, k, _ = mesh_case(case)
    node = np.ldexp(node, e)
    N, NT = node.shape[0], elem.shape[0]
    a_ok, b_ok = _expect_in_range(d, node, elem)
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    nd, kd = dev(node), dev(k if k is not None else np.ones(NT))
    _, _, vo, so = oracle.assemble(d, node, elem, k)
    bo = oracle.rhs(d, node, elem, oracle.F_CONST)
    for path, te in ((fa.FEM_PATH_TILES, 128), (fa.FEM_PATH_TILES_FUSED, 256), (fa.FEM_PATH_BLOCKED, 0)):
        fa.fem_pattern_force_path(p, path, te or 256)
        val = torch.empty(p.nnz, dtype=torch.float64, device="cuda")
        b = torch.empty(N, dtype=torch.float64, device="cuda")
        stiff = lambda: fa.fem_assemble_stiffness(p, nd, kd, val)
        load = lambda: fa.fem_assemble_rhs(p, nd, fa.FEM_F_CONST, None, b)
        if a_ok:
            stiff()
            fa.get_error()
            assert_close_scaled(host(val), vo, so, what="stiffness at 2^%d" % e)
        else:
            _expect_range_error(stiff)
        if b_ok:
            load()
            fa.get_error()
            assert_close_scaled(host(b), bo, np.abs(bo) + 1e-300, what="rhs at 2^%d" % e)
        else:
            _expect_range_error(load)
    if not (a_ok and b_ok):
        return
    rp, col = host(p.row_ptr).astype(np.int64), host(p.col_idx).astype(np.int64)
    slot = oracle.slots(d, N, elem, rp, col)
    w, r = meshgen.normal(5, meshgen.TAG_W, p.nnz), meshgen.normal(5, meshgen.TAG_R, N)
    gno, gko, gnm, gkm = oracle.backward(d, node, elem, k, oracle.F_CONST, None, slot, w, r, with_scale=True)
    gn = torch.empty((N, d), dtype=torch.float64, device="cuda")
    gk = torch.empty(NT, dtype=torch.float64, device="cuda")
    fa.fem_assemble_backward(p, nd, kd, fa.FEM_F_CONST, None, dev(w), dev(r), gn, gk)
    fa.get_error()
    assert_close_scaled(host(gn), gno, gnm, tol=BWD_TOL, what="node gradient at 2^%d" % e)
    assert_close_scaled(host(gk), gko, gkm, tol=BWD_TOL, what="k gradient at 2^%d" % e)


@pytest.mark.parametrize("shear", [0.0, 40.0, 200.0])
def test_2d_stiffness_within_its_error_bound_on_sheared_meshes(shear):
    """The per-entry error bound of the 2-D stiffness (the design's section 2: (65.1 + 0.1 kappa_A) u^2 per
    contribution against its scale term, 3 u^2 per running-sum step, u = 2^-24), on meshes sheared so
    that the conditioning of the element area kappa_A = (|e1x e2y| + |e1y e2x|) / |2 area| grows to
    about 2 shear: every CSR value of the GPU path within that bound, with kappa_A the mesh's largest and
    m the entry's number of contributions, plus the FP64 oracle's own rounding of the area
    ((2 kappa_A + 1) 2^-53). The bound's kappa_A term comes from the one FP64 cross product; the
    largest error seen is printed in u^2."""
    m = meshgen.square_mesh(48, 0.2, 77, permute=True)
    node, elem = m["node"].copy(), m["elem"]
    node[:, 0] += shear * node[:, 1]
    node[:, 1] *= 1e-3
    NT = elem.shape[0]
    k = meshgen.lognormal(77, meshgen.TAG_COEF, NT)
    X = node[elem]
    e1, e2 = X[:, 0] - X[:, 2], X[:, 1] - X[:, 0]
    kap = (np.abs(e1[:, 0] * e2[:, 1]) + np.abs(e1[:, 1] * e2[:, 0])) / np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    kmax = float(kap.max())
    p = fa.Pattern(dev(elem), node.shape[0])
    fa.fem_pattern_set_locality(p, dev(node))
    val = torch.empty(p.nnz, dtype=torch.float64, device="cuda")
    fa.fem_assemble_stiffness(p, dev(node), dev(k), val)
    fa.get_error()
    rp, col, vo, so = oracle.assemble(2, node, elem, k)
    # contributions per entry: elements on the edge (off-diagonal) or at the vertex (diagonal)
    N = node.shape[0]
    deg = np.bincount(elem.ravel(), minlength=N)
    rows = np.repeat(np.arange(N), np.diff(rp))
    diag = rows == col
    mcount = np.where(diag, deg[rows], 2)
    u2 = 2.0 ** -48
    per = 65.1 + 0.1 * kmax + (2 * kmax + 1) / 32 + np.where(diag, 3.0, 0.0)
    bound = (per + 3.0 * mcount + 0.05) * u2 * so
    err = np.abs(host(val) - vo)
    assert (err <= bound).all(), (kmax, float((err / np.maximum(so, 1e-300)).max() / u2))
    print("kappa_A max %.1f: worst error %.1f u^2 of the scale" % (kmax, float((err / np.maximum(so, 1e-300)).max() / u2)))


@pytest.mark.parametrize("d", [2, 3])
def test_inputs_beyond_the_float_float_range_are_reported(d):
    """Where a float-float result cannot keep its precision the kernels say so (FEM_ERR_RANGE) instead of
    returning a silently degraded value: a load vector whose element measures are below 2^-96 (mesh
    scaled by 2^-70), or above 2^96 (scaled by 2^60), and a coefficient of 1e-40. Within range the
    same pattern assembles normally afterwards, and a sine-product load on a mesh at 2^-40 (values near
    2^-168) is reported too."""
    d_, node, elem, k, _ = mesh_case("sq37p" if d == 2 else "kuhn5")
    p = fa.Pattern(dev(elem), node.shape[0])
    fa.fem_pattern_set_locality(p, dev(node))
    kd = dev(k if k is not None else np.ones(elem.shape[0]))
    for e in (-70, 60):
        fa.assemble(p, dev(np.ldexp(node, e)), kd, fa.FEM_F_CONST, None, fa.FEM_DETERMINISTIC)
        with pytest.raises(fa.FemError) as err:
            fa.get_error()
        assert err.value.code == fa.FEM_ERR_RANGE, e
    fa.assemble(p, dev(np.ldexp(node, -40)), kd, fa.FEM_F_SINPROD, None, fa.FEM_DETERMINISTIC)
    with pytest.raises(fa.FemError) as err:
        fa.get_error()
    assert err.value.code == fa.FEM_ERR_RANGE
    kk = np.ones(elem.shape[0])
    kk[3] = 1e-40
    fa.assemble(p, dev(node), dev(kk), fa.FEM_F_CONST, None, fa.FEM_DETERMINISTIC)
    with pytest.raises(fa.FemError) as err:
        fa.get_error()
    assert err.value.code == fa.FEM_ERR_RANGE
    fa.assemble(p, dev(node), kd, fa.FEM_F_CONST, None, fa.FEM_DETERMINISTIC)
    fa.get_error()


@pytest.mark.parametrize("d", [2, 3])
def test_every_entry_of_a_fine_mesh(d):
    """Every CSR value and every load entry of a fine jittered mesh (1024^2 triangles, element rows
    permuted; 64^3 Kuhn tetrahedra) against the oracle, sine-product load: the rows next to x = 1 and y = 1,
    where sin(pi x/2) and cos(pi x/2) are taken within 1e-3 of 1/2 and the last bits of x decide the
    cosine's relative accuracy, are among them."""
    m = meshgen.square_mesh(1024, 0.2, 1804, permute=True) if d == 2 else meshgen.kuhn_mesh(64, 0.1, 1807)
    node, elem = m["node"], m["elem"]
    k = meshgen.lognormal(1804, meshgen.TAG_COEF, elem.shape[0])
    p = fa.Pattern(dev(elem), node.shape[0])
    fa.fem_pattern_set_locality(p, dev(node))
    val, b = fa.assemble(p, dev(node), dev(k), fa.FEM_F_SINPROD)
    fa.get_error()
    _, _, vo, so = oracle.assemble(d, node, elem, k)
    bo = oracle.rhs(d, node, elem, oracle.F_SINPROD)
    assert_close_scaled(host(val), vo, so, what="stiffness")
    assert_close_scaled(host(b), bo, np.abs(bo) + 1e-300, what="rhs")


@pytest.mark.parametrize("d", [2, 3])
def test_sine_load_at_large_coordinates(d):
    """The sine-product load on a uniform mesh moved by 2^26 in every coordinate (plus 1 in the first, so
    the sign flips): the coordinates stay exact in FP64 (multiples of 2^-6 or 2^-2), and by periodicity the
    exact load is minus the oracle's load on the unmoved mesh (in 2-D the oracle's own midpoints stay exact
    and it agrees; in 3-D its FP64 quadrature points round at 2^-26 and it does not). The reductions of x
    must keep the parts of x below the leading float's last bit (2^3 at 2^26): every entry within the bar."""
    m = meshgen.square_mesh(64) if d == 2 else meshgen.kuhn_mesh(4)
    node = m["node"] + 2.0 ** 26
    node[:, 0] += 1.0
    elem = m["elem"]
    p = fa.Pattern(dev(elem), node.shape[0])
    fa.fem_pattern_set_locality(p, dev(node))
    bo = -oracle.rhs(d, m["node"], elem, oracle.F_SINPROD)
    if d == 2:
        assert np.array_equal(oracle.rhs(d, node, elem, oracle.F_SINPROD), bo)
    for path, te in ((fa.FEM_PATH_TILES, 128), (fa.FEM_PATH_BLOCKED, 0)):
        fa.fem_pattern_force_path(p, path, te or 256)
        b = torch.empty(p.N, dtype=torch.float64, device="cuda")
        fa.fem_assemble(p, dev(node), None, fa.FEM_F_SINPROD, None, None, b, fa.FEM_DETERMINISTIC)
        fa.get_error()
        assert_close_scaled(host(b), bo, np.abs(bo) + 1e-300, what="rhs at 2^26")


def test_long_rows_take_the_tile_path():
    """A vertex with 40 neighbours (row of 41 entries) is beyond the owner-computes records (32 per
    row) but within the tile path's (256)."""
    node, elem = _fan(40, 4)
    p = fa.Pattern(dev(elem), node.shape[0])
    fa.fem_pattern_set_locality(p, dev(node))
    assert fa.fem_pattern_value_path(p)["path"] in ("tiles", "tiles_fused")
    v, b = fa.assemble(p, dev(node), None, fa.FEM_F_SINPROD, None, fa.FEM_DETERMINISTIC)
    fa.get_error()
    _, _, vo, so = oracle.assemble(2, node, elem, None)
    assert_close_scaled(host(v), vo, so)
    bo = oracle.rhs(2, node, elem, oracle.F_SINPROD)
    assert_close_scaled(host(b), bo, np.abs(bo) + 1e-300, what="rhs")
    with pytest.raises(fa.FemError) as e:
        fa.fem_pattern_force_path(p, fa.FEM_PATH_BLOCKED)
    assert e.value.code == fa.FEM_ERR_STATE


def test_rows_beyond_every_plan_take_the_two_pass_path():
    """A vertex with 300 neighbours (row of 301 entries) is beyond both locality plans: assembly and the
    backward run on the FP64 two-pass and caller-order paths and still match the oracle; the calls that
    need the tile plan (other operators, y = A u) refuse with FEM_ERR_STATE instead of running."""
    node, elem = _fan(300, 6)
    N, NT = node.shape[0], elem.shape[0]
    k = meshgen.lognormal(6, 3, NT)
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    assert fa.fem_pattern_value_path(p)["path"] == "two_pass"
    for variant in VARIANTS:
        v, b = fa.assemble(p, dev(node), dev(k), fa.FEM_F_SINPROD, None, variant)
        fa.get_error()
        rp, col, vo, so = oracle.assemble(2, node, elem, k)
        assert_close_scaled(host(v), vo, so)
        bo = oracle.rhs(2, node, elem, oracle.F_SINPROD)
        assert_close_scaled(host(b), bo, np.abs(bo) + 1e-300, what="rhs")
    slot = oracle.slots(2, N, elem, rp.astype(np.int64), col.astype(np.int64))
    w, r = meshgen.normal(3, meshgen.TAG_W, p.nnz), meshgen.normal(3, meshgen.TAG_R, N)
    gn = torch.empty((N, 2), dtype=torch.float64, device="cuda")
    gk = torch.empty(NT, dtype=torch.float64, device="cuda")
    fa.fem_assemble_backward(p, dev(node), dev(k), fa.FEM_F_SINPROD, None, dev(w), dev(r), gn, gk)
    fa.get_error()
    gno, gko, gnm, gkm = oracle.backward(2, node, elem, k, oracle.F_SINPROD, None, slot, w, r, with_scale=True)
    assert_close_scaled(host(gn), gno, gnm, tol=BWD_TOL, what="node gradient")
    assert_close_scaled(host(gk), gko, gkm, tol=BWD_TOL, what="k gradient")
    for call in (lambda: fa.fem_assemble_operator(p, dev(node), fa.FEM_OP_MASS, None),
                 lambda: fa.fem_apply_stiffness(p, dev(node), dev(k), dev(np.ones(N)))):
        with pytest.raises(fa.FemError) as e:
            call()
        assert e.value.code == fa.FEM_ERR_STATE


def test_qp_values_rhs():
    d, node, elem, k, _ = mesh_case("sq37p")
    rng = np.random.default_rng(5)
    fq = rng.normal(size=(elem.shape[0], 3))
    p = fa.Pattern(dev(elem), node.shape[0])
    b = torch.empty(node.shape[0], dtype=torch.float64, device="cuda")
    fa.fem_assemble_rhs(p, dev(node), fa.FEM_F_QPVALUES, dev(fq.ravel()), b, fa.FEM_DETERMINISTIC)
    bo = oracle.rhs(d, node, elem, oracle.F_QP, fq.ravel())
    bs = oracle.rhs(d, node, elem, oracle.F_QP, np.abs(fq).ravel())
    assert_close_scaled(host(b), bo, bs, what="rhs qp")
    d3, node3, elem3, _, _ = mesh_case("kuhn5")
    fq3 = rng.normal(size=(elem3.shape[0], 4))
    p3 = fa.Pattern(dev(elem3), node3.shape[0])
    b3 = torch.empty(node3.shape[0], dtype=torch.float64, device="cuda")
    fa.fem_assemble_rhs(p3, dev(node3), fa.FEM_F_QPVALUES, dev(fq3.ravel()), b3, fa.FEM_ATOMIC)
    assert_close_scaled(host(b3), oracle.rhs(3, node3, elem3, oracle.F_QP, fq3.ravel()),
                        oracle.rhs(3, node3, elem3, oracle.F_QP, np.abs(fq3).ravel()), what="rhs qp 3d")


def test_const_f_value_and_stiffness_only_calls():
    d, node, elem, k, _ = mesh_case("kuhn5")
    p = fa.Pattern(dev(elem), node.shape[0])
    val = torch.empty(p.nnz, dtype=torch.float64, device="cuda")
    fa.fem_assemble_stiffness(p, dev(node), dev(k), val, fa.FEM_DETERMINISTIC)
    _, _, vo, so = oracle.assemble(d, node, elem, k)
    assert_close_scaled(host(val), vo, so)
    b = torch.empty(p.N, dtype=torch.float64, device="cuda")
    fa.fem_assemble_rhs(p, dev(node), fa.FEM_F_CONST, dev(np.array([2.5])), b, fa.FEM_DETERMINISTIC)
    bo = oracle.rhs(d, node, elem, oracle.F_CONST, np.array([2.5]))
    assert_close_scaled(host(b), bo, np.abs(bo))
    assert abs(float(b.sum()) - 2.5) < 1e-12


def test_deterministic_variant_is_bitwise_reproducible():
    m = meshgen.square_mesh(200, 0.2, 3, permute=True)
    k = meshgen.lognormal(3, 3, m["elem"].shape[0])
    p = fa.Pattern(dev(m["elem"]), m["node"].shape[0])
    outs = [fa.assemble(p, dev(m["node"]), dev(k), fa.FEM_F_SINPROD, None, fa.FEM_DETERMINISTIC) for _ in range(3)]
    for v, b in outs[1:]:
        assert torch.equal(v, outs[0][0]) and torch.equal(b, outs[0][1])
    va, ba = fa.assemble(p, dev(m["node"]), dev(k), fa.FEM_F_SINPROD, None, fa.FEM_ATOMIC)
    _, _, vo, so = oracle.assemble(2, m["node"], m["elem"], k)
    assert_close_scaled(host(va), vo, so)
    assert_close_scaled(host(outs[0][0]), vo, so)


@pytest.mark.parametrize("case", ["sq37p", "kuhn5", "delaunay2", "delaunay3"])
def test_boundary_bit_exact(case):
    d, node, elem, _, _ = mesh_case(case)
    N = node.shape[0]
    p = fa.Pattern(dev(elem), N)
    isbd = torch.empty(N, dtype=torch.uint8, device="cuda")
    fa.fem_boundary_nodes(p, None, isbd)
    assert np.array_equal(host(isbd), oracle.boundary(d, N, elem))
    rng = np.random.default_rng(1)
    flag = (rng.uniform(size=elem.shape) < 0.2).astype(np.int8) * rng.integers(0, 4, size=elem.shape).astype(np.int8)
    fa.fem_boundary_nodes(p, dev(flag), isbd)
    assert np.array_equal(host(isbd), oracle.boundary(d, N, elem, flag))


@pytest.mark.parametrize("with_gd", [False, True])
@pytest.mark.parametrize("case", ["sq37p", "kuhn5", "delaunay2"])
def test_dirichlet_bit_exact(case, with_gd):
    d, node, elem, k, f_kind = mesh_case(case)
    N = node.shape[0]
    p = fa.Pattern(dev(elem), N)
    val, b = fa.assemble(p, dev(node), dev(k), f_kind, None, fa.FEM_DETERMINISTIC)
    isbd = torch.empty(N, dtype=torch.uint8, device="cuda")
    fa.fem_boundary_nodes(p, None, isbd)
    gD = np.cos(3 * node[:, 0]) + node[:, 1] if with_gd else None
    v0, b0 = host(val).copy(), host(b).copy()
    free = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    nf = fa.fem_apply_dirichlet(p, isbd, None if gD is None else dev(gD), val, b, free)
    vo, bo, fo = oracle.dirichlet(host(p.row_ptr).astype(np.int64), host(p.col_idx).astype(np.int64), v0, b0,
                                  host(isbd), gD)
    assert nf == fo.size
    assert np.array_equal(host(free)[:nf], fo)
    assert np.array_equal(host(val), vo)  # bit-exact
    assert np.array_equal(host(b), bo)


@pytest.mark.parametrize("f_kind", [fa.FEM_F_CONST, fa.FEM_F_SINPROD, fa.FEM_F_QPVALUES])
@pytest.mark.parametrize("case", ["sq37p", "kuhn5", "delaunay3"])
def test_backward_matches_oracle_adjoint(case, f_kind):
    d, node, elem, k, _ = mesh_case(case)
    N, NT = node.shape[0], elem.shape[0]
    p = fa.Pattern(dev(elem), N)
    rp, col = host(p.row_ptr).astype(np.int64), host(p.col_idx).astype(np.int64)
    slot = oracle.slots(d, N, elem, rp, col)
    w = meshgen.normal(1808, meshgen.TAG_W, p.nnz)
    r = meshgen.normal(1808, meshgen.TAG_R, N)
    farg = meshgen.normal(7, 9, NT * (d + 1)) if f_kind == fa.FEM_F_QPVALUES else None
    # per-entry scale: the same adjoint with every term replaced by its magnitude
    gno, gko, gnm, gkm = oracle.backward(d, node, elem, k, f_kind, farg, slot, w, r, with_scale=True)
    # tile order (the pattern has a tile plan), then the caller's order (no plan)
    for _ in range(2):
        gn = torch.empty((N, d), dtype=torch.float64, device="cuda")
        gk = torch.empty(NT, dtype=torch.float64, device="cuda")
        fa.fem_assemble_backward(p, dev(node), dev(k), f_kind, None if farg is None else dev(farg), dev(w), dev(r),
                                 gn, gk)
        fa.get_error()
        assert_close_scaled(host(gn), gno, gnm, tol=BWD_TOL, what="node gradient")
        assert_close_scaled(host(gk), gko, gkm, tol=BWD_TOL, what="k gradient")
        fa.fem_pattern_force_path(p, fa.FEM_PATH_TWO_PASS)


@pytest.mark.parametrize("part", ["w", "r"])
@pytest.mark.parametrize("f_kind", [fa.FEM_F_CONST, fa.FEM_F_SINPROD, fa.FEM_F_QPVALUES])
@pytest.mark.parametrize("case", ["sq37p", "kuhn5", "delaunay3"])
def test_backward_one_loss_part_matches_oracle_adjoint(case, f_kind, part):
    """L = w.A alone, or L = r.b alone: each part of the adjoint on its own scale (the load part is far
    smaller than the stiffness part when both are present, so this is where the quadrature weights of
    the load term show their precision)."""
    d, node, elem, k, _ = mesh_case(case)
    N, NT = node.shape[0], elem.shape[0]
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    rp, col = host(p.row_ptr).astype(np.int64), host(p.col_idx).astype(np.int64)
    slot = oracle.slots(d, N, elem, rp, col)
    w = meshgen.normal(1808, meshgen.TAG_W, p.nnz) if part == "w" else None
    r = meshgen.normal(1808, meshgen.TAG_R, N) if part == "r" else None
    farg = meshgen.normal(7, 9, NT * (d + 1)) if f_kind == fa.FEM_F_QPVALUES else None
    gno, gko, gnm, gkm = oracle.backward(d, node, elem, k, f_kind, farg, slot, w, r, with_scale=True)
    gn = torch.empty((N, d), dtype=torch.float64, device="cuda")
    gk = torch.empty(NT, dtype=torch.float64, device="cuda")
    fa.fem_assemble_backward(p, dev(node), dev(k), f_kind, None if farg is None else dev(farg),
                             None if w is None else dev(w), None if r is None else dev(r), gn, gk)
    fa.get_error()
    assert_close_scaled(host(gn), gno, gnm, tol=BWD_TOL, what="node gradient")
    assert_close_scaled(host(gk), gko, gkm, tol=BWD_TOL, what="k gradient")


def test_backward_central_fd_on_gpu():
    """Gradients of L = w.A + r.b from the GPU backward vs central differences of the GPU forward."""
    m = meshgen.kuhn_mesh(3, 0.1, 21)
    node, elem = m["node"], m["elem"]
    N, NT = node.shape[0], elem.shape[0]
    k = meshgen.lognormal(21, 3, NT)
    p = fa.Pattern(dev(elem), N)
    w = dev(meshgen.normal(22, 4, p.nnz))
    r = dev(meshgen.normal(22, 5, N))

    def L(x, kk):
        v, b = fa.assemble(p, dev(x), dev(kk), fa.FEM_F_SINPROD, None, fa.FEM_DETERMINISTIC)
        return float((w * v).sum() + (r * b).sum())

    gn = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    gk = torch.empty(NT, dtype=torch.float64, device="cuda")
    fa.fem_assemble_backward(p, dev(node), dev(k), fa.FEM_F_SINPROD, None, w, r, gn, gk)
    gn, gk = host(gn), host(gk)
    rng = np.random.default_rng(0)
    eps = 1e-6
    for v in rng.choice(N, 40, replace=False):
        for c in range(3):
            xp, xm = node.copy(), node.copy()
            xp[v, c] += eps
            xm[v, c] -= eps
            fd = (L(xp, k) - L(xm, k)) / (2 * eps)
            assert abs(fd - gn[v, c]) <= 1e-6 * max(1.0, abs(gn[v, c]))
    for t in rng.choice(NT, 40, replace=False):
        kp, km = k.copy(), k.copy()
        kp[t] += eps
        km[t] -= eps
        fd = (L(node, kp) - L(node, km)) / (2 * eps)
        assert abs(fd - gk[t]) <= 1e-6 * max(1.0, abs(gk[t]))


def test_autograd_function():
    d, node, elem, k, _ = mesh_case("kuhn5")
    p = fa.Pattern(dev(elem), node.shape[0])
    x = dev(node).requires_grad_(True)
    kk = dev(k).requires_grad_(True)
    val, b = fa.FemAssemble.apply(x, kk, p, fa.FEM_F_SINPROD, None)
    w = torch.randn_like(val)
    r = torch.randn_like(b)
    loss = (w * val).sum() + (r * b).sum()
    gx, gk = torch.autograd.grad(loss, [x, kk])
    gn2 = torch.empty_like(gx)
    gk2 = torch.empty_like(gk)
    fa.fem_assemble_backward(p, dev(node), dev(k), fa.FEM_F_SINPROD, None, w, r, gn2, gk2)
    assert torch.equal(gx, gn2) and torch.equal(gk, gk2)


def test_batched_matches_per_mesh_oracle():
    sides = [3, 5, 8, 2, 13, 1]
    meshes = [meshgen.square_mesh(s, 0.2, 100 + i) for i, s in enumerate(sides)]
    ks = [meshgen.lognormal(100 + i, 3, m["elem"].shape[0]) for i, m in enumerate(meshes)]
    elem_cat = np.concatenate([m["elem"] for m in meshes])
    node_cat = np.concatenate([m["node"] for m in meshes])
    k_cat = np.concatenate(ks)
    bt = fa.Batch(2, [m["node"].shape[0] for m in meshes], [m["elem"].shape[0] for m in meshes], dev(elem_cat))
    bt.set_locality(dev(node_cat))
    val = torch.empty(bt.nnz_off[-1], dtype=torch.float64, device="cuda")
    b = torch.empty(bt.node_off[-1], dtype=torch.float64, device="cuda")
    bt.assemble(dev(node_cat), dev(k_cat), fa.FEM_F_SINPROD, None, val, b, fa.FEM_DETERMINISTIC)
    fa.get_error()
    v, bb = host(val), host(b)
    for i, m in enumerate(meshes):
        rp, col, vo, so = oracle.assemble(2, m["node"], m["elem"], ks[i])
        assert np.array_equal(host(bt.pattern.col_idx)[bt.nnz_off[i]:bt.nnz_off[i + 1]] - bt.node_off[i], col)
        assert_close_scaled(v[bt.nnz_off[i]:bt.nnz_off[i + 1]], vo, so)
        bo = oracle.rhs(2, m["node"], m["elem"], oracle.F_SINPROD)
        assert_close_scaled(bb[bt.node_off[i]:bt.node_off[i + 1]], bo, np.abs(bo) + 1e-30)
    # the batch runs as one launch: the fused tile kernel or the persistent owner-computes kernel
    path = fa.fem_pattern_value_path(bt.pattern)["path"]
    assert path == "tiles_fused" or (path == "blocked" and fa.fem_pattern_launch_shape(bt.pattern)["persistent"])
    n0 = fa.launch_count()
    bt.assemble(dev(node_cat), dev(k_cat), fa.FEM_F_SINPROD, None, val, b, fa.FEM_DETERMINISTIC)
    assert fa.launch_count() - n0 == 1
    # graph replay gives the same bits
    val2, b2 = torch.empty_like(val), torch.empty_like(b)
    n0 = fa.launch_count()
    for _ in range(2):
        bt.assemble(dev(node_cat), dev(k_cat), fa.FEM_F_SINPROD, None, val2, b2, fa.FEM_DETERMINISTIC, graph=True)
    torch.cuda.synchronize()
    assert fa.launch_count() > n0
    assert torch.equal(val, val2) and torch.equal(b, b2)
    # and so does the other one-launch form
    other = fa.FEM_PATH_BLOCKED if path == "tiles_fused" else fa.FEM_PATH_TILES_FUSED
    fa.fem_pattern_force_path(bt.pattern, other, 128)
    if other == fa.FEM_PATH_BLOCKED:
        shp = fa.fem_pattern_launch_shape(bt.pattern)
        fa.fem_pattern_force_launch(bt.pattern, shp["threads"], shp["ctas_per_sm"], True)
    val3, b3 = torch.empty_like(val), torch.empty_like(b)
    bt.assemble(dev(node_cat), dev(k_cat), fa.FEM_F_SINPROD, None, val3, b3, fa.FEM_DETERMINISTIC)
    fa.get_error()
    assert torch.equal(val, val3) and torch.equal(b, b3)


def test_edge_cases():
    # empty mesh
    p = fa.Pattern(torch.zeros((0, 3), dtype=torch.int32, device="cuda"), 5)
    assert p.nnz == 0 and host(p.row_ptr).tolist() == [0] * 6
    val, b = fa.assemble(p, dev(np.zeros((5, 2))))
    assert b.abs().sum().item() == 0.0
    # one element
    node = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    p1 = fa.Pattern(dev(np.array([[0, 1, 2]], np.int32)), 3)
    v1, b1 = fa.assemble(p1, dev(node))
    assert host(v1).tolist() == [1.0, -0.5, -0.5, -0.5, 0.5, 0.0, -0.5, 0.0, 0.5]
    assert np.allclose(host(b1), [0.5 / 3] * 3, rtol=1e-14, atol=0)
    # bad vertex id and repeated vertex are rejected at pattern build
    with pytest.raises(fa.FemError) as e:
        fa.Pattern(dev(np.array([[0, 1, 7]], np.int32)), 3)
    assert e.value.code == fa.FEM_ERR_INDEX
    with pytest.raises(fa.FemError) as e:
        fa.Pattern(dev(np.array([[0, 1, 1]], np.int32)), 3)
    assert e.value.code == fa.FEM_ERR_INDEX
    with pytest.raises(fa.FemError) as e:
        fa.Pattern(dev(np.array([[0, 1, -1]], np.int32)), 3)
    assert e.value.code == fa.FEM_ERR_INDEX
    # degenerate element is reported through the device error word, and the word is then cleared
    flat = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0]])
    for variant in VARIANTS:
        fa.assemble(p1, dev(flat), variant=variant)
        with pytest.raises(fa.FemError) as e:
            fa.get_error()
        assert e.value.code == fa.FEM_ERR_DEGENERATE
        fa.get_error()
    # inverted tetrahedron (signed volume < 0) is degenerate in 3-D
    m = meshgen.kuhn_mesh(1)
    e3 = m["elem"].copy()
    e3[0] = e3[0][[1, 0, 2, 3]]
    p3 = fa.Pattern(dev(e3), m["node"].shape[0])
    fa.assemble(p3, dev(m["node"]))
    with pytest.raises(fa.FemError):
        fa.get_error()


# ---- full-size workloads, in the launch configuration the benchmark times -------------------------

@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("cfg", ["c2", "c3"])
def test_full_size_sampled_rows(cfg, variant):
    m = meshgen.make_config(cfg)
    d = m["d"]
    node, elem, k = m["node"], m["elem"], m["coef"]
    N, NT = node.shape[0], elem.shape[0]
    f_kind = oracle.F_SINPROD if m["f"] == "sinprod" else oracle.F_CONST
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    n = m["n"]
    exp_nnz = N + 2 * (3 * n * n + 2 * n) if d == 2 else N + 2 * (3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3)
    assert p.nnz == exp_nnz
    val, b = fa.assemble(p, dev(node), dev(k), f_kind, None, variant)
    fa.get_error()
    rows = sample_rows(N, 600, 11)
    rp_o, col_o, v_o, s_o = oracle.assemble(d, node, elem, k, rows=rows)
    rp, col, v = host(p.row_ptr), host(p.col_idx), host(val)
    for r in rows:
        seg = slice(rp[r], rp[r + 1])
        oseg = slice(rp_o[r], rp_o[r + 1])
        assert np.array_equal(col[seg], col_o[oseg])
        assert_close_scaled(v[seg], v_o[oseg], s_o[oseg])
    b_o = oracle.rhs(d, node, elem, f_kind, rows=rows)
    bh = host(b)
    assert_close_scaled(bh[rows], b_o[rows], np.abs(b_o[rows]) + 1e-30, what="rhs rows")
    # zero row sums everywhere (constants are in the kernel), relative to the row's magnitude
    rowid = torch.repeat_interleave(torch.arange(N, device="cuda"), (p.row_ptr[1:] - p.row_ptr[:-1]).long())
    rs = torch.zeros(N, dtype=torch.float64, device="cuda").index_add_(0, rowid, val)
    ra = torch.zeros(N, dtype=torch.float64, device="cuda").index_add_(0, rowid, val.abs())
    assert bool((rs.abs() <= 1e-12 * ra).all())
    # symmetry through the slot map, sampled elements
    ts = torch.as_tensor(np.random.default_rng(3).choice(NT, 20000, replace=False), device="cuda")
    sl = host(p.slot.view((d + 1) ** 2, NT)[:, ts]).T.reshape(-1, d + 1, d + 1)
    a = v[sl]
    assert np.all(np.abs(a - np.transpose(a, (0, 2, 1))) <= 1e-13 * np.abs(a).max(axis=(1, 2), keepdims=True))
    # whole-boundary mask equals the generator's geometric one
    isbd = torch.empty(N, dtype=torch.uint8, device="cuda")
    fa.fem_boundary_nodes(p, None, isbd)
    assert np.array_equal(host(isbd), m["is_bd"])


def test_full_size_batch_sampled_meshes():
    """The 256-mesh batch (n ~ U{16..512}, 48.2 M triangles) in the benchmark's launch form: one launch
    replayed from a CUDA graph. Sampled meshes (the smallest, the largest and three more) against the
    oracle, value by value; every mesh's rows sum to zero."""
    c4 = meshgen.make_config("c4")
    ms_ = c4["meshes"]
    elem_cat = np.concatenate([x["elem"] for x in ms_])
    node_cat = np.concatenate([x["node"] for x in ms_])
    k_cat = np.concatenate([x["coef"] for x in ms_])
    bt = fa.Batch(2, [x["node"].shape[0] for x in ms_], [x["elem"].shape[0] for x in ms_], dev(elem_cat))
    bt.set_locality(dev(node_cat))
    val = torch.empty(bt.nnz_off[-1], dtype=torch.float64, device="cuda")
    b = torch.empty(bt.node_off[-1], dtype=torch.float64, device="cuda")
    nd, kd = dev(node_cat), dev(k_cat)
    for _ in range(2):
        bt.assemble(nd, kd, fa.FEM_F_SINPROD, None, val, b, fa.FEM_DETERMINISTIC, graph=True)
    torch.cuda.synchronize()
    fa.get_error()
    v, bb = host(val), host(b)
    sides = c4["sides"]
    pick = sorted({int(np.argmin(sides)), int(np.argmax(sides))} |
                  set(np.random.default_rng(5).choice(len(ms_), 3, replace=False).tolist()))
    for i in pick:
        m = ms_[i]
        rp, col, vo, so = oracle.assemble(2, m["node"], m["elem"], m["coef"])
        assert np.array_equal(host(bt.pattern.col_idx)[bt.nnz_off[i]:bt.nnz_off[i + 1]] - bt.node_off[i], col)
        assert_close_scaled(v[bt.nnz_off[i]:bt.nnz_off[i + 1]], vo, so)
        bo = oracle.rhs(2, m["node"], m["elem"], oracle.F_SINPROD)
        assert_close_scaled(bb[bt.node_off[i]:bt.node_off[i + 1]], bo, np.abs(bo) + 1e-30, what="rhs")
    rp = bt.pattern.row_ptr
    Nt = bt.node_off[-1]
    rowid = torch.repeat_interleave(torch.arange(Nt, device="cuda"), (rp[1:] - rp[:-1]).long())
    rs = torch.zeros(Nt, dtype=torch.float64, device="cuda").index_add_(0, rowid, val)
    ra = torch.zeros(Nt, dtype=torch.float64, device="cuda").index_add_(0, rowid, val.abs())
    assert bool((rs.abs() <= 1e-12 * ra).all())


def test_full_size_backward_matches_oracle_adjoint():
    """The 64^3 Kuhn mesh (1.57 M tetrahedra), L = w.A + r.b with the benchmark's seeded weights and the
    sine-product load: the GPU backward (tile order, as the benchmark runs it) against the oracle's
    adjoint over the whole mesh, every node and element gradient."""
    m = meshgen.make_config("c5")
    node, elem, k = m["node"], m["elem"], m["coef"]
    N, NT = node.shape[0], elem.shape[0]
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    rp, col = host(p.row_ptr).astype(np.int64), host(p.col_idx).astype(np.int64)
    slot = oracle.slots(3, N, elem, rp, col)
    w = meshgen.normal(m["loss_seed"], meshgen.TAG_W, p.nnz)
    r = meshgen.normal(m["loss_seed"], meshgen.TAG_R, N)
    gn = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    gk = torch.empty(NT, dtype=torch.float64, device="cuda")
    val, b = fa.assemble(p, dev(node), dev(k), fa.FEM_F_SINPROD)
    fa.fem_assemble_backward(p, dev(node), dev(k), fa.FEM_F_SINPROD, None, dev(w), dev(r), gn, gk)
    fa.get_error()
    gno, gko, gnm, gkm = oracle.backward(3, node, elem, k, oracle.F_SINPROD, None, slot, w, r, with_scale=True)
    assert_close_scaled(host(gn), gno, gnm, tol=BWD_TOL, what="node gradient")
    assert_close_scaled(host(gk), gko, gkm, tol=BWD_TOL, what="k gradient")


@pytest.mark.parametrize("part", ["w", "r"])
def test_full_size_backward_one_part_with_constant_f(part):
    """The 64^3 mesh with one loss part and f = 1: every gradient against the oracle adjoint. Here a
    gradient's exact value is often 0 (normals of faces on the boundary planes have exact zero
    components) and the float-float result a residue of the terms' roundings, far below the float-float
    range; such a residue is no loss against the terms the error is measured by, and the range check,
    made on the terms' magnitudes, must not report it."""
    m = meshgen.make_config("c5")
    node, elem, k = m["node"], m["elem"], m["coef"]
    N, NT = node.shape[0], elem.shape[0]
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    rp, col = host(p.row_ptr).astype(np.int64), host(p.col_idx).astype(np.int64)
    slot = oracle.slots(3, N, elem, rp, col)
    w = meshgen.normal(m["loss_seed"], meshgen.TAG_W, p.nnz) if part == "w" else None
    r = meshgen.normal(m["loss_seed"], meshgen.TAG_R, N) if part == "r" else None
    gn = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    gk = torch.empty(NT, dtype=torch.float64, device="cuda")
    fa.fem_assemble_backward(p, dev(node), dev(k), fa.FEM_F_CONST, None, None if w is None else dev(w),
                             None if r is None else dev(r), gn, gk)
    fa.get_error()
    gno, gko, gnm, gkm = oracle.backward(3, node, elem, k, oracle.F_CONST, None, slot, w, r, with_scale=True)
    assert_close_scaled(host(gn), gno, gnm, tol=BWD_TOL, what="node gradient")
    assert_close_scaled(host(gk), gko, gkm, tol=BWD_TOL, what="k gradient")


@pytest.mark.parametrize("d", [2, 3])
def test_backward_reports_loss_weights_beyond_the_range(d):
    """Loss weights of 1e-40 put the adjoint's terms below the float-float range: FEM_ERR_RANGE, for the
    stiffness part (w) and the load part (r) alike; weights of 1 on the same pattern then pass."""
    _, node, elem, k, _ = mesh_case("sq37p" if d == 2 else "kuhn5")
    N, NT = node.shape[0], elem.shape[0]
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    kd = dev(k if k is not None else np.ones(NT))
    gn = torch.empty((N, d), dtype=torch.float64, device="cuda")
    gk = torch.empty(NT, dtype=torch.float64, device="cuda")
    for w, r in ((np.full(p.nnz, 1e-40), None), (None, np.full(N, 1e-40))):
        fa.fem_assemble_backward(p, dev(node), kd, fa.FEM_F_SINPROD, None, None if w is None else dev(w),
                                 None if r is None else dev(r), gn, gk)
        with pytest.raises(fa.FemError) as err:
            fa.get_error()
        assert err.value.code == fa.FEM_ERR_RANGE
    fa.fem_assemble_backward(p, dev(node), kd, fa.FEM_F_SINPROD, None, dev(np.ones(p.nnz)), dev(np.ones(N)), gn, gk)
    fa.get_error()


# ---- Neumann / Robin sides and the pure-Neumann fixes ------------------------------------------------

@pytest.mark.parametrize("d", [2, 3])
def test_neumann_robin_terms_bit_exact(d):
    """Side terms on top of an assembled system: the same val and b in, the same bits out as the oracle
    (per-row order and operations are fixed on both sides)."""
    m = meshgen.square_mesh(9, 0.2, 51, True) if d == 2 else meshgen.kuhn_mesh(3, 0.1, 51)
    node, elem = m["node"], m["elem"]
    N, NT = node.shape[0], elem.shape[0]
    flags = meshgen.side_flags(m, {"x0": 2, "x1": 2, "y1": 3, "y0": 1, "z1": 3, "z0": 2})
    k = meshgen.lognormal(51, 3, NT)
    p = fa.Pattern(dev(elem), N)
    val, b = fa.assemble(p, dev(node), dev(k), fa.FEM_F_SINPROD, None, fa.FEM_DETERMINISTIC)
    v0, b0 = host(val), host(b)
    rp, col = host(p.row_ptr).astype(np.int64), host(p.col_idx).astype(np.int64)
    g = meshgen.normal(52, 9, NT * (d + 1)).reshape(NT, d + 1)
    for g_side, g_const in ((g, 0.0), (None, 1.75)):
        v, bb = val.clone(), b.clone()
        fa.fem_boundary_terms(p, dev(node), dev(flags), None if g_side is None else dev(g_side), g_const, 0.7, v, bb)
        fa.get_error()
        vo, bo = oracle.boundary_terms(d, node, elem, flags, rp, col, v0, b0, g_side=g_side, g_const=g_const, alpha=0.7)
        assert np.array_equal(host(v), vo) and np.array_equal(host(bb), bo)
        assert not np.array_equal(vo, v0) and not np.array_equal(bo, b0)
    # load only, matrix only
    bb = b.clone()
    fa.fem_boundary_terms(p, dev(node), dev(flags), None, 1.0, 0.7, None, bb)
    _, bo = oracle.boundary_terms(d, node, elem, flags, rp, col, v0, b0, g_const=1.0, alpha=0.7)
    assert np.array_equal(host(bb), bo)
    pts = torch.empty((NT, d + 1, d), dtype=torch.float64, device="cuda")
    fa.fem_side_points(p, dev(node), pts)
    assert np.array_equal(host(pts), oracle.side_points(d, node, elem))


@pytest.mark.parametrize("d", [2, 3])
def test_mean_shift_and_zero_average_match_oracle(d):
    m = meshgen.square_mesh(40, 0.2, 53, True) if d == 2 else meshgen.kuhn_mesh(8, 0.1, 53)
    node, elem = m["node"], m["elem"]
    N = node.shape[0]
    p = fa.Pattern(dev(elem), N)
    rng = np.random.default_rng(53)
    x = rng.normal(size=N) + 2.0
    xd = dev(x)
    fa.fem_mean_shift(xd)
    xo = oracle.mean_shift(x)
    assert np.all(np.abs(host(xd) - xo) <= 1e-13 * np.abs(x).max())
    assert abs(float(xd.sum())) <= 1e-11
    u = rng.normal(size=N)
    ud = dev(u)
    c = torch.empty(1, dtype=torch.float64, device="cuda")
    fa.fem_zero_average(p, dev(node), ud, c)
    uo, co = oracle.zero_average(d, node, elem, u)
    assert abs(float(c.item()) - co) <= 1e-13 * np.abs(u).max()
    assert np.all(np.abs(host(ud) - uo) <= 1e-13 * np.abs(u).max())
    # deterministic: the same bits again
    ud2 = dev(u)
    fa.fem_zero_average(p, dev(node), ud2)
    assert torch.equal(ud, ud2)
    # empty input is a no-op
    fa.fem_mean_shift(torch.empty(0, dtype=torch.float64, device="cuda"))
    fa.get_error()


# ---- other operators: mass matrix and -div(K grad u) --------------------------------------------------

@pytest.mark.parametrize("case", ["sq37p", "kuhn5", "delaunay2", "delaunay3"])
def test_mass_and_anisotropic_operators_match_oracle(case):
    d, node, elem, k, _ = mesh_case(case)
    N, NT = node.shape[0], elem.shape[0]
    p = fa.Pattern(dev(elem), N)
    rng = np.random.default_rng(71)
    c = meshgen.lognormal(71, 3, NT)
    nk = d * (d + 1) // 2
    # SPD tensors: diagonal in [0.5, 2], off-diagonal up to 0.3
    K = np.zeros((NT, nk))
    diag_pos = [0, 2] if d == 2 else [0, 3, 5]
    off_pos = [1] if d == 2 else [1, 2, 4]
    K[:, diag_pos] = rng.uniform(0.5, 2.0, size=(NT, d))
    K[:, off_pos] = rng.uniform(-0.3, 0.3, size=(NT, len(off_pos)))
    for op, coef in ((fa.FEM_OP_MASS, None), (fa.FEM_OP_MASS, c), (fa.FEM_OP_ANISO, K)):
        v = fa.fem_assemble_operator(p, dev(node), op, None if coef is None else dev(coef))
        fa.get_error()
        rp, col, vo, so = oracle.operator(d, node, elem, op, coef)
        assert np.array_equal(host(p.col_idx), col)
        assert_close_scaled(host(v), vo, so, what="operator %d" % op)
        # deterministic and the same bits in the fused form
        v2 = fa.fem_assemble_operator(p, dev(node), op, None if coef is None else dev(coef))
        assert torch.equal(v, v2)
        fa.fem_pattern_force_path(p, fa.FEM_PATH_TILES_FUSED, 128)
        v3 = fa.fem_assemble_operator(p, dev(node), op, None if coef is None else dev(coef))
        fa.fem_pattern_force_path(p, fa.FEM_PATH_TILES, 128)
        assert torch.equal(v, v3)
    # the stiffness operator is fem_assemble_stiffness
    vs = fa.fem_assemble_operator(p, dev(node), fa.FEM_OP_STIFFNESS, dev(k))
    vref = torch.empty_like(vs)
    fa.fem_assemble_stiffness(p, dev(node), dev(k), vref, fa.FEM_DETERMINISTIC)
    assert torch.equal(vs, vref)
    with pytest.raises(fa.FemError):
        fa.fem_assemble_operator(p, dev(node), fa.FEM_OP_ANISO, None)


# ---- load vector with rules of any order ------------------------------------------------------------

@pytest.mark.parametrize("case", ["sq37p", "kuhn5", "delaunay2", "delaunay3"])
def test_rule_load_vector_matches_oracle(case):
    d, node, elem, k, _ = mesh_case(case)
    N, NT = node.shape[0], elem.shape[0]
    p = fa.Pattern(dev(elem), N)
    for n in (1, 3, 5):
        bary, w = fa.fem_quad_rule(d, n)
        pts = fa.fem_rule_points(p, dev(node), n)
        ref_pts = np.einsum("qi,tim->tqm", bary, node[elem])
        assert np.allclose(host(pts), ref_pts, rtol=0, atol=1e-15)
        vals = np.cos(3.0 * ref_pts[..., 0]) + ref_pts[..., 1]
        for fk, farg, sarg in ((fa.FEM_F_SINPROD, None, None), (fa.FEM_F_CONST, np.array([1.5]), None),
                               (fa.FEM_F_QPVALUES, vals.ravel(), np.abs(vals).ravel())):
            b = fa.fem_assemble_rhs_rule(p, dev(node), n, fk, None if farg is None else dev(farg))
            fa.get_error()
            ok = {fa.FEM_F_SINPROD: oracle.F_SINPROD, fa.FEM_F_CONST: oracle.F_CONST, fa.FEM_F_QPVALUES: oracle.F_QP}[fk]
            bo = oracle.rhs_rule(d, node, elem, bary, w, ok, farg)
            scale = np.abs(oracle.rhs_rule(d, node, elem, bary, w, ok, sarg)) if sarg is not None else np.abs(bo)
            assert_close_scaled(host(b), bo, scale + 1e-300, what="rule rhs n=%d f=%d" % (n, fk))
            b2 = fa.fem_assemble_rhs_rule(p, dev(node), n, fk, None if farg is None else dev(farg))
            assert torch.equal(b, b2)


# ---- matrix-free operator ---------------------------------------------------------------------------

def sp_csr(rp, col, val, n):
    """Row-by-row product helper: a callable CSR matrix (numpy only)."""
    rp, col, val = np.asarray(rp), np.asarray(col), np.asarray(val)

    class _M:
        def __matmul__(self, x):
            out = np.zeros(rp.size - 1)
            for r in range(rp.size - 1):
                seg = slice(rp[r], rp[r + 1])
                out[r] = np.dot(val[seg], x[col[seg]])
            return out
    return _M()

@pytest.mark.parametrize("case", ["sq37p", "kuhn5", "delaunay2", "delaunay3"])
def test_matrix_free_apply_matches_assembled_operator(case):
    """y = A u without forming A equals the oracle's assembled A times u (within the scale |A| |u|), for
    the plain and the Dirichlet-eliminated operator; the same bits on every call."""
    d, node, elem, k, _ = mesh_case(case)
    N = node.shape[0]
    p = fa.Pattern(dev(elem), N)
    rng = np.random.default_rng(91)
    u = rng.normal(size=N)
    rp, col, vo, so = oracle.assemble(d, node, elem, k)
    isbd = oracle.boundary(d, N, elem)
    for bd in (None, isbd):
        y = fa.fem_apply_stiffness(p, dev(node), dev(k), dev(u), None if bd is None else dev(bd))
        fa.get_error()
        if bd is None:
            A = sp_csr(rp, col, vo, N)
            yo = A @ u
        else:
            v2, _, _ = oracle.dirichlet(rp, col, vo, np.zeros(N), bd)
            yo = sp_csr(rp, col, v2, N) @ u
        scale = sp_csr(rp, col, np.abs(vo) + so, N) @ np.abs(u)
        if bd is not None:
            scale = np.where(bd == 1, np.abs(u), scale)
        assert_close_scaled(host(y), yo, scale, what="A u")
        y2 = fa.fem_apply_stiffness(p, dev(node), dev(k), dev(u), None if bd is None else dev(bd))
        assert torch.equal(y, y2)
    # constants are in the kernel of A
    y1 = fa.fem_apply_stiffness(p, dev(node), dev(k), dev(np.full(N, 3.0)))
    assert float(y1.abs().max()) <= 1e-12 * float(np.abs(vo).max()) * 3.0


@pytest.mark.parametrize("case", ["sq37p", "delaunay3"])
def test_host_steps_match_device_assembly(case):
    """fem_assemble_host: several pipelined steps from and to host memory (pinned and pageable, with and
    without k, with and without the load vector) give the bits of fem_assemble on device arrays, and
    match the oracle."""
    d, node, elem, k, _ = mesh_case(case)
    N, NT = node.shape[0], elem.shape[0]
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    rng = np.random.default_rng(77)
    steps = 5
    nodes = [node * (1.0 + 0.1 * i) + 0.01 * i for i in range(steps)]  # affine copies: valid meshes
    ks = [rng.lognormal(size=NT) if i != 1 else None for i in range(steps)]
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()
    node_h = [pin(x) if i != 2 else torch.as_tensor(np.ascontiguousarray(x)) for i, x in enumerate(nodes)]
    k_h = [None if x is None else pin(x) for x in ks]
    val_h = [torch.zeros(p.nnz, dtype=torch.float64).pin_memory() for _ in range(steps)]
    b_h = [torch.zeros(N, dtype=torch.float64).pin_memory() if i != 3 else torch.zeros(N, dtype=torch.float64)
           for i in range(steps)]
    fa.fem_assemble_host(p, node_h, k_h, fa.FEM_F_SINPROD, None, val_h, b_h)
    fa.get_error()
    for i in range(steps):
        v, b = fa.assemble(p, dev(nodes[i]), None if ks[i] is None else dev(ks[i]), fa.FEM_F_SINPROD)
        assert torch.equal(val_h[i], v.cpu()) and torch.equal(b_h[i], b.cpu()), i
        _, _, vo, so = oracle.assemble(d, nodes[i], elem, ks[i])
        assert_close_scaled(val_h[i].numpy(), vo, so)
    # outputs left out, one step, and no steps
    val1 = [torch.zeros(p.nnz, dtype=torch.float64).pin_memory()]
    fa.fem_assemble_host(p, node_h[:1], k_h[:1], fa.FEM_F_SINPROD, None, val1, None)
    assert torch.equal(val1[0], val_h[0])
    fa.fem_assemble_host(p, [], None, fa.FEM_F_SINPROD, None, None, None)


@pytest.mark.parametrize("case", ["sq37p", "kuhn5"])
def test_assemble_system_one_call(case):
    """assemble_system: pattern, values, load and Dirichlet elimination in one call; the same bits as the
    calls it is made of, and the eliminated system of the oracle (bit-exact rows, values within 1e-12)."""
    d, node, elem, k, _ = mesh_case(case)
    N = node.shape[0]
    gD = np.cos(3 * node[:, 0]) + node[:, 1]
    rp, col, val, b = fa.assemble_system(dev(node), dev(elem), dev(k), fa.FEM_F_SINPROD, None,
                                         dirichlet=True, gD=dev(gD))
    fa.get_error()
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    v2, b2 = fa.assemble(p, dev(node), dev(k), fa.FEM_F_SINPROD)
    isbd = torch.empty(N, dtype=torch.uint8, device="cuda")
    fa.fem_boundary_nodes(p, None, isbd)
    fa.fem_apply_dirichlet(p, isbd, dev(gD), v2, b2, want_count=False)
    assert torch.equal(rp, p.row_ptr) and torch.equal(col, p.col_idx)
    assert torch.equal(val, v2) and torch.equal(b, b2)
    rpo, colo, vo, so = oracle.assemble(d, node, elem, k)
    bo = oracle.rhs(d, node, elem, oracle.F_SINPROD)
    vo2, bo2, _ = oracle.dirichlet(rpo, colo, vo, bo, oracle.boundary(d, N, elem), gD)
    assert np.array_equal(host(rp), rpo) and np.array_equal(host(col), colo)
    assert_close_scaled(host(val), vo2, so + (vo2 == 1.0))
    A, bb = fa.assemble_system(dev(node), dev(elem), dev(k), fa.FEM_F_SINPROD, None, sparse=True)
    assert A.layout == torch.sparse_csr and torch.equal(A.values(), fa.assemble(p, dev(node), dev(k), fa.FEM_F_SINPROD)[0])


@pytest.mark.parametrize("d", [2, 3])
def test_gpu_system_solves_poisson_at_second_order(d):
    """The GPU's eliminated system (assemble_system with Dirichlet rows), solved on the host: the nodal
    error against the exact solution f / (d pi^2) of -Laplace u = sin-product falls by about 4 per
    halving of h, as the oracle's does."""
    sp = pytest.importorskip("scipy.sparse")
    spla = pytest.importorskip("scipy.sparse.linalg")
    errs = []
    for n in ((8, 16, 32) if d == 2 else (4, 8, 16)):
        m = meshgen.square_mesh(n) if d == 2 else meshgen.kuhn_mesh(n)
        node, elem = m["node"], m["elem"]
        N = node.shape[0]
        rp, col, val, b = fa.assemble_system(dev(node), dev(elem), None, fa.FEM_F_SINPROD, dirichlet=True)
        fa.get_error()
        A = sp.csr_matrix((host(val), host(col), host(rp)), shape=(N, N))
        u = spla.spsolve(A.tocsc(), host(b))
        errs.append(float(np.abs(u - np.prod(np.sin(np.pi * node), axis=1) / (d * np.pi ** 2)).max()))
    rates = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.5 < r < 4.5 for r in rates), (errs, rates)


# ---- reduced solve by matrix-free conjugate gradients (Sec. 3.3) ----------------------------------------

def _cg_case(d, n, seed):
    m = meshgen.square_mesh(n, 0.2, seed, permute=True) if d == 2 else meshgen.kuhn_mesh(n, 0.1, seed)
    node, elem = m["node"], m["elem"]
    k = meshgen.lognormal(seed, meshgen.TAG_COEF, elem.shape[0])
    return node, elem, k


@pytest.mark.parametrize("d", [2, 3])
def test_cg_matches_the_direct_reduced_solve(d):
    """fem_cg_solve (matrix-free operator, nonzero g_D, lognormal k, sine-product load from the GPU)
    against the oracle's direct solve of the same reduced system: boundary values exact, free values
    within the CG tolerance; a second solve gives the same bits and iteration count."""
    node, elem, k = _cg_case(d, 24 if d == 2 else 6, 91 + d)
    N = node.shape[0]
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    val, b = fa.assemble(p, dev(node), dev(k), fa.FEM_F_SINPROD)
    fa.get_error()
    isbd = torch.empty(N, dtype=torch.uint8, device="cuda")
    fa.fem_boundary_nodes(p, None, isbd)
    gD = 0.5 + node @ np.arange(1.0, d + 1.0)
    u, it, rel = fa.fem_cg_solve(p, dev(node), dev(k), isbd, b, dev(gD), rtol=1e-13)
    fa.get_error()
    assert 0 < it < 10 * N and rel <= 1e-13
    rp, col, vo, _ = oracle.assemble(d, node, elem, k)
    uo = oracle.solve_reduced(rp, col, vo, host(b), host(isbd), gD)
    bd = host(isbd).astype(bool)
    assert np.array_equal(host(u)[bd], gD[bd])
    assert np.abs(host(u) - uo).max() <= 1e-10 * np.abs(uo).max(), np.abs(host(u) - uo).max()
    u2, it2, rel2 = fa.fem_cg_solve(p, dev(node), dev(k), isbd, b, dev(gD), rtol=1e-13)
    assert torch.equal(u, u2) and it == it2 and rel == rel2
    # a zero iteration budget leaves the lift; an exact start stops at once
    u0, it0, _ = fa.fem_cg_solve(p, dev(node), dev(k), isbd, b, dev(gD), max_iter=0)
    assert it0 == 0 and np.array_equal(host(u0)[bd], gD[bd]) and not host(u0)[~bd].any()
    uz, itz, relz = fa.fem_cg_solve(p, dev(node), dev(k), isbd, torch.zeros_like(b), None)
    assert itz == 0 and relz == 0.0 and not host(uz).any()


@pytest.mark.parametrize("case", ["sq37p", "kuhn7s", "delaunay3"])
def test_csr_spmv_matches_the_assembled_product(case):
    """fem_csr_spmv with the GPU's own assembled values: the plain product against scipy's CSR product of
    the same arrays (within 1e-13 of each row's sum of |a_ij x_j|), the eliminated one against
    fem_apply_stiffness's eliminated operator (within the parity bar of the same magnitudes: both sides
    round differently), and the same bits on a second call."""
    import scipy.sparse as sp
    d, node, elem, k, _ = mesh_case(case)
    N = node.shape[0]
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    kd = dev(k if k is not None else np.ones(elem.shape[0]))
    val = torch.empty(p.nnz, dtype=torch.float64, device="cuda")
    fa.fem_assemble_stiffness(p, dev(node), kd, val)
    isbd = torch.empty(N, dtype=torch.uint8, device="cuda")
    fa.fem_boundary_nodes(p, None, isbd)
    x = meshgen.normal(41, 3, N)
    y = fa.fem_csr_spmv(p, val, dev(x))
    fa.get_error()
    rp, col, v = host(p.row_ptr).astype(np.int64), host(p.col_idx).astype(np.int64), host(val)
    A = sp.csr_matrix((v, col, rp), shape=(N, N))
    mag = sp.csr_matrix((np.abs(v), col, rp), shape=(N, N)) @ np.abs(x)
    assert_close_scaled(host(y), A @ x, mag, tol=1e-13, what="csr product")
    assert torch.equal(y, fa.fem_csr_spmv(p, val, dev(x)))
    ye = fa.fem_csr_spmv(p, val, dev(x), isbd)
    ya = torch.empty_like(ye)
    fa.fem_apply_stiffness(p, dev(node), kd, dev(x), isbd, ya)
    fa.get_error()
    bd = host(isbd).astype(bool)
    assert np.array_equal(host(ye)[bd], x[bd])
    xm = np.where(bd, 0.0, x)
    mag_e = sp.csr_matrix((np.abs(v), col, rp), shape=(N, N)) @ np.abs(xm)
    assert_close_scaled(host(ye)[~bd], host(ya)[~bd], mag_e[~bd], what="eliminated csr product")


@pytest.mark.parametrize("d", [2, 3])
def test_cg_on_the_assembled_matrix_matches_the_direct_reduced_solve(d):
    """fem_cg_solve_csr with the GPU's assembled values (nonzero g_D, lognormal k, sine-product load)
    against the oracle's direct solve of the same reduced system, and against the matrix-free CG: boundary
    values exact, free values within the CG tolerance; the same bits and iteration count twice."""
    node, elem, k = _cg_case(d, 24 if d == 2 else 6, 91 + d)
    N = node.shape[0]
    p = fa.Pattern(dev(elem), N)
    fa.fem_pattern_set_locality(p, dev(node))
    val, b = fa.assemble(p, dev(node), dev(k), fa.FEM_F_SINPROD)
    fa.get_error()
    isbd = torch.empty(N, dtype=torch.uint8, device="cuda")
    fa.fem_boundary_nodes(p, None, isbd)
    gD = 0.5 + node @ np.arange(1.0, d + 1.0)
    u, it, rel = fa.fem_cg_solve_csr(p, val, isbd, b, dev(gD), rtol=1e-13)
    fa.get_error()
    assert 0 < it < 10 * N and rel <= 1e-13
    rp, col, vo, _ = oracle.assemble(d, node, elem, k)
    uo = oracle.solve_reduced(rp, col, vo, host(b), host(isbd), gD)
    bd = host(isbd).astype(bool)
    assert np.array_equal(host(u)[bd], gD[bd])
    assert np.abs(host(u) - uo).max() <= 1e-10 * np.abs(uo).max(), np.abs(host(u) - uo).max()
    um, itm, _ = fa.fem_cg_solve(p, dev(node), dev(k), isbd, b, dev(gD), rtol=1e-13)
    assert np.abs(host(u) - host(um)).max() <= 1e-10 * np.abs(uo).max() and abs(it - itm) <= max(3, itm // 20)
    u2, it2, rel2 = fa.fem_cg_solve_csr(p, val, isbd, b, dev(gD), rtol=1e-13)
    assert torch.equal(u, u2) and it == it2 and rel == rel2


@pytest.mark.parametrize("d", [2, 3])
def test_cg_solution_converges_at_second_order(d):
    """-Laplace u = sin-product with u = 0 on the boundary, solved on the GPU by the load vector and the
    matrix-free CG: the nodal error against f / (d pi^2) falls by about 4 per halving of h."""
    errs = []
    for n in ((8, 16, 32) if d == 2 else (4, 8, 16)):
        m = meshgen.square_mesh(n) if d == 2 else meshgen.kuhn_mesh(n)
        node, elem = m["node"], m["elem"]
        N = node.shape[0]
        p = fa.Pattern(dev(elem), N)
        _, b = fa.assemble(p, dev(node), None, fa.FEM_F_SINPROD)
        isbd = torch.empty(N, dtype=torch.uint8, device="cuda")
        fa.fem_boundary_nodes(p, None, isbd)
        u, it, rel = fa.fem_cg_solve(p, dev(node), None, isbd, b, None, rtol=1e-12)
        fa.get_error()
        errs.append(float(np.abs(host(u) - np.prod(np.sin(np.pi * node), axis=1) / (d * np.pi ** 2)).max()))
    rates = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.5 < r < 4.5 for r in rates), (errs, rates)


def test_cg_reports_breakdown():
    """Vertices that no element touches have a zero operator row: with a nonzero right side there, the
    first step finds p.Ap = 0 and the call reports the breakdown (FEM_ERR_STATE) instead of dividing by 0."""
    p = fa.Pattern(torch.zeros((0, 3), dtype=torch.int32, device="cuda"), 4)
    node = dev(np.zeros((4, 2)))
    isbd = dev(np.array([1, 0, 0, 0], np.uint8))
    b = dev(np.ones(4))
    with pytest.raises(fa.FemError) as e:
        fa.fem_cg_solve(p, node, None, isbd, b, None, max_iter=10)
    assert e.value.code == fa.FEM_ERR_STATE
    assert b"breakdown" in fa.lib().fem_last_error_string()
