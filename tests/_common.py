"""Helpers shared by the GPU parity tests: input preparation and comparisons (no method arithmetic)."""
import numpy as np
import torch

import meshgen
import oracle

TOL = 1e-12  # relative to the per-slot magnitude scale returned by the oracle
BWD_TOL = 1e-10  # gradients: relative to the per-entry magnitude of the adjoint's terms (oracle with_scale)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def gpu_slot_to_tij(slot_flat, NT, d1):
    """GPU slot map [(i*d1+j)*NT + t] -> [NT, d1, d1]."""
    return slot_flat.reshape(d1 * d1, NT).T.reshape(NT, d1, d1)


def assert_close_scaled(got, exp, scale, tol=TOL, what="values"):
    got, exp, scale = np.asarray(got), np.asarray(exp), np.asarray(scale)
    err = np.abs(got - exp)
    bad = err > tol * scale
    if bad.any():
        i = int(np.argmax(np.where(bad, err / np.maximum(scale, 1e-300), 0)))
        raise AssertionError("%s: %d of %d outside %g*scale; worst at %d: got %r exp %r scale %r" % (
            what, int(bad.sum()), got.size, tol, i, got.flat[i], exp.flat[i], scale.flat[i]))


def sample_rows(N, count, seed):
    rng = np.random.default_rng(seed)
    rows = set(rng.choice(N, size=min(count, N), replace=False).tolist())
    rows.update([0, N - 1, N // 2])
    return np.array(sorted(rows), dtype=np.int64)


def mesh_case(name):
    """Named small/medium parity cases: (d, node, elem, k, f_kind)."""
    if name == "c1":
        m = meshgen.make_config("c1")
        return 2, m["node"], m["elem"], None, oracle.F_CONST
    if name == "sq37p":
        m = meshgen.square_mesh(37, 0.2, 99, permute=True)
        return 2, m["node"], m["elem"], meshgen.lognormal(99, 3, m["elem"].shape[0]), oracle.F_SINPROD
    if name == "sq2":
        m = meshgen.square_mesh(2, 0.2, 5)
        return 2, m["node"], m["elem"], meshgen.lognormal(5, 3, m["elem"].shape[0]), oracle.F_SINPROD
    if name == "kuhn5":
        m = meshgen.kuhn_mesh(5, 0.1, 77)
        return 3, m["node"], m["elem"], meshgen.lognormal(77, 3, m["elem"].shape[0]), oracle.F_CONST
    if name == "kuhn7s":
        m = meshgen.kuhn_mesh(7, 0.1, 78)
        return 3, m["node"], m["elem"], meshgen.lognormal(78, 3, m["elem"].shape[0]), oracle.F_SINPROD
    if name in ("delaunay2", "delaunay3"):
        d = 2 if name == "delaunay2" else 3
        from scipy.spatial import Delaunay
        rng = np.random.default_rng(2024 + d)
        pts = rng.uniform(0, 1, size=(700 if d == 2 else 300, d))
        tri = Delaunay(pts)
        elem = tri.simplices.astype(np.int32)
        # positive orientation (Sec. 1.1): swap two vertices where the signed measure is negative
        e = pts[elem]
        det = np.linalg.det(e[:, 1:, :] - e[:, :1, :])
        keep = np.abs(det) > 1e-9
        elem, det = elem[keep], det[keep]
        neg = det < 0
        elem[neg, 0], elem[neg, 1] = elem[neg, 1].copy(), elem[neg, 0].copy()
        # two isolated vertices at the end give empty rows
        pts = np.vstack([pts, [[0.5] * d, [0.25] * d]])
        k = np.exp(rng.normal(size=elem.shape[0]))
        return d, pts, np.ascontiguousarray(elem), k, oracle.F_SINPROD
    raise KeyError(name)
