"""Seeded synthetic inputs for P1 assembly: simplicial meshes, coefficients, loss weights.

This module only builds inputs. It holds none of the assembly arithmetic (no measures, gradients,
local matrices, quadrature or sparse summation), so the CPU oracle and the CUDA library can both be
fed from it without sharing any of the method.

Data layout follows the paper's mesh data structure (Sec. 1.1): ``node`` is float64 [N, d] and
``elem`` is int32 [NT, d+1]; indices here are 0-based. Every element is positively oriented
(counter-clockwise triangles, right-handed tetrahedra), as Sec. 1.1 requires. Orientation is fixed
combinatorially: a Kuhn tetrahedron built from an odd axis permutation gets its last two vertices
swapped. ``bdflag`` follows Sec. 1.2: side i of an element is the side opposite vertex i and carries
1 when it lies on the boundary of the unit square/cube (whole-boundary Dirichlet), else 0.

Random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): output i of a stream with
state s is mix(s + (i+1)*0x9E3779B97F4A7C15), where mix is the published finaliser
(xor-shift 30, multiply 0xBF58476D1CE4E5B9, xor-shift 27, multiply 0x94D049BB133111EB, xor-shift 31).
Uniform doubles take the top 53 bits; normals use Box-Muller on consecutive uniform pairs.
Each array draws from its own stream, whose state is mix(seed ^ tag * 0xD1B54A32D192ED03).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "splitmix64", "uniform", "normal", "lognormal", "square_mesh", "kuhn_mesh",
    "batch_sides", "CONFIGS", "make_config",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TAGMUL = 0xD1B54A32D192ED03

# stream tags (one per kind of random array)
TAG_JITTER, TAG_PERM, TAG_COEF, TAG_W, TAG_R, TAG_SIDES, TAG_GD = 1, 2, 3, 4, 5, 6, 7


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _state(seed: int, tag: int) -> np.uint64:
    s = (int(seed) ^ ((int(tag) * _TAGMUL) & 0xFFFFFFFFFFFFFFFF)) & 0xFFFFFFFFFFFFFFFF
    with np.errstate(over="ignore"):
        return _mix(np.array([s], dtype=np.uint64))[0]


def splitmix64(seed: int, tag: int, n: int) -> np.ndarray:
    """n raw 64-bit outputs of the SplitMix64 stream (seed, tag)."""
    s = _state(seed, tag)
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(s + i * _GAMMA)


def uniform(seed: int, tag: int, n: int) -> np.ndarray:
    """n doubles uniform on [0, 1): top 53 bits of each SplitMix64 output times 2^-53."""
    return (splitmix64(seed, tag, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, tag: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller: z = sqrt(-2 ln(1-u1)) cos(2 pi u2) on pairs (u1, u2)."""
    u = uniform(seed, tag, 2 * n)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def lognormal(seed: int, tag: int, n: int) -> np.ndarray:
    """n draws of exp(z), z ~ N(0, 1)."""
    return np.exp(normal(seed, tag, n))


def square_mesh(n: int, jitter: float = 0.0, seed: int = 0, permute: bool = False) -> dict:
    """Unit square, n x n cells, each cut along the same diagonal into two triangles.

    Node (i, j) has index j*(n+1)+i and sits at (i/n, j/n). Cell (i, j) gives triangles
    (v00, v10, v11) and (v00, v11, v01), both counter-clockwise. Interior nodes move by independent
    U(-jitter*h, jitter*h) offsets per coordinate (h = 1/n); boundary nodes stay put. With
    ``permute`` the element rows are put in a seeded uniformly random order.
    """
    n1 = n + 1
    jj, ii = np.meshgrid(np.arange(n1), np.arange(n1), indexing="ij")
    node = np.stack([ii.ravel() / n, jj.ravel() / n], axis=1).astype(np.float64)
    onb = (ii.ravel() == 0) | (ii.ravel() == n) | (jj.ravel() == 0) | (jj.ravel() == n)
    if jitter > 0.0:
        h = 1.0 / n
        u = uniform(seed, TAG_JITTER, 2 * node.shape[0]).reshape(-1, 2)
        off = (2.0 * u - 1.0) * (jitter * h)
        off[onb] = 0.0
        node = node + off
    cj, ci = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ci, cj = ci.ravel(), cj.ravel()
    v00 = cj * n1 + ci
    v10, v01, v11 = v00 + 1, v00 + n1, v00 + n1 + 1
    elem = np.empty((2 * n * n, 3), dtype=np.int32)
    elem[0::2] = np.stack([v00, v10, v11], axis=1)
    elem[1::2] = np.stack([v00, v11, v01], axis=1)
    # side m is opposite vertex m: T1 sides (v10,v11) right, (v11,v00) diagonal, (v00,v10) bottom;
    # T2 sides (v11,v01) top, (v01,v00) left, (v00,v11) diagonal.
    bd = np.zeros((2 * n * n, 3), dtype=np.int8)
    bd[0::2, 0] = ci == n - 1
    bd[0::2, 2] = cj == 0
    bd[1::2, 0] = cj == n - 1
    bd[1::2, 1] = ci == 0
    if permute:
        keys = splitmix64(seed, TAG_PERM, elem.shape[0])
        order = np.argsort(keys, kind="stable")
        elem = np.ascontiguousarray(elem[order])
        bd = np.ascontiguousarray(bd[order])
    return {"d": 2, "n": n, "node": np.ascontiguousarray(node), "elem": elem,
            "is_bd": onb.astype(np.uint8), "bdflag": bd}


_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
_ODD = [False, True, True, False, False, True]


def kuhn_mesh(n: int, jitter: float = 0.0, seed: int = 0) -> dict:
    """Unit cube, n^3 cells, each split into the 6 Kuhn tetrahedra.

    Grid point (a, b, c) has index a + (n+1)*(b + (n+1)*c). For an axis permutation p the tet is
    v0 -> v0+e_p0 -> v0+e_p0+e_p1 -> v0+e_p0+e_p1+e_p2; odd permutations swap the last two
    vertices so that every tet is right-handed. Interior nodes are jittered as in ``square_mesh``.
    """
    n1 = n + 1
    cc, bb, aa = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    aa, bb, cc = aa.ravel(), bb.ravel(), cc.ravel()
    node = np.stack([aa / n, bb / n, cc / n], axis=1).astype(np.float64)
    onb = (aa == 0) | (aa == n) | (bb == 0) | (bb == n) | (cc == 0) | (cc == n)
    if jitter > 0.0:
        h = 1.0 / n
        u = uniform(seed, TAG_JITTER, 3 * node.shape[0]).reshape(-1, 3)
        off = (2.0 * u - 1.0) * (jitter * h)
        off[onb] = 0.0
        node = node + off
    kc, jc, ic = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ic, jc, kc = ic.ravel(), jc.ravel(), kc.ravel()
    ncell = ic.size
    stride = np.array([1, n1, n1 * n1], dtype=np.int64)
    base = ic + n1 * (jc + n1 * kc)
    elem = np.empty((6 * ncell, 4), dtype=np.int32)
    grid = np.empty((6 * ncell, 4, 3), dtype=np.int64)  # integer grid coordinates, for bdflag
    cell_xyz = np.stack([ic, jc, kc], axis=1)
    for q, (p, odd) in enumerate(zip(_PERMS, _ODD)):
        v = [base.copy()]
        g = [cell_xyz.copy()]
        for ax in p:
            v.append(v[-1] + stride[ax])
            gg = g[-1].copy()
            gg[:, ax] += 1
            g.append(gg)
        if odd:
            v[2], v[3] = v[3], v[2]
            g[2], g[3] = g[3], g[2]
        elem[q::6] = np.stack(v, axis=1)
        grid[q::6] = np.stack(g, axis=1)
    bd = np.zeros((6 * ncell, 4), dtype=np.int8)
    for m in range(4):
        others = [x for x in range(4) if x != m]
        fg = grid[:, others, :]  # [NT, 3, 3]
        on = np.zeros(6 * ncell, dtype=bool)
        for ax in range(3):
            c = fg[:, :, ax]
            on |= ((c == 0).all(axis=1)) | ((c == n).all(axis=1))
        bd[:, m] = on
    return {"d": 3, "n": n, "node": np.ascontiguousarray(node), "elem": elem,
            "is_bd": onb.astype(np.uint8), "bdflag": bd}


def side_flags(mesh: dict, faces: dict) -> np.ndarray:
    """bdFlag [NT, d+1] (int8) for the unit square / cube meshes above: every boundary side gets the
    flag its face name maps to ("x0", "x1", "y0", "y1", and "z0", "z1" in 3-D; missing names give 1),
    interior sides 0. Boundary nodes are not jittered, so a side lies on face "x0" when all its
    vertices have x == 0 exactly."""
    d, node, elem, bd = mesh["d"], mesh["node"], mesh["elem"], mesh["bdflag"]
    out = np.zeros(bd.shape, dtype=np.int8)
    names = ["x", "y", "z"][:d]
    for j in range(d + 1):
        others = [k for k in range(d + 1) if k != j]
        xs = node[elem[:, others]]  # [NT, d, d]
        onb = bd[:, j] != 0
        flag = np.where(onb, 1, 0).astype(np.int8)
        for ax, nm in enumerate(names):
            for val, tag in ((0.0, "0"), (1.0, "1")):
                on = onb & np.all(xs[:, :, ax] == val, axis=1)
                flag[on] = faces.get(nm + tag, 1)
        out[:, j] = flag
    return out


def batch_sides(seed: int = 1806, count: int = 256, lo: int = 16, hi: int = 512) -> np.ndarray:
    """Mesh sides n uniform on {lo, ..., hi}."""
    u = uniform(seed, TAG_SIDES, count)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


# Named workloads. f: "const" (f = 1), "sinprod" (product of sin(pi x_m) over coordinates).
CONFIGS = {
    "c1": dict(kind="square", n=64, jitter=0.0, seed=0, permute=False, coef=None, f="const"),
    "c2": dict(kind="square", n=2048, jitter=0.2, seed=1804, permute=True, coef="lognormal", f="sinprod"),
    "c3": dict(kind="kuhn", n=128, jitter=0.1, seed=1805, permute=False, coef="lognormal", f="const"),
    "c4": dict(kind="batch", count=256, lo=16, hi=512, jitter=0.2, seed=1806, coef="lognormal", f="sinprod"),
    "c5": dict(kind="kuhn", n=64, jitter=0.1, seed=1807, permute=False, coef="lognormal", f="sinprod",
               loss_seed=1808),
}


def make_config(name: str, n: int | None = None, count: int | None = None) -> dict:
    """Build a named workload; ``n`` (or ``count`` for the batch) overrides the size for small cases."""
    c = dict(CONFIGS[name])
    if c["kind"] == "batch":
        cnt = c["count"] if count is None else count
        sides = batch_sides(c["seed"], cnt, c["lo"], c["hi"])
        if n is not None:  # small test variant: same draw, scaled down
            sides = np.maximum(2, (sides * n) // c["hi"])
        meshes = []
        for m, s in enumerate(sides):
            sub = c["seed"] * 1000 + m
            mesh = square_mesh(int(s), c["jitter"], sub, False)
            mesh["coef"] = lognormal(sub, TAG_COEF, mesh["elem"].shape[0])
            meshes.append(mesh)
        return {"name": name, "kind": "batch", "d": 2, "sides": sides, "meshes": meshes, "f": c["f"]}
    nn = c["n"] if n is None else n
    if c["kind"] == "square":
        mesh = square_mesh(nn, c["jitter"], c["seed"], c["permute"])
    else:
        mesh = kuhn_mesh(nn, c["jitter"], c["seed"])
    nt = mesh["elem"].shape[0]
    mesh["coef"] = None if c["coef"] is None else lognormal(c["seed"], TAG_COEF, nt)
    mesh["name"], mesh["kind"], mesh["f"] = name, c["kind"], c["f"]
    mesh["seed"] = c["seed"]
    if "loss_seed" in c:
        mesh["loss_seed"] = c["loss_seed"]
    return mesh
