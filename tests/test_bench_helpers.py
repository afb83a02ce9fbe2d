"""Host-side pieces of the benchmark (no GPU): the oracle's sample patch, the algorithmic byte count and
the lookup of ncu records by kernel, workload, plan and source digest."""
import importlib.util
import os

import numpy as np
import pytest

import meshgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_patch_sample_is_a_connected_region_over_its_own_vertices(bench):
    m = meshgen.square_mesh(40, 0.2, 3, permute=True)
    node, elem = m["node"], m["elem"]
    k = meshgen.lognormal(3, 3, elem.shape[0])
    n_s, e_s, k_s, nv = bench.patch_sample(node, elem, k, 600)
    assert e_s.shape == (600, 3) and n_s.shape == (nv, 2) and k_s.shape == (600,)
    # renumbered: every local vertex is used, ids are 0 .. nv-1
    assert np.array_equal(np.unique(e_s), np.arange(nv))
    # a patch of the grid, not scattered triangles: about half a vertex per element (plus its rim)
    assert nv < 0.75 * 600
    # the same elements of the mesh, with their own coefficients, in ascending element order
    pick = np.sort(np.argsort(elem.max(axis=1), kind="stable")[:600])
    assert np.array_equal(k_s, k[pick])
    assert np.allclose(n_s[e_s], node[elem[pick]])
    # the whole mesh: the identity numbering
    n_a, e_a, _, nv_a = bench.patch_sample(node, elem, None, elem.shape[0])
    assert nv_a == node.shape[0] and np.array_equal(e_a, elem) and np.array_equal(n_a, node)


def test_algorithmic_bytes(bench):
    # elem (d+1) int32 + node once (d doubles) + k + val + b
    assert bench.algorithmic_bytes(2, 4198401, 8388608, 29372417) == 503513120
    assert bench.algorithmic_bytes(3, 10, 7, 100) == 7 * 16 + 10 * 24 + 7 * 8 + 100 * 8 + 10 * 8


def test_profile_records_follow_the_kernel_source(bench, tmp_path, monkeypatch):
    from paper_1804_05156_gb300 import buildlib
    d = buildlib.tu_digest("values_tiles.cu")
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "x.md").write_text(
        "traffic-record: kernel=(ka<2, 128>); config=c2; plan=128; bytes_per_launch=100; source=values_tiles.cu; "
        "source_digest=%s\n"
        "traffic-record: kernel=(kb<2, 128>); config=c2; plan=128; bytes_per_launch=20; source=values_tiles.cu; "
        "source_digest=%s\n"
        "traffic-record: kernel=(kb<2, 128>); config=c3; plan=128; bytes_per_launch=999; source=values_tiles.cu; "
        "source_digest=%s\n"
        "inst-record: kernel=(ka<2, 128>); config=c2; plan=128; warp_inst_per_launch=7; source=values_tiles.cu; "
        "source_digest=%s\n" % (d, d, d, "0" * 64))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    path = {"path": "tiles", "tile_elems": 128}
    v, src = bench.profiled(["(ka<2, 128>)", "(kb<2, 128>)"], "c2", path, {})
    assert v == 120 and src == "x.md"
    # another workload, another plan, or a record taken from other source code: no figure
    assert bench.profiled(["(ka<2, 128>)", "(kb<2, 128>)"], "c1", path, {})[0] is None
    assert bench.profiled(["(ka<2, 128>)"], "c2", {"path": "tiles", "tile_elems": 256}, {})[0] is None
    assert bench.profiled(["(ka<2, 128>)"], "c2", path, {}, "inst", "warp_inst_per_launch")[0] is None
    # comments do not change the digest; code does
    assert buildlib._code_only("int a; // x\n/* y */ int b;") == buildlib._code_only("int a;\nint b; // z")
    assert buildlib._code_only("int a;") != buildlib._code_only("int b;")
