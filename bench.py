#!/usr/bin/env python3
"""Benchmark: P1 assembly throughput (Melem/s, FP64) on the 2048^2 jittered, element-permuted
triangle mesh (N = 4,198,401 vertices, NT = 8,388,608 elements, lognormal k, f = sin(pi x) sin(pi y)).

A step is one pass of the value phase of the assembly on a built pattern: stiffness values and the
load vector (one fem_assemble call), inputs resident in HBM. The pattern build (once per topology)
is timed separately and reported as pattern_build_ms. e2e repeats the step through the C ABI's
host-buffer call (fem_assemble_host): every step copies its inputs from page-locked host memory and
its outputs (val, b) back inside the timed region, the steps pipelined within the call (the
one-step-per-call time is reported beside it). The L2 is flushed (a 512 MB write) between timed
steps, outside the timed events.

--impl reference times the CPU oracle (the plain FP64 reference) on a bounded sample of the same
workload, on this host's cores. Under torchrun each rank assembles its own copy of the mesh
(independent problems, no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import meshgen  # noqa: E402

METRIC = "P1 assembly Melem/s (FP64) + % HBM peak; batched & fwd+bwd vs plain fwd"


def _measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(p)) if os.path.exists(p) else {}


def peaks():
    j = _measured_peaks()
    if "hbm_gbs" in j:
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def algorithmic_bytes(d, N, NT, nnz, part="all"):
    """Minimum bytes of the value phase: elem, node (each vertex once), k, val, b (part "stiffness": no b;
    "load": no k and no val)."""
    geo = NT * (d + 1) * 4 + N * d * 8
    if part == "stiffness":
        return geo + NT * 8 + nnz * 8
    if part == "load":
        return geo + N * 8
    return geo + NT * 8 + nnz * 8 + N * 8


def cg_csr_iteration_bytes(N, nnz):
    """Minimum bytes of one CG iteration on the assembled matrix: the product (val, col_idx, row_ptr, the
    boundary mask and the direction p read, A p written) and the same vector kernels as cg_iteration_bytes."""
    return nnz * 12 + (N + 1) * 4 + N + N * 8 + N * 8 + 8 * N * (2 + 6 + 3)


def cg_iteration_bytes(d, N, NT):
    """Minimum bytes of one matrix-free CG iteration: the operator (elem, node, k, the direction p and
    the boundary mask read, A p written) and the vector kernels (p.q: p, q read; update: p, q, u, r read,
    u, r written; direction: r, p read, p written), all FP64 vectors of N entries."""
    return NT * (d + 1) * 4 + N * d * 8 + NT * 8 + N * 8 + N + N * 8 + 8 * N * (2 + 6 + 3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.rows, self.proc, self.idx = [], None, gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _nvtx(torch):
    """(push, pop) of an NVTX range, or no-ops where this torch build has no NVTX."""
    try:
        torch.cuda.nvtx.range_push("probe")
        torch.cuda.nvtx.range_pop()
        return torch.cuda.nvtx.range_push, torch.cuda.nvtx.range_pop
    except (RuntimeError, AttributeError):
        return (lambda name: None), (lambda: None)


def profiled(kernels, config, path, shape, kind="traffic", field="bytes_per_launch"):
    """Per-step sum over the step's kernels of a per-launch ncu figure, from the committed summaries
    under profiles/ (lines starting '<kind>-record:'), if every kernel was captured on this config and
    plan from its current source (the record names the kernel's source file and that file's digest);
    else None. kind "traffic": DRAM bytes read + written; kind "inst": warp instructions executed."""
    from paper_1804_05156_gb300 import buildlib
    digests = {}

    def current(kv):
        src = kv.get("source")
        if src not in digests:
            digests[src] = buildlib.tu_digest(src) if src else buildlib.source_digest()
        return digests[src]
    plan = str(path["tile_elems"]) if path["path"].startswith("tiles") else str(shape.get("rows_per_block"))
    pdir = os.path.join(ROOT, "profiles")
    found = {}
    tag = kind + "-record:"
    if os.path.isdir(pdir):
        for fn in sorted(os.listdir(pdir)):
            if not fn.endswith(".md"):
                continue
            for line in open(os.path.join(pdir, fn)):
                if not line.startswith(tag):
                    continue
                kv = dict(x.strip().split("=", 1) for x in line[len(tag):].split(";") if "=" in x)
                if (kv.get("kernel") in kernels and kv.get("config") == config and kv.get("plan") == plan
                        and field in kv and kv.get("source_digest") == current(kv)):
                    found[kv["kernel"]] = (float(kv[field]), fn)
    if kernels and all(k in found for k in kernels):
        return sum(found[k][0] for k in kernels), ", ".join(sorted({found[k][1] for k in kernels}))
    return None, "no ncu capture of these kernels on this plan and source digest under profiles/"


def patch_sample(node, elem, k, m):
    """A bounded sample of the mesh for the oracle: the m elements of lowest largest vertex id (a connected
    patch, whatever the element order), in ascending element order, over their own vertices renumbered
    (so the per-vertex share of the oracle's work is the whole mesh's). Returns (node, elem, k, vertices)."""
    pick = np.sort(np.argsort(elem.max(axis=1), kind="stable")[:m])
    used, sub = np.unique(elem[pick], return_inverse=True)
    return (np.ascontiguousarray(node[used]), sub.reshape(m, -1).astype(np.int32),
            None if k is None else k[pick], len(used))


def cpu_baseline(mesh, f_kind, target_s=12.0):
    """The oracle as it stands on a bounded sample (a patch of M elements of the same mesh), one core."""
    import oracle
    oracle.build()
    d, node, elem, k = mesh["d"], mesh["node"], mesh["elem"], mesh["coef"]
    NT = elem.shape[0]

    def run(m):
        n_s, e_s, k_s, nv = patch_sample(node, elem, k, m)
        t0 = time.perf_counter()
        oracle.assemble(d, n_s, e_s, k_s)
        oracle.rhs(d, n_s, e_s, f_kind)
        return time.perf_counter() - t0, nv

    m = min(NT, 100_000)
    dt, nv = run(m)
    m2 = int(min(NT, max(m, m * target_s / max(dt, 1e-3))))
    if m2 > m:
        m, (dt, nv) = m2, run(m2)
    return {"value": m / dt / 1e6, "unit": "Melem/s", "cores": 1, "kind": "oracle",
            "sample": "a patch of %d of the %d elements of the same mesh, over its %d vertices (stiffness "
                      "triples + sparse summation + load vector), single-threaded C, %.1f s" % (m, NT, nv, dt)}


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
        return dist, dist.get_rank(), ws
    return None, 0, 1


def max_over_ranks(dist, x: float) -> float:
    """The largest value of x over all ranks (a timing reduction, not part of the assembly)."""
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    dist, rank, ws = dist_init(args)
    if rank != 0:
        return
    mesh = meshgen.make_config(args.config)
    import oracle
    f_kind = oracle.F_SINPROD if mesh["f"] == "sinprod" else oracle.F_CONST
    d, node, elem, k = mesh["d"], mesh["node"], mesh["elem"], mesh["coef"]
    oracle.build()
    m = min(elem.shape[0], args.ref_sample)
    n_s, e_s, k_s, nv = patch_sample(node, elem, k, m)
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.assemble(d, n_s, e_s, k_s)
        oracle.rhs(d, n_s, e_s, f_kind)
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    v = m / (ms * 1e-3) / 1e6
    line = {"metric": METRIC, "value": v, "unit": "Melem/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(args.config), "sample_elements": m},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": v, "unit": "Melem/s",
                             "sample": "a patch of %d elements of the mesh (over its %d vertices) per step, "
                                       "single-threaded C oracle" % (m, nv)},
            "e2e": {"value": v, "unit": "Melem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_name(cfg):
    return {"c1": "2-D unit square 64x64, uniform, k=1, f=1",
            "c2": "2-D unit square 2048x2048, jittered 0.2h, element rows permuted, k~LN(0,1), f=sin(pi x)sin(pi y)",
            "c3": "3-D unit cube 128^3 Kuhn tets, jittered 0.1h, k~LN(0,1), f=1"}[cfg]


def _time_steps(fn, steps, flush, s):
    """Mean ms of `fn` over `steps` calls, CUDA events on stream s, L2 flushed between calls."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(s)
        fn()
        evs[i][1].record(s)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / steps


def extras(fa, args, flush, plain_melem):
    """Secondary rows of the metric: 3-D (C3), batched (C4), fwd+bwd (C5), the CG solve on C5, and C1."""
    import torch
    s = torch.cuda.current_stream()
    out = {}
    steps = max(3, min(args.steps, 10))
    # 3-D 128^3 Kuhn (C3)
    m = meshgen.make_config("c3")
    nd, kd = torch.as_tensor(m["node"]).cuda(), torch.as_tensor(m["coef"]).cuda()
    t0 = time.perf_counter()
    p = fa.Pattern(torch.as_tensor(m["elem"]).cuda(), m["node"].shape[0])
    fa.fem_pattern_set_locality(p, nd)
    torch.cuda.synchronize()
    pms = 1e3 * (time.perf_counter() - t0)
    val = torch.empty(p.nnz, dtype=torch.float64, device="cuda")
    b = torch.empty(p.N, dtype=torch.float64, device="cuda")
    f = lambda: fa.fem_assemble(p, nd, kd, fa.FEM_F_CONST, None, val, b, fa.FEM_DETERMINISTIC)
    for _ in range(3):
        f()
    ms = _time_steps(f, steps, flush, s)
    NT = m["elem"].shape[0]
    out["c3_3d_128cube"] = {"ms": ms, "Melem_s": NT / (ms * 1e-3) / 1e6, "NT": NT, "nnz": p.nnz,
                            "pattern_build_ms": pms, "launch": fa.fem_pattern_launch_shape(p),
                            "path": fa.fem_pattern_value_path(p),
                            "algorithmic_GBs": algorithmic_bytes(3, p.N, NT, p.nnz) / (ms * 1e-3) / 1e9}
    del p, val, b, nd, kd, m
    torch.cuda.empty_cache()
    # batched: 256 squares, n ~ U{16..512}, one persistent launch replayed from a CUDA graph (C4)
    c4 = meshgen.make_config("c4")
    ms_ = c4["meshes"]
    elem_cat = np.concatenate([x["elem"] for x in ms_])
    node_cat = torch.as_tensor(np.concatenate([x["node"] for x in ms_])).cuda()
    k_cat = torch.as_tensor(np.concatenate([x["coef"] for x in ms_])).cuda()
    t0 = time.perf_counter()
    bt = fa.Batch(2, [x["node"].shape[0] for x in ms_], [x["elem"].shape[0] for x in ms_],
                  torch.as_tensor(elem_cat).cuda())
    bt.set_locality(node_cat)
    torch.cuda.synchronize()
    bpms = 1e3 * (time.perf_counter() - t0)
    val = torch.empty(bt.nnz_off[-1], dtype=torch.float64, device="cuda")
    b = torch.empty(bt.node_off[-1], dtype=torch.float64, device="cuda")
    f = lambda: bt.assemble(node_cat, k_cat, fa.FEM_F_SINPROD, None, val, b, fa.FEM_DETERMINISTIC, graph=True)
    for _ in range(3):
        f()
    ms = _time_steps(f, steps, flush, s)
    NT = elem_cat.shape[0]
    bm = NT / (ms * 1e-3) / 1e6
    out["c4_batched_256"] = {"ms": ms, "Melem_s": bm, "NT": NT, "meshes": len(ms_), "nnz": bt.nnz_off[-1],
                             "plan_ms": bpms, "launch": fa.fem_pattern_launch_shape(bt.pattern),
                             "path": fa.fem_pattern_value_path(bt.pattern),
                             "graph": True, "vs_plain_fwd": bm / plain_melem}
    del bt, val, b, node_cat, k_cat, elem_cat, c4, ms_
    torch.cuda.empty_cache()
    # differentiable: 64^3 Kuhn, forward then backward of L = w.A + r.b (C5)
    m = meshgen.make_config("c5")
    nd, kd = torch.as_tensor(m["node"]).cuda(), torch.as_tensor(m["coef"]).cuda()
    p = fa.Pattern(torch.as_tensor(m["elem"]).cuda(), m["node"].shape[0])
    fa.fem_pattern_set_locality(p, nd)
    w = torch.as_tensor(meshgen.normal(m["loss_seed"], meshgen.TAG_W, p.nnz)).cuda()
    r = torch.as_tensor(meshgen.normal(m["loss_seed"], meshgen.TAG_R, p.N)).cuda()
    val = torch.empty(p.nnz, dtype=torch.float64, device="cuda")
    b = torch.empty(p.N, dtype=torch.float64, device="cuda")
    gn = torch.empty((p.N, 3), dtype=torch.float64, device="cuda")
    gk = torch.empty(p.NT, dtype=torch.float64, device="cuda")
    fwd = lambda: fa.fem_assemble(p, nd, kd, fa.FEM_F_SINPROD, None, val, b, fa.FEM_DETERMINISTIC)

    def fwdbwd():
        fwd()
        fa.fem_assemble_backward(p, nd, kd, fa.FEM_F_SINPROD, None, w, r, gn, gk)
    for _ in range(3):
        fwdbwd()
    ms_f = _time_steps(fwd, steps, flush, s)
    ms_fb = _time_steps(fwdbwd, steps, flush, s)
    NT = m["elem"].shape[0]
    out["c5_fwd_bwd_64cube"] = {"fwd_ms": ms_f, "fwd_bwd_ms": ms_fb, "NT": NT,
                                "fwd_Melem_s": NT / (ms_f * 1e-3) / 1e6, "fwd_bwd_Melem_s": NT / (ms_fb * 1e-3) / 1e6,
                                "fwd_bwd_vs_plain_fwd": ms_f / ms_fb}
    # the reduced Dirichlet solve on the same mesh (Sec. 3.3) by matrix-free CG: whole boundary, g_D = 0
    isbd = torch.empty(p.N, dtype=torch.uint8, device="cuda")
    fa.fem_boundary_nodes(p, None, isbd)
    fwd()
    u = torch.empty(p.N, dtype=torch.float64, device="cuda")
    fa.fem_cg_solve(p, nd, kd, isbd, b, None, u, max_iter=16, rtol=1e-8)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, its, rel = fa.fem_cg_solve(p, nd, kd, isbd, b, None, u, max_iter=5000, rtol=1e-8)
    torch.cuda.synchronize()
    cg_ms = 1e3 * (time.perf_counter() - t0)
    fa.get_error()
    fa.fem_assemble(p, nd, kd, fa.FEM_F_SINPROD, None, val, b, fa.FEM_DETERMINISTIC)
    fa.fem_cg_solve_csr(p, val, isbd, b, None, u, max_iter=16, rtol=1e-8)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, its_c, rel_c = fa.fem_cg_solve_csr(p, val, isbd, b, None, u, max_iter=5000, rtol=1e-8)
    torch.cuda.synchronize()
    cgc_ms = 1e3 * (time.perf_counter() - t0)
    fa.get_error()
    out["c5_cg_solve_64cube"] = {"iterations": its, "relres": rel, "rtol": 1e-8, "ms": cg_ms,
                                 "ms_per_iteration": cg_ms / max(its, 1),
                                 "operator": "matrix-free fem_apply_stiffness (Dirichlet-eliminated), FP64 vectors",
                                 "assembled": {"api": "fem_cg_solve_csr", "iterations": its_c, "relres": rel_c,
                                               "ms": cgc_ms, "ms_per_iteration": cgc_ms / max(its_c, 1)}}
    del p, val, b, gn, gk, w, r, nd, kd, u, isbd
    torch.cuda.empty_cache()
    # the small, launch-bound end of the metric: 64 x 64 uniform, k = 1, f = 1 (C1)
    m = meshgen.make_config("c1")
    nd = torch.as_tensor(m["node"]).cuda()
    p = fa.Pattern(torch.as_tensor(m["elem"]).cuda(), m["node"].shape[0])
    fa.fem_pattern_set_locality(p, nd)
    val = torch.empty(p.nnz, dtype=torch.float64, device="cuda")
    b = torch.empty(p.N, dtype=torch.float64, device="cuda")
    f = lambda: fa.fem_assemble(p, nd, None, fa.FEM_F_CONST, None, val, b, fa.FEM_DETERMINISTIC)
    for _ in range(3):
        f()
    ms = _time_steps(f, max(steps, 20), flush, s)
    NT = m["elem"].shape[0]
    out["c1_2d_64sq"] = {"ms": ms, "Melem_s": NT / (ms * 1e-3) / 1e6, "NT": NT, "nnz": p.nnz,
                         "path": fa.fem_pattern_value_path(p)}
    fa.get_error()
    return out


def run_ours(args):
    import torch
    import paper_1804_05156_gb300 as fa

    dist, rank, ws = dist_init(args)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0:
        fa.build()  # one build (a no-op when the library is current); the other ranks wait for it
    if dist:
        dist.barrier()
    mesh = meshgen.make_config(args.config, n=args.grid)
    d, node, elem, k = mesh["d"], mesh["node"], mesh["elem"], mesh["coef"]
    NT_job = elem.shape[0] * ws  # weak scaling: every rank assembles its own copy of the workload
    if args.shard == "rows" and ws > 1:
        # strong scaling: rank r assembles the rows it owns of the one mesh (no exchange of data)
        from paper_1804_05156_gb300 import partition
        lo, hi = partition.row_ranges(node.shape[0], ws, elem)[rank]
        sh = partition.shard_mesh(elem, lo, hi)
        NT_job = elem.shape[0]
        node, elem = node[sh["vert_ids"]], sh["elem_local"]
        k = None if k is None else k[sh["elem_ids"]]
    N, NT = node.shape[0], elem.shape[0]
    f_name = mesh["f"] if args.f == "workload" else args.f
    f_kind = fa.FEM_F_SINPROD if f_name == "sinprod" else fa.FEM_F_CONST
    variant = fa.FEM_ATOMIC if args.variant == "atomic" else fa.FEM_DETERMINISTIC
    # a slice of the call (stiffness or load alone, or another f) times part of the workload: a
    # diagnostic run, without the e2e, secondary and CPU rows
    diagnostic = args.part != "all" or f_name != mesh["f"]
    s = torch.cuda.current_stream()

    elem_d = torch.as_tensor(elem).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    node_d = torch.as_tensor(node).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p = fa.Pattern(elem_d, N)
    fa.fem_pattern_set_locality(p, node_d)
    torch.cuda.synchronize()
    pattern_ms = 1e3 * (time.perf_counter() - t0)

    k_d = torch.as_tensor(k).cuda() if k is not None else None
    val = torch.empty(p.nnz, dtype=torch.float64, device="cuda")
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def step():
        if args.part == "stiffness":
            fa.fem_assemble_stiffness(p, node_d, k_d, val, variant)
        elif args.part == "load":
            fa.fem_assemble_rhs(p, node_d, f_kind, None, b, variant)
        else:
            fa.fem_assemble(p, node_d, k_d, f_kind, None, val, b, variant)

    for _ in range(args.warmup):
        step()
    fa.get_error()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    fa.fem_timing_report()
    fa.fem_timing_enable(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = fa.launch_count()
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        nvtx = _nvtx(torch)
        nvtx[0]("timed_steps")  # lets a profiler select exactly the timed launches
        for i in range(args.steps):
            flush.zero_()
            evs[i][0].record(s)
            step()
            evs[i][1].record(s)
        nvtx[1]()
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    launches = fa.launch_count() - l0
    fa.fem_timing_enable(False)
    kt = fa.fem_timing_report()
    fa.get_error()
    step_ms = [a.elapsed_time(bb) for a, bb in evs]
    ms = sum(step_ms) / len(step_ms)
    if dist:
        ms = max_over_ranks(dist, ms)
    value = NT_job / (ms * 1e-3) / 1e6

    # roofline of the step's kernels (one or two launches per step, depending on the tuned path):
    # algorithmic bytes of the step / the summed mean durations of the kernels launched every step
    peak, peak_kind = peaks()
    alg = algorithmic_bytes(d, N, NT, p.nnz, args.part)
    per_step = {n: (c, t) for n, (c, t) in kt.items() if c >= args.steps}
    if not per_step:
        per_step = {"step": (args.steps, ms * args.steps)}
    k_ms = sum(t / c for c, t in per_step.values())
    names = sorted(per_step, key=lambda n: -per_step[n][1])
    achieved = alg / (k_ms * 1e-3) / 1e9
    shape = fa.fem_pattern_launch_shape(p)
    path = fa.fem_pattern_value_path(p)
    prof_cfg = args.config if args.grid is None else "%s@%d" % (args.config, args.grid)  # records are per workload
    if diagnostic:
        prof_cfg += "/%s/%s" % (args.part, f_name)
    traffic, traffic_src = profiled(names, prof_cfg, path, shape)
    inst, inst_src = profiled(names, prof_cfg, path, shape, "inst", "warp_inst_per_launch")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_source": traffic_src,
            # the DRAM bytes ncu counted for these kernels over their time here: the rate the memory system
            # ran at, including the design's own traffic (packets, plan arrays), not an efficiency
            "dram_GBs": (traffic / (k_ms * 1e-3) / 1e9) if traffic else None,
            "dram_frac": (traffic / (k_ms * 1e-3) / 1e9 / peak) if traffic else None,
            "kernel": " + ".join(names), "kernel_ms": k_ms,
            "peak_source": peak_kind, "algorithmic_bytes": alg, "step_algorithmic_GBs": alg / (ms * 1e-3) / 1e9,
            "kernels": {n: {"launches": c, "mean_ms": t / c, "share": (t / c) / k_ms} for n, (c, t) in kt.items()}}
    # what does bind the step: instruction issue (the float-float arithmetic runs on the FP32/INT32 pipes).
    # Peak = SMs x 4 schedulers x 1 warp-instruction per clock at the median SM clock sampled during the
    # timed steps; achieved = the ncu-counted warp instructions of the step's kernels / their time.
    clocks = clk.summary()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clocks.get("sm_mhz") or _measured_peaks().get("sm_max_mhz") or 2070.0
    issue_peak = nsm * 4 * mhz * 1e6
    roof["issue"] = {"bound": "alu", "unit": "warp-inst/s", "peak": issue_peak,
                     "peak_basis": "%d SMs x 4 schedulers x 1 warp-instruction/clock at %.0f MHz" % (nsm, mhz),
                     "warp_inst_per_step": inst, "source": inst_src,
                     "achieved": (inst / (k_ms * 1e-3)) if inst else None,
                     "frac": (inst / (k_ms * 1e-3) / issue_peak) if inst else None}

    e2e = None
    if not diagnostic:
        # e2e: host buffers through the C ABI (fem_assemble_host): every step copies its inputs in from
        # page-locked host memory and its outputs (val, b) back; the call pipelines the steps (inputs of
        # step i+1 and outputs of step i-1 in flight while step i computes)
        node_h = torch.as_tensor(node).pin_memory()
        k_h = torch.as_tensor(k).pin_memory() if k is not None else None
        val_hs = [torch.empty(p.nnz, dtype=torch.float64).pin_memory() for _ in range(2)]
        b_hs = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in range(2)]
        e2e_steps = max(3, args.steps)
        nodes_l, ks_l = [node_h] * e2e_steps, [k_h] * e2e_steps
        vals_l = [val_hs[i % 2] for i in range(e2e_steps)]
        bs_l = [b_hs[i % 2] for i in range(e2e_steps)]
        fa.fem_assemble_host(p, nodes_l[:2], ks_l[:2], f_kind, None, vals_l[:2], bs_l[:2], s)  # warm-up
        torch.cuda.synchronize()
        e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_a.record(s)
        fa.fem_assemble_host(p, nodes_l, ks_l, f_kind, None, vals_l, bs_l, s)
        e_b.record(s)
        torch.cuda.synchronize()
        e2e_ms = e_a.elapsed_time(e_b) / e2e_steps
        # the same, one step per call (no overlap between steps)
        one = []
        for i in range(3):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(s)
            fa.fem_assemble_host(p, nodes_l[:1], ks_l[:1], f_kind, None, vals_l[:1], bs_l[:1], s)
            a1.record(s)
            torch.cuda.synchronize()
            one.append(a0.elapsed_time(a1))
        e2e_one_ms = sum(one) / len(one)
        fa.get_error()
        if dist:
            e2e_ms = max_over_ranks(dist, e2e_ms)
            e2e_one_ms = max_over_ranks(dist, e2e_one_ms)
        h2d = node_h.numel() * 8 + (k_h.numel() * 8 if k_h is not None else 0)
        d2h = (p.nnz + N) * 8
        e2e = {"value": NT_job / (e2e_ms * 1e-3) / 1e6, "unit": "Melem/s", "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps,
               "api": "fem_assemble_host (page-locked host buffers, steps pipelined in one call)",
               "one_step_per_call_ms": e2e_one_ms}

    out = {"metric": METRIC, "value": value, "unit": "Melem/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "strong" if (args.shard == "rows" and ws > 1) else "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "arithmetic": ("float-float on the FP32 pipe (pairs of floats, ~2^-48 relative); every FP64 output "
                          "rounded once; within 1e-12 of the FP64 oracle" if args.variant == "deterministic"
                          else "FP64 (atomicAdd in FP64)"),
           "config": {"workload": workload_name(args.config) + ("" if args.grid is None else
                                                                    " (recipe at %d cells per side)" % args.grid),
                      "N": N, "NT": NT, "nnz": p.nnz, "part": args.part, "f": f_name,
                      "variant": args.variant, "l2": "flushed by a 512 MB write between steps (outside timing)",
                      "parallelism": ("single GPU" if ws == 1 else
                                      "row ownership, rank-local rows of one mesh" if args.shard == "rows" else
                                      "independent mesh per rank")},
           "wall_s_timed_region": wall, "pattern_build_ms": pattern_ms,
           "launch_shape": shape,
           "value_path": path,
           "roofline": roof,
           "e2e": e2e,
           "gpu_launches": launches,
           "clocks": clocks}
    if diagnostic:
        print(json.dumps(out), flush=True)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    # secondary timings on the same mesh: atomic variant, boundary + Dirichlet elimination
    fa.fem_assemble(p, node_d, k_d, f_kind, None, val, b, fa.FEM_ATOMIC)
    ms_at = _time_steps(lambda: fa.fem_assemble(p, node_d, k_d, f_kind, None, val, b, fa.FEM_ATOMIC),
                        max(3, min(args.steps, 10)), flush, s)
    isbd = torch.empty(N, dtype=torch.uint8, device="cuda")
    free = torch.empty(N, dtype=torch.int32, device="cuda")

    def dirich():
        fa.fem_boundary_nodes(p, None, isbd)
        fa.fem_apply_dirichlet(p, isbd, None, val, b, free, want_count=False)
    dirich()
    ms_di = _time_steps(dirich, max(3, min(args.steps, 10)), flush, s)
    out["atomic_variant"] = {"ms": ms_at, "Melem_s": NT / (ms_at * 1e-3) / 1e6}
    out["dirichlet_ms"] = ms_di
    if "bdflag" in mesh and args.shard != "rows":
        # Neumann on x = 0 and x = 1, Robin on y = 1, Dirichlet on y = 0 (the mixed problem of Sec. 3.3)
        faces = {"x0": 2, "x1": 2, "y1": 3, "y0": 1, "z0": 2, "z1": 3}
        flags = torch.as_tensor(meshgen.side_flags(mesh, faces)).cuda()
        fa.fem_assemble(p, node_d, k_d, f_kind, None, val, b, variant)
        steps_b = max(3, min(args.steps, 10))
        ms_nr = _time_steps(lambda: fa.fem_boundary_terms(p, node_d, flags, None, 1.0, 1.0, val, b), steps_b, flush, s)
        ms_ms = _time_steps(lambda: fa.fem_mean_shift(b), steps_b, flush, s)
        ms_za = _time_steps(lambda: fa.fem_zero_average(p, node_d, b), steps_b, flush, s)
        out["neumann_robin"] = {"boundary_terms_ms": ms_nr, "mean_shift_ms": ms_ms, "zero_average_ms": ms_za}
        # the other operators on the same pattern: mass matrix (coefficient k) and -div(K grad u)
        Kt = np.array([1.5, 0.2, 0.8]) if d == 2 else np.array([1.5, 0.2, -0.1, 0.8, 0.1, 1.2])
        K_d = torch.as_tensor(np.tile(Kt, (NT, 1))).cuda()
        fa.fem_assemble_operator(p, node_d, fa.FEM_OP_MASS, k_d, val)
        fa.fem_assemble_operator(p, node_d, fa.FEM_OP_ANISO, K_d, val)
        ms_mass = _time_steps(lambda: fa.fem_assemble_operator(p, node_d, fa.FEM_OP_MASS, k_d, val), steps_b, flush, s)
        ms_an = _time_steps(lambda: fa.fem_assemble_operator(p, node_d, fa.FEM_OP_ANISO, K_d, val), steps_b, flush, s)
        fa.get_error()
        out["operators"] = {"mass_ms": ms_mass, "mass_Melem_s": NT / (ms_mass * 1e-3) / 1e6,
                            "aniso_ms": ms_an, "aniso_Melem_s": NT / (ms_an * 1e-3) / 1e6}
        # the load vector with the 3-point-per-direction conical rule (exact to degree 5)
        fa.fem_assemble_rhs_rule(p, node_d, 3, f_kind, None, b)
        ms_rule = _time_steps(lambda: fa.fem_assemble_rhs_rule(p, node_d, 3, f_kind, None, b), steps_b, flush, s)
        out["operators"]["rhs_rule3_ms"] = ms_rule
        # y = A u matrix-free, next to a library CSR SpMV (cuSPARSE through torch) of the assembled A
        u_d = torch.as_tensor(meshgen.normal(5, 5, N)).cuda()
        y_d = torch.empty_like(u_d)
        fa.fem_apply_stiffness(p, node_d, k_d, u_d, None, y_d)
        ms_ap = _time_steps(lambda: fa.fem_apply_stiffness(p, node_d, k_d, u_d, None, y_d), steps_b, flush, s)
        fa.fem_assemble(p, node_d, k_d, f_kind, None, val, b, variant)
        import warnings
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            A_csr = torch.sparse_csr_tensor(p.row_ptr.long(), p.col_idx.long(), val, size=(N, N))
        ms_sp = _time_steps(lambda: torch.mv(A_csr, u_d), steps_b, flush, s)
        fa.get_error()
        out["operators"]["apply_ms"] = ms_ap
        out["operators"]["apply_Melem_s"] = NT / (ms_ap * 1e-3) / 1e6
        out["operators"]["assembled_spmv_cusparse_ms"] = ms_sp
        del A_csr, u_d, y_d
        # matrix-free CG on the reduced system (Sec. 3.3; whole boundary, g_D = 0): a fixed iteration count
        # (rtol 0), so the rate does not depend on convergence; the call synchronises every 8 iterations
        fa.fem_boundary_nodes(p, None, isbd)
        fa.fem_assemble(p, node_d, k_d, f_kind, None, val, b, variant)
        u_cg = torch.empty(N, dtype=torch.float64, device="cuda")
        fa.fem_cg_solve(p, node_d, k_d, isbd, b, None, u_cg, max_iter=8, rtol=0.0)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, its, rel = fa.fem_cg_solve(p, node_d, k_d, isbd, b, None, u_cg, max_iter=64, rtol=0.0)
        torch.cuda.synchronize()
        cg_ms = 1e3 * (time.perf_counter() - t0)
        fa.get_error()
        it_ms = cg_ms / max(its, 1)
        it_bytes = cg_iteration_bytes(d, N, NT)
        # the same iterations on the assembled matrix (val of this call): CSR product instead of recomputing
        fa.fem_cg_solve_csr(p, val, isbd, b, None, u_cg, max_iter=8, rtol=0.0)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, its_c, _ = fa.fem_cg_solve_csr(p, val, isbd, b, None, u_cg, max_iter=64, rtol=0.0)
        torch.cuda.synchronize()
        cgc_ms = 1e3 * (time.perf_counter() - t0)
        fa.get_error()
        itc_ms = cgc_ms / max(its_c, 1)
        itc_bytes = cg_csr_iteration_bytes(N, p.nnz)
        out["cg_iterations"] = {"iterations": its, "ms": cg_ms, "ms_per_iteration": it_ms,
                                "iterations_per_s": 1e3 / it_ms, "relres_after": rel,
                                "algorithmic_bytes_per_iteration": it_bytes,
                                "hbm_frac": it_bytes / (it_ms * 1e-3) / 1e9 / peak, "peak_GBs": peak,
                                "assembled": {"api": "fem_cg_solve_csr", "iterations": its_c, "ms": cgc_ms,
                                              "ms_per_iteration": itc_ms, "iterations_per_s": 1e3 / itc_ms,
                                              "algorithmic_bytes_per_iteration": itc_bytes,
                                              "hbm_frac": itc_bytes / (itc_ms * 1e-3) / 1e9 / peak},
                                "timing": "wall clock around one call (lift and start included, host "
                                          "convergence tests every 8 iterations)"}
        del u_cg
        del K_d
    if not args.no_extras and ws == 1:
        out["extras"] = extras(fa, args, flush, value)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(mesh, 1 if mesh["f"] == "sinprod" else 0, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=["c1", "c2", "c3"], default="c2")
    ap.add_argument("--variant", choices=["deterministic", "atomic"], default="deterministic")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the 3-D, batched and fwd+bwd rows")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-sample", type=int, default=400_000)
    ap.add_argument("--grid", type=int, default=None,
                    help="cells per side instead of the workload's own (the same recipe at another size; for profiling "
                         "captures on a smaller case)")
    ap.add_argument("--part", choices=["all", "stiffness", "load"], default="all",
                    help="time the whole call (default), or the stiffness or the load vector alone (diagnostic)")
    ap.add_argument("--f", choices=["workload", "const", "sinprod"], default="workload",
                    help="the workload's load function (default) or another one (diagnostic)")
    ap.add_argument("--shard", choices=["copies", "rows"], default="copies",
                    help="N>1: every rank assembles its own copy (weak scaling) or its rows of one mesh (strong)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
