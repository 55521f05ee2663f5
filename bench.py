"""Benchmark: plain random walker on the 256^3 three-ellipsoid phantom.

One step = one complete rw_solve (normalisation/quantisation, FP32 PCG with
FP64 reductions, FP64-residual refinement to ||r|| <= 1e-8 ||b||) on inputs
already resident in HBM.  Metric: voxel-CG-iterations/s = sum over the step of
free voxels x PCG iterations, divided by the device time (CUDA events, max
over ranks).  The 256^3 working set streamed per sweep (about 470 MB) is
larger than L2, so no flush is needed between steps.

Beside the headline (one GPU, rank 0): the FP64 oracle's solve of the same
system, run on the host cores in a spawned process while the GPU works, gives
max_abs_err_vs_oracle for the timed step's output; `secondary` holds the
hierarchical 1024^3 vessel-tree workload (brick 32) with its roofline and the
batched mixed-precision vs per-brick FP64 comparison on its own leaf level.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload plain|hier|adjoint|multiclass|bricks]

--impl reference times the FP64 CPU oracle (test infrastructure, as it
stands) on the host cores: each step is a bounded number of its PCG
iterations on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-CG-iterations/s and HBM GB/s (% of peak) at <=1e-4 prob error vs FP64"
UNIT = "voxel-iter/s"
BETA = 130.0
TOL = 1e-8
# algorithmic bytes per voxel-iteration (the method's minimum in mixed
# precision): x, r, p FP32 read + written (24 B), unorm16 g (2 B), seed code
# (1 B).  The sweep kernel itself moves 28 B (g and code packed in one word).
SWEEP_BYTES_PER_VOXEL = 27
KERNEL_BYTES_PER_VOXEL = 28
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_sweep5
# launch on the 256^3 workload, per tile, from one ncu capture of that tile
# (`ncu --set full -k regex:k_sweep5 -s 40 -c 1` over `bench.py --steps 2
# --warmup 3 --no-cpu-baseline --no-oracle-check --no-secondary --e2e-steps 0
# --tile <tile>`).  Valid only for the sweep sources they were measured on
# (SHA-256 of the files below, first 16 hex digits); any other source, or a
# tile without a capture, gives traffic null.
SWEEP_SOURCES = ("paper_2103_09564_gb300/csrc/sweep5_kernel.cuh", "paper_2103_09564_gb300/csrc/sweep5_f32.cu",
                 "paper_2103_09564_gb300/csrc/sweep_kernel.cuh")
SWEEP_TRAFFIC_256 = {"sha": "514747d189580643", "bytes": {"r64x14_d2": 432.51e6}}


def _sweep_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _sweep_traffic(tile_name, n):
    if n != 256 or SWEEP_TRAFFIC_256["sha"] != _sweep_source_sha():
        return None
    return SWEEP_TRAFFIC_256["bytes"].get(tile_name)


def _workload(n):
    return f"plain random walker, {n}^3 three-ellipsoid phantom (phantoms.plain_ellipsoids, seed 0), beta 130"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            p = [v.strip() for v in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _aggregate(pg, ms, vi, dev):
    """Whole-job figures over the ranks of process group `pg` (None: one
    rank): the slowest rank's time and the sum of the voxel-iterations."""
    if pg is None:
        return ms, float(vi)
    import torch
    t = torch.tensor([ms, float(vi)], device=dev, dtype=torch.float64)
    tm = t.clone()
    pg.all_reduce(tm, op=pg.ReduceOp.MAX)
    ts = t.clone()
    pg.all_reduce(ts, op=pg.ReduceOp.SUM)
    return float(tm[0]), float(ts[1])


def _cpu_baseline(c, seconds=15.0):
    """The FP64 oracle as it stands on the host cores, on a bounded sample:
    its first M PCG iterations on the same 256^3 system (M sized to ~seconds)."""
    import oracle as O
    q = O.quantize(c["volume"])
    g = O.dequantize(q)
    xin = np.where(c["code"] == 1, c["value"].astype(np.float64), 0.0)
    nfree = int(np.count_nonzero(c["code"] == 0))
    t0 = time.perf_counter()
    O.rw_solve(g, c["code"], xin, BETA, tol=1e-13, max_iter=5)
    t1 = time.perf_counter()
    per = max((t1 - t0) / 6.0, 1e-3)           # ~ setup + 5 iterations
    m = int(max(5, min(2000, seconds / per)))
    t0 = time.perf_counter()
    _, it, _, _ = O.rw_solve(g, c["code"], xin, BETA, tol=1e-13, max_iter=m)
    dt = time.perf_counter() - t0
    return {"value": nfree * it / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle Jacobi-PCG, first {it} iterations of the {c['volume'].shape[0]}^3 system ({nfree} free voxels), "
                      f"{dt:.1f} s incl. weight set-up"}


def _oracle_solve_child(n, threads, path):
    """Child process (spawned): the FP64 oracle's solve of the benchmark system
    as it stands (tol 1e-13), written to `path` as FP64 .npy."""
    os.environ["OMP_NUM_THREADS"] = str(threads)
    sys.path.insert(0, ROOT)
    import oracle as O
    import phantoms as P
    c = P.plain_ellipsoids(n=n, seed=0)
    x, it, rr, st = O.solve_volume(c["volume"], c["code"], c["value"], BETA)
    np.save(path, x)
    with open(path + ".json", "w") as f:
        json.dump({"iters": it, "rel_resid": rr, "status": st, "threads": threads}, f)


class OracleCheck:
    """The FP64 oracle's solution of the benchmark system, computed in a
    spawned process on the host cores while the GPU runs (started before the
    first GPU call); compared with the GPU result after the timed region."""

    def __init__(self, n):
        import multiprocessing as mp
        import tempfile
        self.dir = tempfile.mkdtemp(prefix="rw_oracle_")
        self.path = os.path.join(self.dir, "x.npy")
        self.threads = max(1, (os.cpu_count() or 2) - 2)   # two cores left to the GPU's host thread
        self.t0 = time.perf_counter()
        self.proc = mp.get_context("spawn").Process(target=_oracle_solve_child, args=(n, self.threads, self.path),
                                                    daemon=True)
        self.proc.start()

    def result(self, x_gpu, timeout=1800):
        self.proc.join(timeout)
        wall = time.perf_counter() - self.t0
        try:
            if self.proc.is_alive() or self.proc.exitcode != 0:
                if self.proc.is_alive():
                    self.proc.terminate()
                return {"max_abs_err": None, "why": f"oracle process failed (exit {self.proc.exitcode})"}
            xo = np.load(self.path)
            with open(self.path + ".json") as f:
                info = json.load(f)
            d = np.abs(x_gpu.astype(np.float64) - xo)
            far = np.abs(xo - 0.5) > 1e-3
            return {"max_abs_err": float(d.max()), "mean_abs_err": float(d.mean()),
                    "label_mismatches_far_from_half": int(np.count_nonzero((x_gpu[far] > 0.5) != (xo[far] > 0.5))),
                    "voxels_far_from_half": int(np.count_nonzero(far)),
                    "oracle": f"FP64 Jacobi-PCG to 1e-13 ({info['iters']} iterations, rel. residual "
                              f"{info['rel_resid']:.2e}, {info['threads']} threads, {wall:.0f} s wall)",
                    "gpu_output": "the last timed step's x (FP32)"}
        finally:
            for f in (self.path, self.path + ".json"):
                if os.path.exists(f):
                    os.remove(f)
            os.rmdir(self.dir)


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import phantoms as P
    import oracle as O
    N = args.n or 256
    c = P.plain_ellipsoids(n=N, seed=0)
    q = O.quantize(c["volume"])
    g = O.dequantize(q)
    xin = np.where(c["code"] == 1, c["value"].astype(np.float64), 0.0)
    nfree = int(np.count_nonzero(c["code"] == 0))
    iters_per_step = 20
    for _ in range(args.warmup):
        O.rw_solve(g, c["code"], xin, BETA, tol=1e-13, max_iter=2)
    tot_it, t0 = 0, time.perf_counter()
    for _ in range(args.steps):
        _, it, _, _ = O.rw_solve(g, c["code"], xin, BETA, tol=1e-13, max_iter=iters_per_step)
        tot_it += it
    dt = time.perf_counter() - t0
    v = nfree * tot_it / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload(N), "voxels": N ** 3, "free_voxels": nfree,
                       "step": f"{iters_per_step} FP64 PCG iterations of the oracle (plus its weight set-up)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"{iters_per_step} iterations per step x {args.steps} steps"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    import paper_2103_09564_gb300 as rw
    import phantoms as P
    N = args.n or 256
    c = P.plain_ellipsoids(n=N, seed=0)
    solo = ws == 1 and rank == 0
    cpu_base = _cpu_baseline(c) if solo and not args.no_cpu_baseline else None
    check = OracleCheck(N) if solo and not args.no_oracle_check else None
    vol = torch.from_numpy(c["volume"]).to(dev)
    code = torch.from_numpy(c["code"]).to(dev)
    val = torch.from_numpy(c["value"]).to(dev)
    out = torch.empty_like(vol)
    opts = rw.Opts(beta=BETA, tol=TOL, tile=args.tile)

    def step():
        _, st = rw.rw_solve(vol, code, val, opts, out=out)
        return st

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    stats = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            stats.append(step())
        e1.record()
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms = e0.elapsed_time(e1)
    vi = sum(s["voxel_iters"] for s in stats)
    sweeps = sum(s["sweeps"] for s in stats)
    ms_sweeps = sum(s["ms_sweeps"] for s in stats)
    launches = sum(s["launches"] for s in stats)
    ms_all, vi_all = _aggregate(pg, ms, vi, dev)
    value = vi_all / (ms_all / 1e3)

    # end to end through the C ABI with pinned host buffers (the library's
    # copies in and out inside the timed region)
    vol_h = torch.from_numpy(np.ascontiguousarray(c["volume"])).pin_memory()
    code_h = torch.from_numpy(np.ascontiguousarray(c["code"])).pin_memory()
    val_h = torch.from_numpy(np.ascontiguousarray(c["value"])).pin_memory()
    out_h = torch.empty(vol_h.shape, dtype=vol_h.dtype, pin_memory=True)
    e2e_steps = max(0, min(args.steps, args.e2e_steps))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    vi_e2e = 0
    for _ in range(e2e_steps):
        _, st = rw.rw_solve(vol_h, code_h, val_h, opts, out=out_h)
        vi_e2e += st["voxel_iters"]
    t_e2e = time.perf_counter() - t0
    e2e = {"value": vi_e2e / t_e2e if e2e_steps else None, "unit": UNIT,
           "h2d_bytes_per_step": int(sum(t.numel() * t.element_size() for t in (vol_h, code_h, val_h))),
           "d2h_bytes_per_step": int(out_h.numel() * out_h.element_size()), "host_memory": "pinned"}

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0
    peak, src = _peaks()
    tile_name = {v: k for k, v in rw._abi.RW_TILE.items()}.get(stats[0]["tile"], str(stats[0]["tile"]))
    # sweeps that did work: the PCG iterations plus the restart / replacement
    # sweep that opens each refinement round (launches after convergence exit
    # at once; their time stays in ms_sweeps, which makes this conservative)
    work_sweeps = sum(s["iters"] + s["refine_rounds"] for s in stats)
    t_launch_s = (ms_sweeps / max(work_sweeps, 1)) / 1e3
    alg = SWEEP_BYTES_PER_VOXEL * int(stats[0]["free_voxels"])
    achieved = alg / t_launch_s / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": _workload(N), "voxels": N ** 3, "free_voxels": int(stats[0]["free_voxels"]),
                       "precision": "FP32 vectors/stencil, FP64 reductions + FP64-residual refinement",
                       "tol": TOL, "iters_per_solve": stats[0]["iters"], "refine_rounds": stats[0]["refine_rounds"],
                       "rel_resid": stats[0]["rel_resid"], "replicas": ws,
                       "tile": tile_name,
                       "sweeps_per_graph": stats[0]["iters_per_graph"],
                       "l2": "inputs larger than L2 (about 470 MB streamed per sweep), no flush"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": _sweep_traffic(tile_name, N),
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of this "
                                           "tile on the 256^3 workload, taken on the current sweep sources "
                                           "(null when they changed since)",
                         "kernel": "k_sweep5 (fused PCG sweep)", "peak_source": src,
                         "algorithmic_bytes_per_launch": alg, "basis": "27 B per free voxel per sweep",
                         "kernel_bytes_per_voxel": KERNEL_BYTES_PER_VOXEL, "launch_ms": t_launch_s * 1e3,
                         "sweeps_per_step": sweeps / args.steps, "work_sweeps_per_step": work_sweeps / args.steps},
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary()}
    if cpu_base is not None:
        line["cpu_baseline"] = cpu_base
    if solo and not args.no_secondary and N == 256:
        line["secondary"] = {"hierarchical_1024": _hier_secondary(rw, P, torch, dev, peak, src, args)}
    if check is not None:
        line["max_abs_err_vs_oracle"] = check.result(out.cpu().numpy())
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def _hier_secondary(rw, P, torch, dev, peak, src, args):
    """The hierarchical workload beside the headline: the 1024^3 uint16 vessel
    tree, brick 32, pruning hom + dt, bricks solved to 1e-10 (the tolerance
    of the hierarchy parity tests); one step = a full top-down run.  Then its
    own leaf level solved twice from the same parent levels: batched
    mixed-precision launches (the default) and the plain per-brick FP64 solve
    (one brick per launch), both to 1e-10."""
    s, tol, n = 32, 1e-10, 1024
    ph = P.vessel_tree(n=n, seed=0, device=dev)
    xyz, val = _labels_np(ph)
    pyr = rw.rw_build_pyramid(ph["volume"], s, lo=0.0, hi=5000.0, normalize=True)
    del ph
    torch.cuda.empty_cache()
    tree = rw.Tree(pyr, rw.Opts(brick_size=s, beta=BETA, tol=tol))
    for _ in range(3):
        tree.run(xyz, val)
    torch.cuda.synchronize()
    steps = max(3, min(args.steps, 10))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record()
    for _ in range(steps):
        stats.append(tree.run(xyz, val))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    vi = sum(st["voxel_iters"] for st in stats)
    sweep_ms = sum(st["ms_sweeps"] for st in stats)
    eff = SWEEP_BYTES_PER_VOXEL * vi / (sweep_ms / 1e3) / 1e9 if sweep_ms > 0 else None
    K = pyr.levels - 1
    leaf = {}
    res = {}
    for name, kw in (("batched_mixed", {}), ("per_brick_fp64", {"batch_bricks": 0, "precision": "fp64"})):
        t = tree if not kw else rw.Tree(pyr, rw.Opts(brick_size=s, beta=BETA, tol=tol, **kw))
        for k in range(K):       # the parent levels (the batched solve's) before the timed leaf level
            t.refine_level(k, xyz if k == 0 else None, val if k == 0 else None)
        torch.cuda.synchronize()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record()
        st = t.refine_level(K)
        eb.record()
        torch.cuda.synchronize()
        lms = ea.elapsed_time(eb)
        res[name] = {"leaf_bricks_solved": st["bricks_solved"], "leaf_voxel_iters": st["voxel_iters"],
                     "leaf_ms": lms, "voxel_iter_per_s": st["voxel_iters"] / (lms / 1e3) if lms > 0 else None,
                     "max_rel_resid": st["rel_resid"], "not_converged": st["not_converged"]}
        leaf[name] = torch.empty(tuple(reversed(pyr.dims[K])), dtype=torch.float32, device=dev)
        t.read_level(K, out=leaf[name])
        if kw:
            t.free()
    a, b = res["batched_mixed"]["voxel_iter_per_s"], res["per_brick_fp64"]["voxel_iter_per_s"]
    diff = (leaf["batched_mixed"] - leaf["per_brick_fp64"]).abs()
    res["speedup"] = (a / b) if a and b else None
    res["max_abs_diff_leaf"] = float(diff.max())
    res["voxels_diff_above_1e-4"] = int((diff > 1e-4).sum())
    res["accuracy"] = "both solve every leaf brick to ||r|| <= 1e-10 ||b|| (FP64 true residual)"
    tree.free()
    pyr.free()
    torch.cuda.empty_cache()
    return {"workload": f"hierarchical random walker, {n}^3 uint16 vessel tree (phantoms.vessel_tree, seed 0, "
                        f"200 segments), brick {s}, e 1.25, pruning hom+dt, tol {tol}",
            "value": vi / (ms / 1e3), "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
            "bricks_solved_per_run": stats[0]["bricks_solved"], "bricks_pruned_per_run": stats[0]["bricks_pruned"],
            "gpu_launches_per_run": stats[0]["launches"],
            "roofline": {"bound": "hbm", "achieved": eff, "peak": peak, "unit": "GB/s",
                         "frac": (eff / peak) if eff else None, "traffic": None, "peak_source": src,
                         "kernel": "fused PCG sweeps over the brick batches (device time of the sweeps)",
                         "basis": "27 B per free-voxel iteration"},
            "leaf_batched_vs_per_brick_fp64": res}


def _labels_np(ph):
    return np.asarray(ph["labels_xyz"], dtype=np.float64), np.asarray(ph["labels_value"], dtype=np.float32)


def run_hier(args):
    """Hierarchical random walker on the vessel-tree phantom (n^3 uint16,
    window [0, 5000]): one step = a full top-down run of all levels
    (batched brick solves with pruning).  Beside it, the leaf level of a
    256^3 phantom is solved twice from the same parent levels: batched FP32
    sweeps (the default) and the per-brick FP64 solve, one brick per launch."""
    import torch
    import paper_2103_09564_gb300 as rw
    import phantoms as P
    n = args.n or 1024
    s = args.brick
    dev = torch.device("cuda", 0)
    ph = P.vessel_tree(n=n, seed=0, device=dev)
    xyz, val = _labels_np(ph)
    torch.cuda.synchronize()
    rw.release_workspace()
    free0 = torch.cuda.mem_get_info(dev)[0]
    pyr = rw.rw_build_pyramid(ph["volume"], s, lo=0.0, hi=5000.0, normalize=True, leaf_in_host=args.leaf_host,
                              all_in_host=args.all_host)
    opts = rw.Opts(brick_size=s, beta=BETA, tol=args.tol)
    tree = rw.Tree(pyr, opts)
    rw.release_workspace()
    dev_bytes = free0 - torch.cuda.mem_get_info(dev)[0]     # what the pyramid and the tree hold in HBM
    level_vox = [x * y * z for x, y, z in pyr.dims]
    held = {"pyramid_bytes": 2 * level_vox[-1] + 4 * sum(level_vox[:-1]), "tree_field_bytes": 4 * sum(level_vox),
            "device_bytes_of_pyramid_and_tree": int(dev_bytes)}
    del ph
    torch.cuda.empty_cache()
    for _ in range(max(3, args.warmup)):
        tree.run(xyz, val)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    with Clocks(0) as clk:
        e0.record()
        for _ in range(args.steps):
            stats.append(tree.run(xyz, val))
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    vi = sum(st["voxel_iters"] for st in stats)
    sweep_ms = sum(st["ms_sweeps"] for st in stats)
    per_level = []
    for k in range(pyr.levels):
        fl, mn, mx, md = tree.node_stats(k)
        per_level.append({"level": k, "dims": pyr.dims[k], "solved": int(np.count_nonzero(fl & rw.RW_NODE_SOLVED)),
                          "prunable": int(np.count_nonzero(fl & rw.RW_NODE_PRUNABLE)),
                          "conflict": int(np.count_nonzero(fl & rw.RW_NODE_CFL))})
    # batched mixed vs per-brick FP64 on the leaf level of a 256^3 phantom
    cmp = _compare_batched_vs_fp64(rw, P, s, args.tol)
    peak, src = _peaks()
    eff = SWEEP_BYTES_PER_VOXEL * vi / (sweep_ms / 1e3) / 1e9 if sweep_ms > 0 else None
    line = {"metric": METRIC, "value": vi / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"hierarchical random walker, {n}^3 uint16 vessel tree (phantoms.vessel_tree, "
                                   f"seed 0, 200 segments), brick {s}, e 1.25, pruning hom+dt, tol {args.tol}"
                                   + (", leaf level in host memory" if args.leaf_host else "")
                                   + (", every level in host memory" if args.all_host else ""),
                       "memory": held,
                       "levels": per_level, "bricks_solved_per_run": stats[0]["bricks_solved"],
                       "bricks_pruned_per_run": stats[0]["bricks_pruned"], "labels": int(len(val))},
            "roofline": {"bound": "hbm", "achieved": eff, "peak": peak, "unit": "GB/s",
                         "frac": (eff / peak) if eff else None, "traffic": None,
                         "kernel": "fused PCG sweep over the brick batches",
                         "basis": "27 B per free-voxel iteration / device time of the sweeps", "peak_source": src},
            "batched_vs_per_brick_fp64": cmp, "gpu_launches": int(sum(st["launches"] for st in stats)),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_bricks(args):
    """Batched brick solves, the unit of work of a hierarchy level: n systems
    (default 200) of 40^3 voxels (brick 32 with its 1.25 neighbourhood), each
    a noisy ball or ellipsoid (phantoms.ball_case, seeds 0..n-1), beta 130,
    solved together to tol (default 1e-10).  One step = one batched solve:
    full-batch sweeps, then looped sweeps and the cluster-resident solver as
    the systems converge."""
    import torch
    import paper_2103_09564_gb300 as rw
    import phantoms as P
    nb = args.n or 200
    cs = [P.ball_case(n=40, seed=s, radius=10.0 + (s % 5), ellipsoid=(s % 2 == 1)) for s in range(nb)]
    dev = torch.device("cuda", 0)
    vol, code, val = (torch.from_numpy(np.stack([c[k] for c in cs])).to(dev) for k in ("volume", "code", "value"))
    opts = rw.Opts(beta=BETA, tol=args.tol, tile=args.tile)
    for _ in range(max(3, args.warmup)):
        rw.rw_solve(vol, code, val, opts)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    with Clocks(0) as clk:
        e0.record()
        for _ in range(args.steps):
            stats.append(rw.rw_solve(vol, code, val, opts)[1])
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    vi = sum(st["voxel_iters"] for st in stats)
    sweep_ms = sum(st["ms_sweeps"] for st in stats)
    peak, src = _peaks()
    eff = SWEEP_BYTES_PER_VOXEL * vi / (sweep_ms / 1e3) / 1e9 if sweep_ms > 0 else None
    tile_name = {v: k for k, v in rw._abi.RW_TILE.items()}.get(stats[0]["tile"], str(stats[0]["tile"]))
    line = {"metric": METRIC, "value": vi / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"batched brick solves, {nb} systems of 40^3 (phantoms.ball_case, seeds 0..{nb - 1}), "
                                   f"beta {BETA}, tol {args.tol}",
                       "iters": stats[0]["iters"], "sweeps": stats[0]["sweeps"], "tile": tile_name,
                       "free_voxels": stats[0]["free_voxels"], "rel_resid": stats[0]["rel_resid"]},
            "roofline": {"bound": "hbm", "achieved": eff, "peak": peak, "unit": "GB/s",
                         "frac": (eff / peak) if eff else None, "traffic": None,
                         "kernel": "fused PCG sweeps over the brick batch (device time of the sweeps)",
                         "basis": "27 B per free-voxel iteration", "peak_source": src},
            "gpu_launches": int(sum(st["launches"] for st in stats)), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def _compare_batched_vs_fp64(rw, P, s, tol):
    ph = P.vessel_tree(n=256, seed=1, n_segments=60)
    xyz, val = _labels_np(ph)
    pyr = rw.rw_build_pyramid(ph["volume"], s, lo=0.0, hi=5000.0, normalize=True)
    res = {}
    leaf = {}
    for name, kw in (("batched_mixed", {}), ("per_brick_fp64", {"batch_bricks": 0, "precision": "fp64"})):
        t = rw.Tree(pyr, rw.Opts(brick_size=s, beta=BETA, tol=tol, **kw))
        t.run(xyz, val)                       # warm-up (and autotuning)
        st = None
        for k in range(pyr.levels):
            st = t.refine_level(k, xyz if k == 0 else None, val if k == 0 else None)
        res[name] = {"leaf_voxel_iters": st["voxel_iters"], "leaf_ms": st["ms"], "leaf_bricks": st["bricks_solved"],
                     "voxel_iter_per_s": st["voxel_iters"] / (st["ms"] / 1e3) if st["ms"] > 0 else None}
        leaf[name] = t.read_level(pyr.levels - 1)
    a, b = res["batched_mixed"]["voxel_iter_per_s"], res["per_brick_fp64"]["voxel_iter_per_s"]
    res["speedup"] = (a / b) if a and b else None
    res["max_abs_diff_leaf"] = float(np.max(np.abs(leaf["batched_mixed"] - leaf["per_brick_fp64"])))
    res["workload"] = f"leaf level of the 256^3 vessel phantom (seed 1), brick {s}"
    return res


def run_adjoint(args):
    """Differentiable solve on a batch of 32 volumes of 96^3 (balls / random
    ellipsoids): one step = forward solve + adjoint solve + gradient kernel."""
    import torch
    import paper_2103_09564_gb300 as rw
    import phantoms as P
    n = args.n or 96
    b = P.adjoint_batch(n=n, batch=32)
    dev = torch.device("cuda", 0)
    g = torch.from_numpy(b["volume"]).to(dev)
    code = torch.from_numpy(b["code"]).to(dev)
    val = torch.from_numpy(b["value"]).to(dev)
    y = torch.from_numpy(b["mask"].astype(np.float32)).to(dev)
    opts = rw.Opts(beta=BETA, tol=args.tol)

    def step():
        x, s1 = rw.rw_solve(g, code, val, opts, storage=rw.RW_STORE_F32)
        inter = (x * y).sum(dim=(1, 2, 3))
        ssum = x.sum(dim=(1, 2, 3)) + y.sum(dim=(1, 2, 3))
        num = 2 * inter + 1e-6
        den = ssum + 1e-6
        dl = ((num[:, None, None, None] - 2 * y * den[:, None, None, None]) /
              (den[:, None, None, None] ** 2)) / x.shape[0]
        dg, db, s2 = rw.rw_solve_adjoint(g, code, x, dl.contiguous(), opts)
        return s1, s2

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = []
    with Clocks(0) as clk:
        e0.record()
        for _ in range(args.steps):
            st.append(step())
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    vi = sum(a["voxel_iters"] + c["voxel_iters"] for a, c in st)
    line = {"metric": METRIC, "value": vi / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"differentiable random walker, 32 x {n}^3 (phantoms.adjoint_batch), forward + "
                                   f"adjoint per step, soft-Dice loss, tol {args.tol}",
                       "forward_iters": st[0][0]["iters"], "adjoint_iters": st[0][1]["iters"]},
            "gpu_launches": int(sum(a["launches"] + c["launches"] for a, c in st)), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_multiclass(args):
    """Incremental multi-class hierarchy: one tree per class (vessel tree,
    cell blobs, background) on one pyramid, hom-only pruning.  Initial solve
    from three 200-voxel strokes per class; then each step adds one stroke of
    a random class: all three trees are updated together (Sec. IV-E;
    rw_update_seeds_trees: their bricks share batched solves) and the argmax
    labels of the leaf are recomputed on the leaf bricks that changed in any
    tree (after one full-leaf argmax of the initial solve).  Default volume 1024 x 1024 x 2048
    (x, y, z); --n 2048 runs the full 2048 x 2048 x 4096 workload (three
    trees of 78.5 GB and 17 GB of labels in HBM, the pyramid's 34 GB leaf in
    host memory, batches of --max-batch bricks)."""
    import torch
    import paper_2103_09564_gb300 as rw
    import phantoms as P
    shape = (2 * args.n, args.n, args.n) if args.n else (2048, 1024, 1024)
    s = args.brick
    dev = torch.device("cuda", 0)
    n_up = max(3, args.warmup) + args.steps
    t0 = time.perf_counter()
    c = P.multiclass_case(shape, seed=0, n_segments=200, n_blobs=400, n_updates=n_up, device=dev)
    t_phantom = time.perf_counter() - t0
    torch.cuda.empty_cache()  # the library allocates outside torch's cache
    nvox = shape[0] * shape[1] * shape[2]
    # full size: the leaf intensities (read only by the leaf-level gathers) in
    # host memory, so that the trees and the labels fit in HBM
    leaf_host = args.leaf_host or nvox > (1 << 32)
    pyr = rw.rw_build_pyramid(c["volume"], s, lo=0.0, hi=5000.0, normalize=True, leaf_in_host=leaf_host)
    del c["volume"]
    torch.cuda.empty_cache()
    kw = {"max_batch": args.max_batch} if args.max_batch else {}
    opts = rw.Opts(brick_size=s, beta=BETA, tol=args.tol, prune_hom=1, prune_dt=0, leaf_field="hbm", **kw)
    trees = [rw.Tree(pyr, opts) for _ in range(3)]
    labels = torch.empty(shape, dtype=torch.uint8, device=dev)
    free_after_trees = torch.cuda.mem_get_info(dev)[0] / 1e9
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, t in enumerate(trees):
        t.run(*P.class_labels(c["strokes"], k))
    rw.trees_argmax(trees, out=labels)
    torch.cuda.synchronize()
    t_init = time.perf_counter() - t0

    def update(stroke):
        # the three trees updated together (their bricks share batched solves)
        xyz, cls = stroke
        vals = [np.full(len(xyz), 1.0 if k == cls else 0.0, np.float32) for k in range(len(trees))]
        st = [rw.update_trees(trees, xyz, vals, np.full(len(xyz), cls, np.int32))]
        rw.trees_argmax_changed(trees, labels)  # relabel the leaf bricks that changed
        return st

    ups = c["updates"]
    for i in range(max(3, args.warmup)):
        update(ups[i])
    torch.cuda.synchronize()
    lat, stats = [], []
    with Clocks(0) as clk:
        for i in range(max(3, args.warmup), n_up):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            stats.append(update(ups[i]))
            e1.record()
            torch.cuda.synchronize()
            lat.append(e0.elapsed_time(e1))
    ms = float(np.sum(lat))
    vi = sum(x["voxel_iters"] for st in stats for x in st)
    # sampled check of the leaf labels kept up to date brick by brick: the
    # argmax of the three trees' own fields on 8 boxes of 32^3
    rs = np.random.default_rng(0)
    lab_np = labels.cpu().numpy()
    n_chk = n_bad = 0
    for _ in range(8):
        z0, y0, x0 = (int(rs.integers(0, d - 32 + 1)) for d in shape)
        box = [x0, y0, z0, x0 + 32, y0 + 32, z0 + 32]
        f = np.stack([t.read_level(pyr.levels - 1, box=box) for t in trees])
        ref = np.argmax(f, axis=0).astype(np.uint8)
        got = lab_np[z0:z0 + 32, y0:y0 + 32, x0:x0 + 32]
        n_chk += ref.size
        n_bad += int(np.count_nonzero(ref != got))
    # one full-leaf argmax on its own, for comparison
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record()
    rw.trees_argmax(trees, out=labels)
    eb.record()
    torch.cuda.synchronize()
    argmax_ms = ea.elapsed_time(eb)
    line = {"metric": METRIC, "value": vi / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "labels_check": {"voxels": n_chk, "mismatches": n_bad, "how": "argmax of the trees' fields on 8 "
                                                                              "random 32^3 leaf boxes"},
            "config": {"workload": f"incremental 3-class hierarchical random walker, {shape[2]} x {shape[1]} x "
                                   f"{shape[0]} uint16 (phantoms.multiclass_case, seed 0), brick {s}, hom pruning, "
                                   f"tol {args.tol}; one step = one added stroke: 3 tree updates + argmax "
                                   f"over the changed leaf bricks"
                                   + (" (leaf intensities in host memory; trees and labels in HBM)" if leaf_host else "")
                                   + (f", batches of {args.max_batch} bricks" if args.max_batch else ""),
                       "update_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                             "max": float(np.max(lat))},
                       "leaf_voxels_per_s": nvox / (float(np.median(lat)) / 1e3),
                       "initial_solve_s": t_init, "phantom_s": t_phantom,
                       "device_free_gb_after_trees": free_after_trees,
                       "tree_ms_per_update": float(np.mean([sum(x["ms"] for x in st) for st in stats])),
                       "pcg_loop_ms_per_update": float(np.mean([sum(x["ms_solve"] for x in st) for st in stats])),
                       "sweep_ms_per_update": float(np.mean([sum(x["ms_sweeps"] for x in st) for st in stats])),
                       "full_leaf_argmax_ms": argmax_ms,
                       "bricks_resolved_per_update": float(np.mean([sum(x["bricks_solved"] for x in st)
                                                                    for st in stats]))},
            "gpu_launches": int(sum(x["launches"] for st in stats for x in st)), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the FP64 oracle solve of the benchmark system (max_abs_err_vs_oracle)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the hierarchical 1024^3 workload reported beside the headline")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--tile", default="auto", help="sweep tile (default: autotuned)")
    ap.add_argument("--workload", default="plain", choices=["plain", "hier", "adjoint", "multiclass", "bricks"],
                    help="plain: the 256^3 headline workload; hier: hierarchical 1024^3 vessel tree; "
                         "adjoint: 32 x 96^3 differentiable batch; multiclass: incremental 3-class "
                         "hierarchy on 1024 x 1024 x 2048")
    ap.add_argument("--brick", type=int, default=32)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--max-batch", type=int, default=0, help="bricks per batched solve (0: library default)")
    ap.add_argument("--leaf-host", action="store_true",
                    help="hier: leaf level in mapped host memory (out-of-core placement)")
    ap.add_argument("--all-host", action="store_true",
                    help="hier: every pyramid level and tree field in mapped host memory (out-of-core placement)")
    ap.add_argument("--n", type=int, default=0,
                    help="volume edge (default: 256 plain, 1024 hier, 96 adjoint; smaller for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "hier":
        return run_hier(args)
    if args.workload == "bricks":
        return run_bricks(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "multiclass":
        return run_multiclass(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
