"""Benchmark of the SFC linear-octree neighbour search on one GB300 per rank.

One step = the whole path over one synthetic 10M-point LiDAR-like tile already resident
in HBM: octree_build (bounding box, Hilbert codes, radix sort, gather, linear octree),
an all-points sphere search with r = 2 m (count, scan, fill) and an all-points kNN
search with k = 16.  value = queries answered per second (10M radius + 10M kNN queries
per step).  With --gpus N (launched by torchrun) every rank runs its own replica of the
workload (weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--workload serving replays a seeded Poisson trace of requests (200/s) through the request
server and through a one-request-at-a-time server, reporting queries/s and p50/p99 latency.
--workload batch256 times the batched path instead: 256 clouds of uneven sizes
(log-uniform 10k-2M points, uniform / LiDAR / Gaussian clusters), each with an
all-points sphere or kNN search, answered by one batch_search per step, next to the
plain per-cloud path (octree_build + radius search or kNN, cloud after cloud on one
stream) on the same clouds.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {
    "workload": "lidar_tile_10M",
    "description": "synthetic aerial LiDAR-like tile, 1 km x 1 km, 10 pts/m^2 (60% ground, 30% vegetation, "
                   "10% buildings, 3 cm jitter)",
    "points": 10_000_000,
    "encoding": "hilbert",
    "leaf_capacity": 96,
    "radius": {"kernel": "sphere", "r": 2.0},
    "knn_k": 16,
}
METRIC = "radius/kNN queries/s on 1 GB300 (all-points sphere r=2 m + kNN k=16 over a fresh octree per step)"
UNIT = "queries/s"
L2_FLUSH_BYTES = 512 << 20

# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant kernel,
# with the sha256 of the source file it was measured on (null once the source changes).
NCU_TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum, 10M-point tile, k = 16 (profiles/)
    "knn": {"bytes_per_launch": 191145984 + 1250382592, "sha256": "51c8a6a8cf18055376e50cfd48ca5b7cfe4172f1761a0710b3a6bdbc6c96d7ff"},
    "radius_fill": {"bytes_per_launch": 3155717376 + 4238458880, "sha256": "1c00063f58f40fbe7c3fde014e85c4931210ed8d0da2630aba09371f3e580692"},
    "radius_count": {"bytes_per_launch": 309096448 + 911621120, "sha256": "1c00063f58f40fbe7c3fde014e85c4931210ed8d0da2630aba09371f3e580692"},
}


# warp instructions per group of 32 centres of the dominant kernels (ncu
# smsp__inst_executed.sum on the 2M-point tile, profiles/), keyed like the traffic
NCU_INST_PER_GROUP = {
    "knn": {"warp_inst": 1368283468 / 62500, "sha256": "51c8a6a8cf18055376e50cfd48ca5b7cfe4172f1761a0710b3a6bdbc6c96d7ff"},
    "radius_count": {"warp_inst": 707143347 / 62500, "sha256": "1c00063f58f40fbe7c3fde014e85c4931210ed8d0da2630aba09371f3e580692"},
    "radius_fill": {"warp_inst": 497206502 / 62500, "sha256": "1c00063f58f40fbe7c3fde014e85c4931210ed8d0da2630aba09371f3e580692"},
}
SMS, SMSP_PER_SM = 152, 4  # GB300: one warp instruction per sub-partition per cycle
FP32_LANES_PER_SM = 128      # GB300: 4 sub-partitions x 32 FP32 lanes, one operation each per cycle
# binary32 operations of one centre-point test (subtractions, products, sums or maxima, and
# the comparison): the secondary, ALU side of the roofline
FP32_OPS_PER_TEST = {"sphere": 9, "circle": 6, "cube": 6, "square": 4, "knn": 9}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--points", type=int, default=WORKLOAD["points"], help="override the cloud size (testing)")
    ap.add_argument("--leaf-capacity", type=int, default=WORKLOAD["leaf_capacity"])
    ap.add_argument("--encoding", choices=["none", "morton", "hilbert"], default=WORKLOAD["encoding"])
    ap.add_argument("--radius", type=float, default=WORKLOAD["radius"]["r"])
    ap.add_argument("--kernel", choices=["sphere", "circle", "cube", "square"], default=WORKLOAD["radius"]["kernel"])
    ap.add_argument("--k", type=int, default=WORKLOAD["knn_k"])
    ap.add_argument("--radius-output", choices=["ids", "ranges"], default="ids",
                    help="neighbour ids (CSR) or runs of sorted positions (range output)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-counters", action="store_true",
                    help="skip the untimed work-counter pass after the timed region")
    ap.add_argument("--clocks-csv", default=None, help="directory for the raw nvidia-smi clock samples")
    ap.add_argument("--workload", choices=["lidar_tile_10M", "batch256", "serving", "sweep"], default="lidar_tile_10M")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--no-big", action="store_true", help="serving: leave out the 200M-point cloud")
    ap.add_argument("--clouds", type=int, default=256, help="batch256: number of clouds (testing)")
    ap.add_argument("--no-tune", action="store_true", help="batch256: one leaf capacity for every cloud")
    ap.add_argument("--sweep-oracle-sample", type=int, default=20000,
                    help="sweep: seeded centres per oracle search (scaled to all centres)")
    return ap.parse_args(argv)


# ----------------------------------------------------------------------------- distributed
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world: int, backend: str):
    import torch.distributed as dist

    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def aggregate(step_ms_total: float, units: float, world: int, device=None):
    """Max of the timed region over ranks and the sum of the units processed."""
    import torch
    import torch.distributed as dist

    if world == 1:
        return step_ms_total, units
    t = torch.tensor([step_ms_total], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str | None = None):
        self.gpu = gpu_index
        self.path = path
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [ln for ln in out.splitlines() if ln.strip()]
        if self.path:
            with open(self.path, "w") as f:
                f.write(self.FIELDS + "\n" + "\n".join(self.lines) + "\n")
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- the step
def run_step(sfc, pts, cfg, sphere_events=None):
    """The whole path once; returns (tree, row_ptr, cols, nnz, idx, d2).  With the range
    output, (row_ptr, cols, nnz) are the run pointers, the runs and their number.
    sphere_events: a pair of CUDA events recorded around the radius search (count, scan
    and fill) on the current stream."""
    tree = sfc.octree_build(pts, cfg["encoding"], leaf_capacity=cfg["leaf_capacity"])
    if sphere_events is not None:
        sphere_events[0].record()
    if cfg["radius"].get("output") == "ranges":
        row_ptr, cols = sfc.radius_search_ranges(tree, None, cfg["radius"]["r"], cfg["radius"]["kernel"])
        nnz = int(cols.shape[0])
    else:
        row_ptr, nnz = sfc.radius_count(tree, None, cfg["radius"]["r"], cfg["radius"]["kernel"])
        cols = sfc.radius_fill(tree, None, cfg["radius"]["r"], cfg["radius"]["kernel"], row_ptr, nnz)
    if sphere_events is not None:
        sphere_events[1].record()
    idx, d2 = sfc.knn(tree, None, cfg["knn_k"])
    return tree, row_ptr, cols, nnz, idx, d2


def algorithmic_bytes(kernel: str, n: int, nnz: int, k: int) -> float | None:
    """Bytes one launch of ``kernel`` must move at minimum: its per-unit algorithmic bytes
    (points and ids read, row pointers, neighbour ids or kNN pairs written) times the units."""
    table = {
        "radius_fill": 16 * n + 8 * (n + 1) + 4 * nnz,   # points + ids, row pointers, neighbour ids
        "radius_ranges_fill": 16 * n + 8 * (n + 1) + 8 * nnz,  # points, run pointers, runs (nnz = runs)
        "radius_ranges_count": 12 * n + 4 * n,
        "radius_count": 12 * n + 4 * n,                  # points, counts
        "knn": 16 * n + 8 * n * k,                       # points + ids, k (id, d2) pairs per centre
        "radix_scatter": 24 * n,                         # read + write (code, index)
        "radix_count": 8 * n,                            # one read of the codes for every pass
        "encode": 12 * n + 12 * n,
        "gather_points": 16 * n + 16 * n,
        "bbox": 12 * n,
    }
    return table.get(kernel)


def search_counters(sfc, fn) -> dict:
    """The library's work counters of the searches ``fn`` runs (instrumented kernels, never
    timed)."""
    with sfc.search_stats() as st:
        fn()
    return st


def alu_side(counters: dict, kind: str, launch_ms: float, sm_mhz: float | None) -> dict:
    """Candidate tests per second of one launch and their binary32 operations against the
    FP32 lanes' peak at the sampled SM clock (152 SMs x 128 lanes x clock)."""
    ops = FP32_OPS_PER_TEST[kind]
    per_s = counters["point_tests"] / (launch_ms / 1e3)
    out = {"point_tests": counters["point_tests"], "needed_tests": counters["needed_tests"],
           "tests_per_s": per_s, "needed_tests_per_s": counters["needed_tests"] / (launch_ms / 1e3),
           "fp32_ops_per_test": ops, "counters": counters}
    if sm_mhz:
        peak = SMS * FP32_LANES_PER_SM * sm_mhz * 1e6
        out.update(fp32_ops_per_s=per_s * ops, fp32_peak=peak, fp32_frac=per_s * ops / peak)
    return out


def source_sha(name: str) -> str:
    """sha256 of a kernel source together with the shared device header it includes."""
    h = hashlib.sha256()
    for part in (name, "sfc_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2603_06771_gb300", "csrc", part), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def load_peaks() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- CPU oracle
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "hardware")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# The oracle's step: the same workload on a smaller tile of the same generator (same
# density and structure, side sqrt(n / 10) m), the whole path measured: build, all-points
# sphere search, all-points kNN.  Nothing is scaled or extrapolated.
ORACLE_TILE_POINTS = 200_000


def oracle_step(xyz: np.ndarray, cfg: dict) -> tuple[float, float, float]:
    """One full oracle step over ``xyz``: seconds of the build, the radius and the kNN search."""
    import oracle

    enc = oracle.ENCODINGS[cfg["encoding"]]
    t0 = time.perf_counter()
    pipe = oracle.Pipeline(xyz, enc, cfg["leaf_capacity"])
    t1 = time.perf_counter()
    pipe.tree.radius(xyz, cfg["radius"]["r"], oracle.KERNELS[cfg["radius"]["kernel"]])
    t2 = time.perf_counter()
    pipe.tree.knn(xyz, cfg["knn_k"])
    t3 = time.perf_counter()
    return t1 - t0, t2 - t1, t3 - t2


def oracle_tile(n: int, step: int) -> np.ndarray:
    """The oracle's bounded sample: a LiDAR-like tile of min(n, ORACLE_TILE_POINTS) points
    (seeded per step)."""
    import synth

    return synth.lidar_tile(min(n, ORACLE_TILE_POINTS), synth.CONFIG_SEED[2] + 7919 * (step + 1))


def bench_config(cfg: dict, n: int, world: int) -> dict:
    """The ``config`` object of both arms' lines (identical keys and values)."""
    return dict(cfg, points=n, l2="flushed before every timed step (512 MiB write)",
                parallelism="replicas" if world > 1 else "single GPU")


def reference_arm(args, cfg):
    import oracle

    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    n = args.points
    cores = oracle.num_cpus()
    m = min(n, ORACLE_TILE_POINTS)
    for w in range(args.warmup):
        oracle_step(oracle_tile(n, 1000 + w), cfg)
    parts = []
    for s in range(args.steps):
        parts.append(oracle_step(oracle_tile(n, s), cfg))
    step_s = statistics.mean(sum(p) for p in parts)
    value = 2 * m / step_s
    mb, mr, mk = (statistics.mean(p[i] for p in parts) for i in range(3))
    sample = (f"each step: the whole path of the oracle (plain C; pointer octree; build on 1 thread, "
              f"searches on {cores} threads) on a {m}-point LiDAR-like tile of the same generator and "
              f"density (its own seed per step): build {mb:.3f} s + all-points sphere r={cfg['radius']['r']} "
              f"{mr:.3f} s + all-points kNN k={cfg['knn_k']} {mk:.3f} s; value = {2 * m} queries / measured "
              f"step time; nothing extrapolated")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(cfg, n, world),
        "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": cores, "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- batched workload
BATCH_METRIC = "batched queries/s on 1 GB300 (256 uneven clouds: build + all-points sphere or kNN per cloud)"
BATCH_NNZ_CAP = 1 << 28   # neighbours per radius cloud; above it the radius is redrawn smaller


def batch_setup(sfc, torch, n_clouds: int, ncap: int, enc: str):
    """The clouds, concatenated on the device, and their searches.  A radius cloud whose
    neighbour count exceeds BATCH_NNZ_CAP takes the next smaller radius of the set (counted
    once here with the plain path, before anything is timed)."""
    import synth

    specs = synth.batch_workload(n_clouds)
    xyz = [synth.batch_cloud(sp) for sp in specs]
    pts = torch.from_numpy(np.concatenate(xyz)).cuda()
    views, p0, redrawn = [], 0, 0
    for sp in specs:
        views.append(pts[p0:p0 + sp["n"]])
        p0 += sp["n"]
    for sp, v in zip(specs, views):
        if sp["search"] != "radius":
            continue
        t = sfc.octree_build(v, enc, leaf_capacity=ncap)
        while True:
            _, nnz = sfc.radius_count(t, None, sp["r"], sp["kernel"])
            smaller = [r for r in synth.BATCH_RADII if r < sp["r"]]
            if nnz <= BATCH_NNZ_CAP or not smaller:
                break
            sp["r"] = smaller[-1]
            redrawn += 1
        sp["nnz"] = nnz
        t.free()
    batch_setup.xyz = xyz  # the host clouds, for checks
    return specs, pts, views, redrawn


def plain_step(sfc, specs, views, enc: str, ncap: int):
    """Every cloud through the single-cloud entry points, one after the other (each at the
    leaf capacity the batch gives it)."""
    for sp, v in zip(specs, views):
        t = sfc.octree_build(v, enc, leaf_capacity=sp.get("leaf_capacity") or ncap)
        if sp["search"] == "radius":
            sfc.radius_search(t, None, sp["r"], sp["kernel"])
        else:
            sfc.knn(t, None, sp["k"])
        t.free()


def batch_main(args):
    import torch

    import paper_2603_06771_gb300 as sfc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    sfc.build()
    enc = args.encoding
    ncap = args.leaf_capacity
    specs, pts, views, redrawn = batch_setup(sfc, torch, args.clouds, ncap, enc)
    n_total = int(pts.shape[0])
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    clouds = [dict(n=sp["n"], search=sp["search"], kernel=sp.get("kernel", "sphere"), r=sp.get("r", 0.0),
                   k=sp.get("k", 0)) for sp in specs]
    tune_s = None
    if not args.no_tune:  # per-cloud leaf capacity, kNN seeding window, centres per warp walk and
        # record slots from the device autotuner
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        clouds = sfc.batch_autotune(pts, clouds, enc, leaf_capacity=ncap)
        tune_s = time.perf_counter() - t0
        for sp, c in zip(specs, clouds):
            sp["leaf_capacity"], sp["knn_window"] = c["leaf_capacity"], c["knn_window"]

    def timed(fn, steps, warmup):
        for w in range(warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for s in range(steps):
            flush.fill_(s)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return ms

    def batch_fn():
        sfc.batch_search(pts, clouds, enc, leaf_capacity=ncap).free()

    # the same pass recorded as a CUDA graph (points copied into the plan once, untimed)
    nnz_total = int(sum(sp.get("nnz", 0) for sp in specs))
    plan = sfc.BatchPlan(clouds, enc, leaf_capacity=ncap, nnz_capacity=nnz_total + nnz_total // 8 + 1)
    plan.points.copy_(pts)

    def plan_fn():
        plan.run()

    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local, os.path.join(args.clocks_csv, f"clocks_batch_rank{rank}.csv")
                          if args.clocks_csv else None)
    clocks.start()
    time.sleep(0.3)
    launches0 = sfc.launch_count()
    b_ms = timed(batch_fn, args.steps, args.warmup)
    launches = (sfc.launch_count() - launches0) * args.steps // (args.steps + args.warmup)
    launches1 = sfc.launch_count()
    g_ms = timed(plan_fn, args.steps, args.warmup)
    plan_launches = (sfc.launch_count() - launches1) * args.steps // (args.steps + args.warmup)
    p_ms = timed(lambda: plain_step(sfc, specs, views, enc, ncap), args.steps, args.warmup)
    clk = clocks.stop()
    # per-kernel device time of one more step of each path (events around every launch)
    breakdown = {}
    for name, fn in (("batch", batch_fn), ("plan", plan_fn),
                     ("plain", lambda: plain_step(sfc, specs, views, enc, ncap))):
        torch.cuda.synchronize()
        sfc.profile_read()
        sfc.profile_enable(True)
        torch.cuda.nvtx.range_push(f"{name}_step")  # lets ncu --nvtx-include "batch_step/" pick one step
        fn()
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        sfc.profile_enable(False)
        breakdown[name] = {k: round(ms, 3) for k, (c, ms) in sorted(sfc.profile_read().items(),
                                                                     key=lambda kv: -kv[1][1])}
    b_total, units = aggregate(sum(b_ms), float(n_total * args.steps), world, torch.device("cuda", local))
    g_total, _ = aggregate(sum(g_ms), float(n_total * args.steps), world, torch.device("cuda", local))
    p_total, _ = aggregate(sum(p_ms), float(n_total * args.steps), world, torch.device("cuda", local))
    if rank == 0:
        n_radius = sum(sp["search"] == "radius" for sp in specs)
        line = {
            "metric": BATCH_METRIC, "value": units / (b_total / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": b_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch256", "clouds": len(specs), "points": n_total, "encoding": enc,
                       "leaf_capacity": ncap, "radius_clouds": n_radius, "knn_clouds": len(specs) - n_radius,
                       "radius_redrawn": redrawn, "nnz_cap_per_cloud": BATCH_NNZ_CAP,
                       "autotune_s": tune_s,
                       "leaf_capacity_chosen": sorted({int(c.get("leaf_capacity") or ncap) for c in clouds}),
                       "knn_window_chosen": sorted({int(c.get("knn_window", 0)) for c in clouds
                                                    if c["search"] == "knn"}),
                       "queries_per_warp_chosen": sorted({int(c.get("queries_per_warp") or 32) for c in clouds}),
                       "record_slots_chosen": sorted({int(c.get("record_slots") or 32) for c in clouds
                                                      if c["search"] == "radius"}),
                       "nnz": int(sum(sp.get("nnz", 0) for sp in specs)),
                       "l2": "flushed before every timed step (512 MiB write)"},
            "plain": {"value": units / (p_total / 1e3), "ms_per_step": p_total / args.steps},
            "speedup_vs_plain": p_total / b_total,
            "graph": {"value": units / (g_total / 1e3), "ms_per_step": g_total / args.steps,
                      "speedup_vs_plain": p_total / g_total, "gpu_launches": plan_launches},
            "gpu_launches": launches, "clocks": clk, "kernel_ms": breakdown,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- serving workload
SERVE_METRIC = "served queries/s on 1 GB300 with p50/p99 request latency (Poisson arrivals, LiDAR-like clouds)"


def serve_trace(seconds: float, rate: float, pool_sizes: list, seed: int):
    """Request arrivals (Poisson, seeded) with their cloud (a pool index, drawn by a
    log-uniform size on [50k, 20M]), centres (all points or a seeded 1 % subset) and search
    (half sphere r in {0.5, 1, 2, 3} m, half kNN k in {8, 16, 32})."""
    import synth

    rng = synth.Rng(seed)
    n_max = int(seconds * rate * 2 + 16)
    gaps = -np.log(1.0 - rng.u01(0, n_max)) / rate
    t = np.cumsum(gaps)
    t = t[t < seconds]
    m = len(t)
    size = np.exp(np.log(50_000) + rng.u01(1, m) * (np.log(20_000_000) - np.log(50_000)))
    logs = np.log(np.asarray(pool_sizes, dtype=np.float64))
    pick = np.abs(np.log(size)[:, None] - logs[None, :]).argmin(axis=1)
    subset = rng.u01(2, m) < 0.5
    radius = rng.u01(3, m) < 0.5
    ri = rng.integers(4, m, 4)
    ki = rng.integers(5, m, 3)
    reqs = []
    for i in range(m):
        spec = (dict(search="radius", kernel="sphere", r=synth.BATCH_RADII[int(ri[i])]) if radius[i]
                else dict(search="knn", k=synth.BATCH_KS[int(ki[i])]))
        reqs.append(dict(t=float(t[i]), cloud=int(pick[i]), subset=bool(subset[i]), seed=seed * 7919 + i, **spec))
    return reqs


def serve_run(sfc, torch, trace, pool, big, server_kw, burst: bool = False):
    """Replay the trace against one server: a submitting thread sleeps until each arrival
    (``burst``: submits every request at once, for the capacity), the main thread waits for
    the requests in order and releases them."""
    import threading

    import synth

    srv = sfc.Server(**server_kw)
    ids = [None] * len(trace)
    ready = [threading.Event() for _ in trace]
    subsets = {}
    for i, rq in enumerate(trace):  # the centres of subset requests, drawn before the clock starts
        if rq["subset"]:
            xyz = big if rq["cloud"] < 0 else pool[rq["cloud"]]
            n = xyz.shape[0]
            rows = np.sort(synth.Rng(rq["seed"]).integers(0, max(1, n // 100), n))
            subsets[i] = torch.from_numpy(np.ascontiguousarray(xyz.numpy()[rows])).pin_memory()
    t0 = time.perf_counter()

    def submitter():
        for i, rq in enumerate(trace):
            delay = 0.0 if burst else rq["t"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            xyz = big if rq["cloud"] < 0 else pool[rq["cloud"]]
            kw = {k: rq[k] for k in ("search", "kernel", "r", "k") if k in rq}
            ids[i] = srv.submit(xyz, queries=subsets.get(i), **kw)
            ready[i].set()

    th = threading.Thread(target=submitter)
    th.start()
    lat, queued, merged, queries = [], [], [], 0
    for i in range(len(trace)):
        ready[i].wait()
        st = srv.wait(ids[i])
        if st != 0:
            raise RuntimeError(f"request {i} failed with status {st}")
        tm = srv.timings(ids[i])
        lat.append(tm["latency_ms"])
        queued.append(tm["queue_ms"])
        merged.append(tm["batched_with"])
        queries += tm["rows"]
        srv.release(ids[i])
    makespan = time.perf_counter() - t0
    th.join()
    srv.close()
    lat = np.asarray(lat)
    return {"queries_per_s": queries / makespan, "requests": len(trace), "queries": queries,
            "makespan_s": makespan, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "mean_queue_ms": float(np.mean(queued)),
            "merged_requests": int(sum(1 for b in merged if b > 1))}


def serve_main(args):
    import torch

    import paper_2603_06771_gb300 as sfc
    import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    sfc.build()
    pool_sizes = [int(round(x)) for x in np.exp(np.linspace(np.log(50_000), np.log(20_000_000), 16))]
    pool = [torch.from_numpy(synth.lidar_tile(n, synth.CONFIG_SEED[5] * 100 + j)).pin_memory()
            for j, n in enumerate(pool_sizes)]
    big = None
    trace = serve_trace(args.serve_seconds, args.serve_rate, pool_sizes, synth.CONFIG_SEED[5] + rank)
    if not args.no_big:  # one 200M-point cloud at 20 pts/m^2 (10 km^2), 1 % of its points as centres
        big = torch.from_numpy(synth.lidar_tile(200_000_000, synth.CONFIG_SEED[5] * 100 + 99,
                                                side=float(np.sqrt(200_000_000 / 20.0)))).pin_memory()
        mid = next(i for i, rq in enumerate(trace) if rq["t"] >= args.serve_seconds / 2)
        trace.insert(mid, dict(t=trace[mid]["t"], cloud=-1, subset=True, seed=12345, search="radius",
                               kernel="sphere", r=2.0))
    kw = dict(slots=args.serve_slots, max_batch=64, batch_points=4_000_000, hbm_budget=150 << 30,
              encoding=args.encoding, leaf_capacity=args.leaf_capacity)
    warm = serve_trace(1.0, 20.0, pool_sizes, 7)  # loads the library paths and the memory pool
    serve_run(sfc, torch, warm, pool, big, kw)
    clocks = ClockSampler(local, os.path.join(args.clocks_csv, f"clocks_serve_rank{rank}.csv")
                          if args.clocks_csv else None)
    clocks.start()
    launches0 = sfc.launch_count()
    ours = serve_run(sfc, torch, trace, pool, big, kw)
    launches = sfc.launch_count() - launches0
    plain_kw = dict(kw, slots=1, max_batch=1, batch_points=0)
    plain = serve_run(sfc, torch, trace, pool, big, plain_kw)
    # capacity: the same requests all at once, so each server runs flat out
    cap_ours = serve_run(sfc, torch, trace, pool, big, kw, burst=True)
    cap_plain = serve_run(sfc, torch, trace, pool, big, plain_kw, burst=True)
    clk = clocks.stop()
    capacity = {"served": {k: cap_ours[k] for k in ("queries_per_s", "makespan_s", "merged_requests")},
                "plain": {k: cap_plain[k] for k in ("queries_per_s", "makespan_s")},
                "speedup_vs_plain": cap_ours["queries_per_s"] / cap_plain["queries_per_s"],
                "how": "every request of the trace submitted at once; queries / time to the last result"}
    if rank == 0:
        line = {
            "metric": SERVE_METRIC, "value": ours["queries_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": ours["makespan_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving", "rate_per_s": args.serve_rate, "seconds": args.serve_seconds,
                       "cloud_sizes": "log-uniform 50k-20M (16 LiDAR-like pool clouds, pinned host memory)",
                       "big_cloud": None if args.no_big else "200M points, 20 pts/m^2, 1% centres, sphere r=2",
                       "centres": "50% all points, 50% seeded 1% subset",
                       "searches": "50% sphere r in {0.5,1,2,3} m, 50% kNN k in {8,16,32}",
                       "hbm_budget_gib": 150, "slots": args.serve_slots, "encoding": args.encoding,
                       "leaf_capacity": args.leaf_capacity,
                       "latency": "submit to result resident on the device"},
            "p50_ms": ours["p50_ms"], "p99_ms": ours["p99_ms"], "serving": ours,
            "plain": plain, "speedup_vs_plain": ours["queries_per_s"] / plain["queries_per_s"],
            "capacity": capacity, "gpu_launches": launches, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- sweep
def sweep_main(args):
    """Every search of the LiDAR-tile workloads on the resident 10M tile, one JSON line each:
    4 kernels x r in {0.5, 1, 2, 3} m x 3 orders (count + fill), kNN k in {8, 16, 50} x 3
    orders, and the build; device time by CUDA events (best of 3, L2 flushed before each),
    queries/s, neighbours/s, the fraction of the HBM roofline (algorithmic bytes of the call
    / time / measured copy bandwidth) and the candidate tests per second with their share of
    the FP32 lanes.  Then the oracle's searches of every combination on a seeded sample of
    centres on the host cores, scaled to all centres (unless --no-cpu-baseline)."""
    import torch

    import paper_2603_06771_gb300 as sfc
    import synth

    torch.cuda.set_device(0)
    sfc.build()
    n = args.points
    xyz = synth.config_cloud(2) if n == WORKLOAD["points"] else synth.lidar_tile(n, synth.CONFIG_SEED[2])
    pts = torch.from_numpy(xyz).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    peak, peak_kind = load_peaks()
    clocks = ClockSampler(0, os.path.join(args.clocks_csv, "clocks_sweep.csv") if args.clocks_csv else None)
    clocks.start()

    def best_ms(fn, reps=3):
        out = None
        for rep in range(reps + 1):
            flush.fill_(rep)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            res = fn()
            b.record(stream)
            b.synchronize()
            if rep:  # the first is a warm-up
                out = min(out, a.elapsed_time(b)) if out is not None else a.elapsed_time(b)
            del res
        return out

    lines = []
    for enc in ("none", "morton", "hilbert"):
        build_ms = best_ms(lambda: sfc.octree_build(pts, enc, leaf_capacity=args.leaf_capacity).free())
        t = sfc.octree_build(pts, enc, leaf_capacity=args.leaf_capacity)
        lines.append({"sweep": "build", "encoding": enc, "points": n, "ms": build_ms})
        print(json.dumps(lines[-1]), flush=True)
        for kern in ("sphere", "cube", "circle", "square"):
            for r in (0.5, 1.0, 2.0, 3.0):
                ms = best_ms(lambda: sfc.radius_search(t, None, r, kern))
                nnz = int(sfc.radius_count(t, None, r, kern)[1])
                cnt = search_counters(sfc, lambda: sfc.radius_count(t, None, r, kern))
                alg = 16 * n + 8 * (n + 1) + 4 * nnz  # points + ids, row pointers, neighbour ids
                lines.append({"sweep": "radius", "encoding": enc, "kernel": kern, "r": r, "ms": ms,
                              "queries_per_s": n / (ms / 1e3), "neighbours_per_s": nnz / (ms / 1e3),
                              "mu": nnz / n, "hbm_frac": alg / (ms / 1e3) / 1e9 / peak,
                              "tests_per_s": cnt["point_tests"] / (ms / 1e3), "counters": cnt,
                              "fp32_ops_per_test": FP32_OPS_PER_TEST[kern]})
                print(json.dumps(lines[-1]), flush=True)
        for k in (8, 16, 50):
            ms = best_ms(lambda: sfc.knn(t, None, k))
            cnt = search_counters(sfc, lambda: sfc.knn(t, None, k))
            alg = 16 * n + 8 * n * k  # points + ids, k (id, d2) pairs per centre
            lines.append({"sweep": "knn", "encoding": enc, "k": k, "ms": ms, "queries_per_s": n / (ms / 1e3),
                          "hbm_frac": alg / (ms / 1e3) / 1e9 / peak,
                          "tests_per_s": cnt["point_tests"] / (ms / 1e3), "counters": cnt,
                          "fp32_ops_per_test": FP32_OPS_PER_TEST["knn"]})
            print(json.dumps(lines[-1]), flush=True)
        t.free()
    clk = clocks.stop()
    sm_mhz = clk.get("sm_mhz") if clk else None
    fp32_peak = SMS * FP32_LANES_PER_SM * sm_mhz * 1e6 if sm_mhz else None
    print(json.dumps({"sweep": "peaks", "hbm_gbs": peak, "hbm_peak_source": peak_kind, "clocks": clk,
                      "fp32_peak_ops_per_s": fp32_peak,
                      "fp32_frac_of": "tests_per_s x fp32_ops_per_test / fp32_peak_ops_per_s"}), flush=True)

    if args.no_cpu_baseline:
        return 0
    # the oracle: one pointer octree (its searches do not depend on the curve), every
    # combination on the same seeded centres, all host threads, scaled to n centres
    import oracle

    t0 = time.perf_counter()
    tree = oracle.PointerOctree(xyz, args.leaf_capacity)
    build_s = time.perf_counter() - t0
    sample = min(n, args.sweep_oracle_sample)
    q = xyz[np.sort(np.random.default_rng(11).choice(n, sample, replace=False))]
    cores = oracle.num_cpus()
    for kern in ("sphere", "cube", "circle", "square"):
        for r in (0.5, 1.0, 2.0, 3.0):
            t0 = time.perf_counter()
            tree.radius(q, r, oracle.KERNELS[kern])
            sec = time.perf_counter() - t0
            print(json.dumps({"sweep": "oracle_radius", "kernel": kern, "r": r, "centres": sample, "s": sec,
                              "queries_per_s": sample / sec, "cores": cores, "extrapolated": sample < n}),
                  flush=True)
    for k in (8, 16, 50):
        t0 = time.perf_counter()
        tree.knn(q, k)
        sec = time.perf_counter() - t0
        print(json.dumps({"sweep": "oracle_knn", "k": k, "centres": sample, "s": sec, "queries_per_s": sample / sec,
                          "cores": cores, "extrapolated": sample < n}), flush=True)
    print(json.dumps({"sweep": "oracle_build", "points": n, "s": build_s, "threads": 1, "cpu_model": cpu_model()}),
          flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def main(argv=None):
    args = parse_args(argv)
    if args.workload == "sweep" and args.impl == "ours":
        return sweep_main(args)
    if args.workload == "batch256" and args.impl == "ours":
        return batch_main(args)
    if args.workload == "serving" and args.impl == "ours":
        return serve_main(args)
    cfg = dict(WORKLOAD, leaf_capacity=args.leaf_capacity, encoding=args.encoding, knn_k=args.k,
               radius={"kernel": args.kernel, "r": args.radius})
    if args.radius_output == "ranges":
        cfg["radius"]["output"] = "ranges"
    if args.impl == "reference":
        return reference_arm(args, cfg)

    import torch

    import paper_2603_06771_gb300 as sfc
    import synth

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    sfc.build()
    n = args.points
    seed = synth.CONFIG_SEED[2] + rank
    xyz = synth.config_cloud(2) if (n == WORKLOAD["points"] and rank == 0) else synth.lidar_tile(n, seed)
    pts = torch.from_numpy(xyz).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    k = cfg["knn_k"]

    # warm-up (also sizes the outputs)
    nnz = 0
    for _ in range(args.warmup):
        tree, row_ptr, cols, nnz, idx, d2 = run_step(sfc, pts, cfg)
        tree.free()
        del row_ptr, cols, idx, d2
    torch.cuda.synchronize()

    # timed region: K steps, L2 flushed before each, CUDA events around each step
    clocks = ClockSampler(local, os.path.join(args.clocks_csv, f"clocks_rank{rank}.csv")
                          if args.clocks_csv else None)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sphere_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = sfc.launch_count()
    sfc.profile_enable(True)
    wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.fill_(s)
        starts[s].record(stream)
        tree, row_ptr, cols, nnz, idx, d2 = run_step(sfc, pts, cfg, sphere_ev[s])
        ends[s].record(stream)
        tree.free()
        del row_ptr, cols, idx, d2
    torch.cuda.synchronize()
    wall_s = time.perf_counter() - wall0
    sfc.profile_enable(False)
    launches = sfc.launch_count() - launches0
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    prof = sfc.profile_read()
    total_ms, units = aggregate(sum(step_ms), 2.0 * n * args.steps, world, torch.device("cuda", local))
    ms_per_step = total_ms / args.steps
    value = units / (total_ms / 1e3)

    # roofline of the dominant kernel (largest share of the timed region)
    peak, peak_kind = load_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dom_name, (dom_launches, dom_ms) = dom
    dom_avg_ms = dom_ms / dom_launches
    alg = algorithmic_bytes(dom_name, n, nnz, k)
    roof = None
    if alg is not None:
        achieved = alg / (dom_avg_ms / 1e3) / 1e9
        src = {"radius_fill": "sfc_radius.cu", "radius_count": "sfc_radius.cu", "knn": "sfc_knn.cu"}.get(
            dom_name, "sfc_runtime.cu")
        rec = NCU_TRAFFIC.get(dom_name)
        traffic = rec["bytes_per_launch"] if rec and rec.get("sha256") == source_sha(src) else None
        roof = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s", "traffic": traffic,
                "algorithmic_bytes_per_launch": alg, "avg_launch_ms": dom_avg_ms}
        # what bounds these kernels: instruction issue (warp instructions per launch from the
        # ncu capture, scaled by the launch's groups) against one per sub-partition per cycle
        ins = NCU_INST_PER_GROUP.get(dom_name)
        if ins and ins.get("sha256") == source_sha(src) and clk and clk.get("sm_mhz"):
            issued = ins["warp_inst"] * ((n + 31) // 32) / (dom_avg_ms / 1e3)
            issue_peak = SMS * SMSP_PER_SM * clk["sm_mhz"] * 1e6
            roof["issue"] = {"achieved": issued, "peak": issue_peak, "unit": "warp instructions/s",
                             "frac": issued / issue_peak,
                             "source": "ncu smsp__inst_executed.sum per group of 32 centres (2M-point tile), "
                                       "peak = 152 SMs x 4 sub-partitions x median SM clock"}
    kernels = {name: {"launches": c, "total_ms": ms, "share": ms / sum(step_ms)} for name, (c, ms) in
               sorted(prof.items(), key=lambda kv: -kv[1][1])}

    # the fixed-radius search as one unit (count, scan of the counts, host read of the total,
    # fill), timed by CUDA events around the two calls in every timed step
    sphere_ms = statistics.mean(a.elapsed_time(b) for a, b in sphere_ev)
    roof_sphere = None
    out_kind = "radius_ranges_fill" if cfg["radius"].get("output") == "ranges" else "radius_fill"
    sph_alg = algorithmic_bytes(out_kind, n, nnz, k)
    if sph_alg is not None:
        sph_ach = sph_alg / (sphere_ms / 1e3) / 1e9
        tr = [NCU_TRAFFIC.get(x) for x in ("radius_count", "radius_fill")]
        sph_traffic = (sum(t["bytes_per_launch"] for t in tr)
                       if all(t and t.get("sha256") == source_sha("sfc_radius.cu") for t in tr) else None)
        roof_sphere = {"bound": "hbm", "search": f"{cfg['radius']['kernel']} r={cfg['radius']['r']} all points",
                       "achieved": sph_ach, "peak": peak, "unit": "GB/s", "frac": sph_ach / peak,
                       "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                       else "fallback 6.8 TB/s", "traffic": sph_traffic, "algorithmic_bytes": sph_alg,
                       "ms": sphere_ms,
                       "kernels_ms": {x: prof[x][1] / prof[x][0] for x in ("radius_count", "radius_fill",
                                                                            "radius_ranges_count",
                                                                            "radius_ranges_fill") if x in prof},
                       "note": "count + scan + fill as one unit: algorithmic bytes 16 N (points and ids) + "
                               "8 (N + 1) (row pointers) + 4 nnz (neighbour ids) over the CUDA-event time "
                               "between the start of the count and the end of the fill"}

    # candidate tests of the two search kernels (instrumented copies, run once, untimed)
    tests = {}
    sm_mhz = clk.get("sm_mhz") if clk else None
    if not args.no_counters:
        t = sfc.octree_build(pts, cfg["encoding"], leaf_capacity=cfg["leaf_capacity"])
        if cfg["radius"].get("output") != "ranges" and "radius_count" in prof:
            c = search_counters(sfc, lambda: sfc.radius_count(t, None, cfg["radius"]["r"], cfg["radius"]["kernel"]))
            tests["radius_count"] = alu_side(c, cfg["radius"]["kernel"], prof["radius_count"][1] /
                                             prof["radius_count"][0], sm_mhz)
        if "knn" in prof:
            c = search_counters(sfc, lambda: sfc.knn(t, None, k))
            tests["knn"] = alu_side(c, "knn", prof["knn"][1] / prof["knn"][0], sm_mhz)
        t.free()
    if roof is not None and dom_name in tests and "fp32_frac" in tests[dom_name]:
        a = tests[dom_name]
        roof["alu"] = {"achieved": a["fp32_ops_per_s"], "peak": a["fp32_peak"], "unit": "FP32 op/s",
                       "frac": a["fp32_frac"], "tests_per_s": a["tests_per_s"],
                       "source": "library work counters (point tests executed per launch) x binary32 operations "
                                 "per test; peak = 152 SMs x 128 FP32 lanes x median SM clock"}

    # end to end through the public API: pinned host points in, every result back to pinned host
    # memory.  Steps are pipelined: a copy stream takes each step's results to the host (the
    # radius output while the kNN runs, the kNN output while the next step builds and
    # searches), into two alternating sets of pinned buffers; the timed region runs from an
    # idle device to the last result of the last step on the host side of the link.
    e2e = None
    if not args.no_e2e:
        h_xyz = torch.from_numpy(xyz).pin_memory()
        per = 2 if cfg["radius"].get("output") == "ranges" else 1  # int32 words per output entry
        h_sets = [{"rp": torch.empty(n + 1, dtype=torch.int64, pin_memory=True),
                   "cols": torch.empty(per * (int(nnz * 1.05) + 1024), dtype=torch.int32, pin_memory=True),
                   "idx": torch.empty((n, k), dtype=torch.int32, pin_memory=True),
                   "d2": torch.empty((n, k), dtype=torch.float32, pin_memory=True)} for _ in range(2)]
        d_pts = torch.empty_like(pts)
        copier = torch.cuda.Stream()

        copied = {}  # step -> event after its last copy

        def e2e_step(s):
            h = h_sets[s % 2]
            if s - 2 in copied:  # at most two steps in flight: the buffers of step s - 2 are free again
                copied.pop(s - 2).synchronize()
            flush.fill_(s)
            d_pts.copy_(h_xyz, non_blocking=True)
            tree = sfc.octree_build(d_pts, cfg["encoding"], leaf_capacity=cfg["leaf_capacity"])
            if per == 2:
                row_ptr, cols = sfc.radius_search_ranges(tree, None, cfg["radius"]["r"], cfg["radius"]["kernel"])
                e_nnz = int(cols.shape[0])
            else:
                row_ptr, e_nnz = sfc.radius_count(tree, None, cfg["radius"]["r"], cfg["radius"]["kernel"])
                cols = sfc.radius_fill(tree, None, cfg["radius"]["r"], cfg["radius"]["kernel"], row_ptr, e_nnz)
            csr_done = torch.cuda.Event()
            csr_done.record(stream)
            with torch.cuda.stream(copier):
                copier.wait_event(csr_done)
                h["rp"].copy_(row_ptr, non_blocking=True)
                h["cols"][:per * e_nnz].copy_(cols.reshape(-1), non_blocking=True)
            idx, d2 = sfc.knn(tree, None, k)
            knn_done = torch.cuda.Event()
            knn_done.record(stream)
            with torch.cuda.stream(copier):
                copier.wait_event(knn_done)
                h["idx"].copy_(idx, non_blocking=True)
                h["d2"].copy_(d2, non_blocking=True)
                copied[s] = torch.cuda.Event()
                copied[s].record(copier)
            for t in (row_ptr, cols, idx, d2):  # freed only after the copy stream has read them
                t.record_stream(copier)
            tree.free()

        for s in range(args.warmup):
            e2e_step(s)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for s in range(args.warmup, args.warmup + args.steps):
            e2e_step(s)
        stream.wait_stream(copier)
        b.record(stream)
        b.synchronize()
        e_total, e_units = aggregate(a.elapsed_time(b), 2.0 * n * args.steps, world, torch.device("cuda", local))
        e2e = {"value": e_units / (e_total / 1e3), "unit": UNIT, "h2d_bytes_per_step": 12 * n,
               "d2h_bytes_per_step": 8 * (n + 1) + 4 * per * nnz + 8 * n * k, "ms_per_step": e_total / args.steps,
               "pipelined": "each step's results cross the link while the next step computes"}

    cpu = None
    if rank == 0 and world >= 1 and not args.no_cpu_baseline and args.gpus == 1:
        import oracle

        m = min(n, ORACLE_TILE_POINTS)
        parts = [oracle_step(oracle_tile(n, s), cfg) for s in range(3)]
        step_s = statistics.mean(sum(p) for p in parts)
        mb, mr, mk = (statistics.mean(p[i] for p in parts) for i in range(3))
        # binary32 decisions that binary64 would take the other way (a brute-force scan over
        # the benchmark's own cloud, so for 2000 seeded centres)
        rows_b = np.sort(np.random.default_rng(7).choice(n, min(n, 2000), replace=False))
        boundary = oracle.boundary_disagreements(xyz, xyz[rows_b], cfg["radius"]["r"],
                                                 oracle.KERNELS[cfg["radius"]["kernel"]])
        cpu = {"value": 2 * m / step_s, "unit": UNIT, "cores": oracle.num_cpus(), "kind": "oracle",
               "cpu_model": cpu_model(),
               "boundary_disagreements": {"centres": len(rows_b), "pairs_decided_differently_in_binary64": boundary},
               "sample": (f"3 steps of the oracle's whole path (plain C; build on 1 thread, searches on "
                          f"{oracle.num_cpus()} threads) on {m}-point LiDAR-like tiles of the same generator "
                          f"and density: build {mb:.3f} s + all-points sphere r={cfg['radius']['r']} {mr:.3f} s "
                          f"+ all-points kNN k={cfg['knn_k']} {mk:.3f} s per step; value = {2 * m} queries / "
                          f"measured step time")}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(cfg, n, world),
            "nnz": nnz, "mu": nnz / n, "neighbours_per_s": nnz * args.steps * world / (total_ms / 1e3),
            "gpu_launches": launches, "wall_s": wall_s, "roofline": roof, "roofline_sphere": roof_sphere,
            "kernels": kernels,
            "candidate_tests": tests, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
