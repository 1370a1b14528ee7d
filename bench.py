#!/usr/bin/env python3
"""Throughput benchmark of hierarchical homogenization on GB300.

Workload: the 512^3 overlapping-sphere sandstone (porosity 0.15, solid K=37
G=44 GPa, pore 1e-4 GPa) cut into 27,000 uneven cores of edge 16/24/32 with
seeded buffers 0..8 (buffered subimages 16..48), coarse unit 8. The cores form
a 30 x 30 x 30 grid; a tile is one z-slab of it by `--tile-rows` rows in y
(default 6: 180 cores, 150 tiles in the image). One step is the full
hierarchical homogenization of one tile: extraction of its buffered
subimages (buffers wrap in the whole image), 6 load cases each solved to
tolerance, C_R = Sigma Eps^-1, assembly of the tile's coarse image, its
level-2 solve and the moduli.

Metric: voxel-iterations per second (one unit = one voxel of one load case
through one conjugate-gradient iteration), whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}]
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

METRIC = "voxel·iters/s; 512³ hierarchical homogenization s vs plain FP64 at ≤0.5% K,G err"
UNIT = "voxel·iters/s"
IMAGE_SEED = 2208023203


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--fused", type=int, default=-1,
                    help="1: level-1 solves by the fused cluster kernel, 0: the multi-pass solver, -1: the "
                         "library's default")
    ap.add_argument("--shape-kernels", type=int, default=1,
                    help="1: plane and column passes compiled for the workload's common shapes (the library "
                         "default), 0: the generic passes for every shape")
    ap.add_argument("--fixed-iters", type=int, default=0,
                    help="> 0: every load case runs exactly this many iterations (short launches for profiling "
                         "runs; the default solves to tol)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--tile-rows", type=int, default=6)
    ap.add_argument("--cost-scaling", type=int, default=0,
                    help="1: also time single-subimage solves and whole hierarchical runs against the subimage "
                         "edge n on a 120^3 crop (Section 3, Fig. 3) and fit power laws in n")
    ap.add_argument("--fp64-compare", type=int, default=0,
                    help="also solve the first N rows of the last timed tile in FP64 (plain CG, no residual "
                         "replacement) and report time and K, G differences")
    ap.add_argument("--cufft", type=int, default=1,
                    help="1: also time cuFFT (through torch.fft) on the forward and inverse 3D real transforms of "
                         "the six components of every problem of the last timed tile (a comparator only)")
    ap.add_argument("--headline-rows", type=int, default=6,
                    help="y-rows of the last timed tile on which the plain FP64 solver (one subimage at a time) "
                         "and the batched FP32 solver are timed against each other (0: skip)")
    ap.add_argument("--surrogate", type=int, default=1,
                    help="1: train a 4-member CNN ensemble on the subimages of the warm-up tiles, labelled by the "
                         "FFT solver's C_R from those warm-up steps, and time the two-level homogenization of the "
                         "headline cores with the surrogate standing in for the subimages its gate accepts "
                         "(needs --headline-rows > 0)")
    ap.add_argument("--surrogate-epochs", type=int, default=60)
    ap.add_argument("--study", default="", choices=["", "richardson"],
                    help="richardson: instead of the benchmark, the subimage-size study on the 256^3 three-phase "
                         "image (direct solve, hierarchical at n = 16..128 and buffers 0, 4, 8, fits in 1/n, "
                         "the planner's choice); one JSON line")
    ap.add_argument("--surrogate-spread", type=float, default=0.02)
    ap.add_argument("--study-buffers", default="0,4,8",
                    help="richardson study: buffer widths b (comma-separated)")
    ap.add_argument("--study-ns", default="16,32,64,128",
                    help="richardson study: core edges n (comma-separated)")
    return ap.parse_args()


def workload(tile_rows: int = 6):
    """Image, phases, partition and the list of tiles (z-slab x tile_rows y-rows)."""
    import numpy as np
    import synth
    img = synth.boolean_spheres(n=512, seed=IMAGE_SEED)
    boxes = synth.uneven_partition(N=512, seed=IMAGE_SEED)
    zs = sorted(set(int(v) for v in boxes[:, 2]))
    ys = sorted(set(int(v) for v in boxes[:, 1]))
    tiles = []
    for z in zs:
        slab = boxes[boxes[:, 2] == z]
        for j in range(0, len(ys), tile_rows):
            tiles.append(slab[np.isin(slab[:, 1], ys[j:j + tile_rows])])
    return img, synth.PHASES_SOLID_PORE, boxes, tiles


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_hash() -> str:
    """SHA-256 (16 hex digits) of the field kernels' sources and compile
    flags, comments and layout removed (a comment edit changes no kernel)."""
    import hashlib
    import re
    h = hashlib.sha256()
    # the sources of the multi-pass field kernels and the compile flags
    for f in ("csrc/hh_device.cuh", "csrc/hh_plane_ct.cuh", "csrc/hh_ct_inst.cu", "csrc/hh_fftcore.cuh",
              "csrc/hh_fft2.cuh", "csrc/hh_fft2_inst.cu", "csrc/hh_ctmath.h", "_build.py"):
        with open(os.path.join(ROOT, "paper_2208_02320_gb300", f)) as fh:
            text = fh.read()
        if f.endswith(".py"):
            text = re.sub(r"#[^\n]*", "", text)
        else:
            text = re.sub(r"/\*.*?\*/", "", re.sub(r"//[^\n]*", "", text), flags=re.S)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per algorithmic byte of each field pass (plane_fwd,
    plane_inv, column) from the committed ncu summary
    (profiles/roofline_traffic.txt); {} if absent or if the kernel sources
    have changed since the capture."""
    p = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    try:
        kv = dict(l.strip().split("=", 1) for l in open(p) if "=" in l and not l.startswith("#"))
        if kv.get("kernel_source_sha256_16") != kernel_source_hash():
            return {}
        return {k[len("ratio."):]: float(v) for k, v in kv.items() if k.startswith("ratio.")}
    except (OSError, ValueError):
        return {}


def cpu_baseline(img, ph, boxes, seconds: float):
    """The FP64 oracle, as it stands, on a bounded sample: conjugate-gradient
    iterations of one buffered subimage of the workload (one load case)."""
    from oracle import hh_oracle as O
    sizes = (boxes[:, 3:6] + 2 * boxes[:, 6:7]).prod(axis=1)
    k = int(sizes.argsort()[len(sizes) // 2])  # a median-size subimage
    b = boxes[k]
    sub = O.extract_box(img, b)
    med = O.IsoMedium.from_labels(sub, ph)
    V = sub.size
    t0 = time.perf_counter()
    O.solve_cg(med, O.unit_load(0), fixed_iters=2)
    per = (time.perf_counter() - t0) / 3.0  # rhs + 2 iterations
    iters = max(2, int(seconds / max(per, 1e-6)))
    t0 = time.perf_counter()
    O.solve_cg(med, O.unit_load(0), fixed_iters=iters)
    dt = time.perf_counter() - t0
    nproc = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    try:
        from threadpoolctl import threadpool_info
        threads = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        threads = nproc
    return {"value": V * iters / dt, "unit": UNIT, "cores": int(min(threads, nproc)), "nproc": int(nproc),
            "kind": "oracle",
            "sample": f"oracle CG, subimage {k} of the partition (Omega_B {tuple(int(v) for v in sub.shape)}, "
                      f"{V} voxels), load case 0 (unit E_11), {iters} iterations in {dt:.1f} s; numpy's "
                      f"BLAS pool of {threads} threads on {nproc} host cores"}


def tile_index(i: int, ws: int, rank: int, ntiles: int) -> int:
    """Tile of step i on this rank: the ranks take consecutive tiles, so every
    step of the job works on ws distinct tiles (weak scaling, no exchange)."""
    return (i * ws + rank) % ntiles


def dist_init():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def reduce_max_sum(vals_max, vals_sum, ws):
    if ws == 1:
        return vals_max, vals_sum
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    a = torch.tensor(vals_max, dtype=torch.float64, device=dev)
    b = torch.tensor(vals_sum, dtype=torch.float64, device=dev)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return a.tolist(), b.tolist()


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def workload_config(args, slabs) -> dict:
    """The workload keys of the JSON line, the same for both arms."""
    return {
        "workload": "spheres512: 512^3 overlapping-sphere sandstone, 27000 uneven cores 16/24/32 + buffers "
                    "0..8 (subimages 16..48), unit 8; one step = full hierarchical homogenization of one "
                    f"tile (one z-slab x {args.tile_rows} y-rows of cores: each x 6 load cases to tol, "
                    "assembly, level-2 solve)",
        "tol": args.tol, "phases": "solid K=37 G=44, pore K=G=1e-4 GPa (contrast 4.4e5)",
        "tiles_in_image": len(slabs), "l2": "working set per step >> 129 MB L2 (inputs larger than L2)",
    }


def run_reference(args):
    ws, rank, local = dist_init()
    if rank != 0:
        return
    img, ph, boxes, slabs = workload(args.tile_rows)
    per = max(2.0, args.cpu_seconds / max(args.steps + args.warmup, 1))
    for _ in range(args.warmup):
        cpu_baseline(img, ph, slabs[0], min(per, 2.0))
    vals = []
    last = None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        last = cpu_baseline(img, ph, slabs[0], per)
        vals.append(last["value"])
    wall = time.perf_counter() - t0
    v = statistics.median(vals)
    last["value"] = v
    config = workload_config(args, slabs)
    config.update(precision="fp64 (the CPU oracle)",
                  step="one bounded sample of the workload: oracle CG iterations of one median-size subimage "
                       "of the first tile (the oracle as it stands)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config, "cpu_baseline": last,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_gb300(args):
    import numpy as np
    import torch

    ws, rank, local = dist_init()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    from paper_2208_02320_gb300 import Context, _build
    _build.build()
    img, ph, boxes, slabs = workload(args.tile_rows)
    dimg = torch.from_numpy(img).to(f"cuda:{local}")
    ctx = Context(local)
    opt = dict(precision=args.precision, tol=args.tol, profile=1, shape_kernels=args.shape_kernels)
    if args.fixed_iters > 0:
        opt["fixed_iters"] = args.fixed_iters
    if args.fused >= 0:
        opt["fused"] = args.fused

    def step(i, device=True):
        sl = slabs[tile_index(i, ws, rank, len(slabs))]
        src = dimg if device else img
        return ctx.homogenize_partition(src, ph, sl, unit=8, **opt)

    warm = []  # (cores, FFT C_R) of the warm-up steps: the surrogate's training set
    for i in range(args.warmup):
        r = step(i)
        warm.append((slabs[tile_index(i, ws, rank, len(slabs))], r["C_boxes"]))
    ctx.profile_reset()
    barrier(ws)
    torch.cuda.synchronize()
    units = 0
    dev_ms = 0.0
    launches = 0
    stats = []
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for i in range(args.warmup, args.warmup + args.steps):
            r = step(i)
            units += r["voxel_iters"]
            dev_ms += r["device_ms"]
            launches += r["kernel_launches"]
            stats.append(r)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    barrier(ws)
    prof = ctx.profile()
    # end to end through the public API with host buffers (image H2D every step)
    e2e_units, e2e_s = 0, 0.0
    for i in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = step(args.warmup + args.steps + i, device=False)
        e2e_s += time.perf_counter() - t0
        e2e_units += r["voxel_iters"]
    (dev_s_max, wall_max, e2e_max), (units_sum, e2e_units_sum) = reduce_max_sum(
        [dev_ms / 1e3, wall, e2e_s], [units, e2e_units], ws)
    if rank != 0:
        return
    peaks, peak_src = measured_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1]["sampled_ms"]) if prof else None
    roof = None
    if dom:
        name, st = dom
        achieved = st["sampled_bytes"] / (st["sampled_ms"] / 1e3) / 1e9
        ratio = ncu_traffic().get(name)
        roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": (ratio * st["sampled_bytes"] / st["sampled"]) if ratio else None,
                "algorithmic_bytes_per_launch": st["sampled_bytes"] / max(st["sampled"], 1),
                "avg_launch_ms": st["sampled_ms"] / max(st["sampled"], 1), "peak_source": peak_src,
                "kernels": {k: {"sampled": v["sampled"], "avg_ms": v["sampled_ms"] / max(v["sampled"], 1),
                                "GBps": v["sampled_bytes"] / max(v["sampled_ms"], 1e-9) / 1e6} for k, v in prof.items()}}
    nbox = sum(len(slabs[tile_index(i, ws, rank, len(slabs))]) for i in range(args.warmup, args.warmup + args.steps))
    value = units_sum / dev_s_max
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dev_s_max * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": dict(
            workload_config(args, slabs),
            precision=args.precision + " fields and FFTs, fp64 scalars and averages",
            cores_per_step=nbox // max(args.steps, 1), parallelism=f"{ws} independent ranks (tiles)",
            wall_s=wall_max, iters_max=max(s["iters_max"] for s in stats),
            resid_max=max(s["resid_max"] for s in stats),
            status=[s["status"] for s in stats], K_G_last=[stats[-1]["K"], stats[-1]["G"]],
        ),
        "clocks": clk.summary(),
        "e2e": {"value": e2e_units_sum / e2e_max if e2e_max > 0 else None, "unit": UNIT,
                "h2d_bytes_per_step": int(img.nbytes + 28 * nbox // max(args.steps, 1)),
                "d2h_bytes_per_step": int((36 * 8 + 6 * 4) * nbox // max(args.steps, 1) + 1024)},
        "gpu_launches": launches,
        "roofline": roof,
    }
    line["cpu_baseline"] = cpu_baseline(img, ph, slabs[0], args.cpu_seconds) if ws == 1 else None
    if args.fp64_compare > 0 and ws == 1:
        sl = slabs[(args.warmup + args.steps - 1) % len(slabs)]
        ys = np.unique(sl[:, 1])[:args.fp64_compare]
        sub = sl[np.isin(sl[:, 1], ys)]
        r32 = ctx.homogenize_partition(dimg, ph, sub, unit=8, precision="fp32", tol=args.tol)
        r64 = ctx.homogenize_partition(dimg, ph, sub, unit=8, precision="fp64", tol=args.tol)
        line["fp64_compare"] = {
            "cores": int(len(sub)), "fp32_ms": r32["device_ms"], "fp64_ms": r64["device_ms"],
            "speedup_fp32": r64["device_ms"] / max(r32["device_ms"], 1e-9),
            "K_rel_diff": abs(r32["K"] - r64["K"]) / r64["K"], "G_rel_diff": abs(r32["G"] - r64["G"]) / r64["G"],
            "iters_max": [r32["iters_max"], r64["iters_max"]]}
    if args.cost_scaling and ws == 1:
        line["cost_scaling"] = cost_scaling(ctx, img, ph, args.tol)
    if args.cufft and ws == 1:
        sl = slabs[tile_index(args.warmup + args.steps - 1, ws, rank, len(slabs))]
        line["cufft_comparator"] = cufft_comparator(sl, value)
    if args.headline_rows > 0 and ws == 1:
        sl = slabs[tile_index(args.warmup + args.steps - 1, ws, rank, len(slabs))]
        ys = np.unique(sl[:, 1])[:args.headline_rows]
        hl, runs = headline(ctx, dimg, ph, sl[np.isin(sl[:, 1], ys)], args.tol, len(slabs), args.fused)
        line["headline"] = hl
        if args.surrogate:
            line["surrogate"] = surrogate_arm(ctx, dimg, ph, warm, sl[np.isin(sl[:, 1], ys)], args, runs, len(slabs))
    print(json.dumps(line))


def cufft_comparator(cores, value):
    """cuFFT (library transforms through torch.fft, timed only; nothing of the
    product uses it) on the transforms of one operator application for every
    (subimage, load case) problem of a tile: the six stress components of each
    problem's buffered box, forward real-to-complex and inverse
    complex-to-real, batched per box shape. Reported as voxel-iterations per
    second of these transforms alone, beside the product's whole-iteration
    rate (constitutive law, transforms, projection, CG update and reductions)."""
    import numpy as np
    import torch
    shapes = {}
    for b in cores:
        sh = (int(b[5] + 2 * b[6]), int(b[4] + 2 * b[6]), int(b[3] + 2 * b[6]))
        shapes[sh] = shapes.get(sh, 0) + 1
    fields = {sh: torch.randn((6 * n * 6,) + sh, device="cuda", dtype=torch.float32) for sh, n in shapes.items()}
    units = sum(6 * n * int(np.prod(sh)) for sh, n in shapes.items())

    def sweep():
        for sh, f in fields.items():
            spec = torch.fft.rfftn(f, dim=(-3, -2, -1))
            torch.fft.irfftn(spec, s=sh, dim=(-3, -2, -1))

    for _ in range(3):
        sweep()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        sweep()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del fields
    torch.cuda.empty_cache()
    return {"what": "cuFFT R2C + C2R of 6 components x 6 load cases per subimage of the tile, batched per shape "
                    f"({len(shapes)} shapes), FP32, torch.fft", "ms_per_operator_application": ms,
            "transform_voxel_iters_per_s": units / (ms / 1e3), "product_whole_iteration_voxel_iters_per_s": value,
            "product_over_cufft_transforms_only": value / (units / (ms / 1e3))}


def voigt_kg(C):
    """Voigt-average K and G of the symmetric part of 6x6 stiffnesses in Voigt notation."""
    import numpy as np
    S = 0.5 * (C + np.swapaxes(C, -1, -2))
    d = S[..., 0, 0] + S[..., 1, 1] + S[..., 2, 2]
    o = S[..., 0, 1] + S[..., 0, 2] + S[..., 1, 2]
    sh = S[..., 3, 3] + S[..., 4, 4] + S[..., 5, 5]
    return (d + 2 * o) / 9.0, (d - o + 3 * sh) / 15.0


def headline(ctx, dimg, ph, cores, tol, ntiles, fused=-1):
    """The same cores homogenized (level 1, assembly, level 2) by the plain
    FP64 solver -- FP64 fields, one subimage per wave of launches, no
    surrogate -- and by the batched FP32 solver, with wall times (host clock
    around each synchronous call) and the FP32 result's error against FP64:
    relative K and G of the two-level result, and of every subimage's C_R
    (isotropic Voigt projection of its symmetric part)."""
    import numpy as np
    import torch

    def run(**o):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = ctx.homogenize_partition(dimg, ph, cores, unit=8, tol=tol, **o)
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    r64, t64 = run(precision="fp64", wave_boxes=1, fused=0)
    r32, t32 = run(precision="fp32", **({"fused": fused} if fused >= 0 else {}))

    K32, G32 = voigt_kg(r32["C_boxes"])
    K64, G64 = voigt_kg(r64["C_boxes"])
    eb = np.maximum(np.abs(K32 - K64) / K64, np.abs(G32 - G64) / G64)
    return ({
        "cores": int(len(cores)), "tol": tol,
        "plain_fp64": {"wall_s": t64, "device_ms": r64["device_ms"], "launches": r64["kernel_launches"],
                       "iters_max": r64["iters_max"], "status": r64["status"], "K": r64["K"], "G": r64["G"]},
        "fp32_batched": {"wall_s": t32, "device_ms": r32["device_ms"], "launches": r32["kernel_launches"],
                         "iters_max": r32["iters_max"], "status": r32["status"], "K": r32["K"], "G": r32["G"]},
        "speedup_vs_plain_fp64": t64 / t32,
        "K_rel_err": abs(r32["K"] - r64["K"]) / r64["K"], "G_rel_err": abs(r32["G"] - r64["G"]) / r64["G"],
        "subimage_KG_rel_err": {"max": float(eb.max()), "median": float(np.median(eb)),
                                "p99": float(np.quantile(eb, 0.99))},
        "whole_image_estimate_s": {"plain_fp64": t64 * ntiles * 180 / len(cores),
                                   "fp32_batched": t32 * ntiles * 180 / len(cores),
                                   "note": "per-tile wall time x tiles in the 512^3 image (one tile measured)"},
    }, {"r64": r64, "t64": t64, "r32": r32, "t32": t32})


def surrogate_arm(ctx, dimg, ph, warm, cores, args, runs, ntiles):
    """The surrogate standing in for subimage solves on the headline cores.

    Training set: every buffered subimage of the warm-up tiles, labelled by
    the upper triangle of the symmetric part of its C_R from the FFT solver
    in those warm-up steps (no oracle, no extra solves). Four members from
    the library's He-uniform initializer, Adam with the cosine step size.
    Then the headline cores are homogenized with the surrogate (the gate's
    accepted subimages take the ensemble mean, the rest the FFT solver) and
    compared with the plain FP64 and the batched FP32 runs of the same
    cores: wall time, the two-level K and G, and every accepted subimage's
    K/G error against the FFT solver's C_R."""
    import numpy as np
    import torch
    from paper_2208_02320_gb300 import binding
    scale = 100.0
    iu = np.triu_indices(6)
    boxes = np.concatenate([w[0] for w in warm])
    C = np.concatenate([w[1] for w in warm])
    labs = ctx.extract_subimages(dimg, boxes)
    tcores = [(int(b[6]), int(b[6]), int(b[6]), int(b[3]), int(b[4]), int(b[5])) for b in boxes]
    y = np.stack([(0.5 * (c + c.T))[iu] for c in C]) / scale
    members, hist = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for m in range(4):
        th, h = ctx.surrogate_train(labs, y.astype(np.float32), binding.cnn_init_params(4100 + m),
                                    epochs=args.surrogate_epochs, batch=8, lr=2e-3, seed=m, cores=tcores)
        members.append(th)
        hist.append([float(h[0]), float(h[-1])])
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    members = np.stack(members)
    opt = dict(precision="fp32", tol=args.tol, **({"fused": args.fused} if args.fused >= 0 else {}))
    ctx.homogenize_partition_surrogate(dimg, ph, cores, members, unit=8, scale=scale, spread=args.surrogate_spread,
                                       **opt)  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rs = ctx.homogenize_partition_surrogate(dimg, ph, cores, members, unit=8, scale=scale,
                                            spread=args.surrogate_spread, **opt)
    torch.cuda.synchronize()
    t_sur = time.perf_counter() - t0
    r64, t64, r32, t32 = runs["r64"], runs["t64"], runs["r32"], runs["t32"]
    acc = rs["accepted"]
    Ks, Gs = voigt_kg(rs["C_boxes"])
    Kf, Gf = voigt_kg(r32["C_boxes"])
    eb = np.maximum(np.abs(Ks - Kf) / Kf, np.abs(Gs - Gf) / Gf)[acc]
    return {
        "training": {"subimages": int(len(boxes)), "shapes": int(len({l.shape for l in labs})), "members": 4,
                     "epochs": args.surrogate_epochs, "batch": 8, "wall_s": t_train,
                     "loss_first_last": hist,
                     "note": "subimages of the warm-up tiles, labelled by their FFT C_R from the warm-up steps"},
        "cores": int(len(cores)), "accepted": int(acc.sum()), "spread": args.surrogate_spread,
        "wall_s": t_sur, "speedup_vs_plain_fp64": t64 / t_sur, "speedup_vs_fp32_batched": t32 / t_sur,
        "K": rs["K"], "G": rs["G"],
        "K_rel_err_vs_plain_fp64": abs(rs["K"] - r64["K"]) / r64["K"],
        "G_rel_err_vs_plain_fp64": abs(rs["G"] - r64["G"]) / r64["G"],
        "accepted_subimage_KG_rel_err_vs_fft": ({"max": float(eb.max()), "median": float(np.median(eb))}
                                                if eb.size else None),
        "whole_image_estimate_s": {"surrogate": t_sur * ntiles * 180 / len(cores) + t_train,
                                   "note": "per-tile wall time x tiles, plus the training once"},
    }


def cost_scaling(ctx, img, ph, tol):
    """Cost of one subimage solve t(n) and of the whole two-level run
    T(n) = (N/n)^3 t(n) + level 2 on a fixed N^3 crop, against the subimage
    edge n (no buffer), with least-squares exponents of t ~ n^a and T ~ n^b
    (the paper's Fig. 3 reports a = 3.66 and b = a - 3 = 0.66 on its CPUs)."""
    import numpy as np
    N = 120
    crop = np.ascontiguousarray(img[:N, :N, :N])
    ns = [15, 20, 24, 30, 40, 60]
    t1, tH, it1 = [], [], []
    for n in ns:
        box = np.array([[0, 0, 0, n, n, n, 0]], dtype=np.int32)
        ctx.solve_subimages(crop, ph, box, precision="fp32", tol=tol)  # warm (autotuner, tables)
        r = ctx.homogenize_partition(crop, ph, box, unit=n, precision="fp32", tol=tol)
        t1.append(r["device_ms"])
        it1.append(r["iters_max"])
        ctx.homogenize_hierarchical(crop, ph, n, 0, precision="fp32", tol=tol)
        tH.append(ctx.homogenize_hierarchical(crop, ph, n, 0, precision="fp32", tol=tol)["device_ms"])
    a = float(np.polyfit(np.log(ns), np.log(t1), 1)[0])
    b = float(np.polyfit(np.log(ns), np.log(tH), 1)[0])
    return {"image": f"{N}^3 crop of the workload image, fp32, tol {tol}", "n": ns, "t_single_ms": t1,
            "iters_single": it1, "t_hierarchical_ms": tH, "exponent_single": a, "exponent_hierarchical": b}


def richardson_study(args):
    """The paper's Section 5 study on a synthetic stand-in: the 256^3
    three-phase Gaussian-random-field image (pore 18 %, clay 12 %, solid;
    correlation length 6), its direct FP32 solve, the two-level scheme at
    n = 16, 32, 64, 128 with buffers 0, 4 and 8, the least-squares fits
    M(n) = M_inf + C / n per buffer, the arithmetic means (AM), a free
    power-law exponent of the HH error, and the planner's choice of (n, b)
    for a 0.5 % target from the fitted constants."""
    import numpy as np
    import torch
    import synth
    from paper_2208_02320_gb300 import Context, _build, plan_partition
    _build.build()
    img = synth.grf_three_phase(n=256, ell=6.0, seed=2208023202)
    ph = synth.PHASES_SOLID_CLAY_PORE
    dimg = torch.from_numpy(img).cuda()
    ctx = Context(0)
    opt = dict(precision=args.precision, tol=args.tol)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d = ctx.homogenize_direct(dimg, ph, **opt)
    t_direct = time.perf_counter() - t0
    print(json.dumps({"direct": dict(K=d["K"], G=d["G"], iters_max=d["iters_max"], status=d["status"],
                                     wall_s=t_direct)}), flush=True)
    ns = [int(v) for v in args.study_ns.split(",")]
    bs = [int(v) for v in args.study_buffers.split(",")]
    rows, fits, crel = [], {}, []
    for b in bs:
        t0 = time.perf_counter()
        e = ctx.extrapolate(dimg, ph, ns, b=b, **opt)
        t = time.perf_counter() - t0
        for n, r in zip(ns, e["per_n"]):
            rows.append(dict(n=n, b=b, K=r["K"], G=r["G"], K_am=r["K_am"], G_am=r["G_am"],
                             K_err=(r["K"] - d["K"]) / d["K"], G_err=(r["G"] - d["G"]) / d["G"],
                             K_am_err=(r["K_am"] - d["K"]) / d["K"], G_am_err=(r["G_am"] - d["G"]) / d["G"],
                             status=r["status"], iters_max=r["iters_max"]))
            print(json.dumps({"row": rows[-1]}), flush=True)
        errs = np.array([[abs(x["K_err"]), abs(x["G_err"])] for x in rows if x["b"] == b])
        slope = [float(np.polyfit(np.log(ns), np.log(np.maximum(errs[:, j], 1e-12)), 1)[0]) for j in range(2)]
        fits[b] = dict(K_inf=e["K_inf"], C_K=e["C_K"], G_inf=e["G_inf"], C_G=e["C_G"],
                       K_inf_vs_direct=(e["K_inf"] - d["K"]) / d["K"], G_inf_vs_direct=(e["G_inf"] - d["G"]) / d["G"],
                       free_exponent_K=slope[0], free_exponent_G=slope[1], wall_s=t)
        print(json.dumps({"fit": {"b": b, **fits[b]}}), flush=True)
        crel.append(max(abs(e["C_K"]) / e["K_inf"], abs(e["C_G"]) / e["G_inf"]))
    plan = plan_partition(img.shape, 1, bs, crel, a=3.66, eps=0.005)
    print(json.dumps({"study": "richardson", "image": "grf_three_phase 256^3 (ell 6, pore 18 %, clay 12 %)",
                      "precision": args.precision, "tol": args.tol,
                      "direct": dict(K=d["K"], G=d["G"], iters_max=d["iters_max"], status=d["status"],
                                     wall_s=t_direct),
                      "rows": rows, "fits": {str(k): v for k, v in fits.items()},
                      "plan_0.5pct": plan}))


def main():
    args = parse()
    if args.study == "richardson":
        richardson_study(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
