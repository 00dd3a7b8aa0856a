"""Benchmark: B-char cell-steps/s of whole time steps on one GB300.

One step is one time step of the whole hot path through the C ABI: setting the
step's velocity (with its checks) and bchar_step -- RK4 tracking of the balls,
ball intersections and row assembly, column balancing, the N = 10 alternating
scalings, the bounded mass-conservation minimisation solved to the library's
default tolerance, the final weights and the update c <- W c.  The default
workload is the 1024 x 1024 stretched-mesh single vortex (FP32 tracking and
intersections, FP64 sums and minimisation), the largest configuration whose
steps finish in seconds; --workload picks another recipe.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own replica of the workload on its
own GPU (the method does not shard: replicas only) and rank 0 prints one JSON
line with the whole-job rate.  --impl reference times the FP64 CPU oracle on
all host cores (one process per core, each on a bounded sample of the same
recipe).
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "B-char cell-steps/s on 1 GB300 (plain vs batched/served); p50/p99 solve latency"
UNIT = "cell-steps/s"
WORKLOAD = "vortex2d_1024"
ORACLE_SAMPLE_N = 128  # cells per axis of each oracle process's sample (same recipe)
# DRAM bytes per launch of kernels, measured by ncu on a named workload, each
# with the hash of the kernel's source when it was measured (a line whose hash
# no longer matches is ignored: the kernel changed since)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "vortex2d_1024_dram_traffic.txt")
CSRC = os.path.join(ROOT, "paper_1908_05834_gb300", "csrc")
# the file holding each kernel, and the definitions its source hash covers
# besides the kernel itself (its line-sum epilogue; the tile loop it runs)
KERNEL_FILES = {"k_spmv": ("sparse.cu", ["struct SpmvEpi"]), "k_scale_tiles": ("sparse.cu", ["struct ScaleEpi"]),
                "k_cg_matvec": ("sparse.cu", ["struct MatvecEpi"])}


def max_over_ranks(x: float, device) -> float:
    """The largest x over the ranks of the process group (x itself without one):
    the whole job is as slow as its slowest replica."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Cell-steps per second of the whole job: every rank steps its own replica."""
    return cells_per_rank * steps * world / seconds


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _definition(text: str, name: str) -> str:
    """The source of the definition of `name` (a kernel, or a struct given as
    "struct Name"): from the name through the brace that closes its body
    (declarations without a body are skipped)."""
    start = 0
    while True:
        i = text.index(name, start)
        start = i + len(name)
        j = i + len(name)
        if name.startswith("struct "):
            k = j
        else:
            if text[j] != "(":
                continue
            depth, k = 0, j
            while True:  # the closing parenthesis of the parameter list
                depth += {"(": 1, ")": -1}.get(text[k], 0)
                k += 1
                if depth == 0:
                    break
        while text[k].isspace():
            k += 1
        if text[k] != "{":
            continue  # a declaration
        depth = 0
        for e in range(k, len(text)):
            depth += {"{": 1, "}": -1}.get(text[e], 0)
            if depth == 0:
                return text[i:e + 1]
        raise ValueError(name)


def kernel_source_hash(kernel: str) -> str:
    """Hash of a kernel's definition, the definitions it depends on and the
    tile loop header: what its DRAM traffic depends on."""
    fname, deps = KERNEL_FILES[kernel]
    with open(os.path.join(CSRC, fname)) as f:
        text = f.read()
    with open(os.path.join(CSRC, "tiles.cuh")) as f:
        tiles = f.read()
    h = hashlib.sha256()
    for name in [kernel] + deps:
        h.update(_definition(text, name).encode())
    h.update(tiles.encode())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, workload: str):
    """(DRAM bytes per launch, the line) for kernel on workload from the traffic
    file, or (None, None) when absent or taken on other sources."""
    if not os.path.exists(TRAFFIC_FILE) or kernel not in KERNEL_FILES:
        return None, None
    want = kernel_source_hash(kernel)
    with open(TRAFFIC_FILE) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel and parts[1] == workload:
                if parts[3] == want:
                    return int(float(parts[2])), line.strip()
    return None, None


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(stage: str, nc: int, nnz: int, c_bytes: int = 8) -> int:
    """Bytes one launch of a stage must move at least: per entry and per node
    (cell, or constraint node of the minimisation: 2 n_c of them), each
    array read or written once; gathered vectors count once (they stay in L2)."""
    if stage == "update":
        # c^{n+1} = W c^n and the mass sums: per entry column 4 B + weight 8 B;
        # per cell row pointer 8 B, c_in and c_out, |K|_phi 8 B
        return nnz * (4 + 8) + nc * (8 + 2 * c_bytes + 8)
    if stage == "scaling":
        # one column and one row pass of eq. volAdj, each over its own view of
        # the entries (index 4 B + value 8 B); per line pointer 8 B, target 8 B,
        # the other side's factor 8 B, own factor written 8 B
        return 2 * (nnz * (4 + 8) + nc * (8 + 8 + 8 + 8))
    if stage == "cg_matvec":
        # the minimisation's product with A-hat D A-hat^T + diag: once through
        # the row view and once through the column view (index 4 B + a^2 D 8 B
        # per entry); per node (2 n_c) pointer 8 B, diagonal 8 B, p 8 B, q 8 B
        return 2 * nnz * (4 + 8) + 2 * nc * (8 + 8 + 8 + 8)
    if stage == "smooth":
        # one damped-Jacobi sweep of the multigrid's finest level: 2 n_c nodes,
        # 2 nnz off-diagonal entries (value 8 B + column 4 B); per node pointer
        # 8 B, x, b, diagonal and weight read and x_out written (8 B each)
        return 2 * nnz * (8 + 4) + 2 * nc * (8 + 5 * 8)
    raise KeyError(stage)


def _face_tensors(wl, st, device=None, pinned=False):
    import torch
    out = []
    for a in wl.faces(st % wl.steps):
        t = torch.from_numpy(np.ascontiguousarray(a).reshape(-1))
        out.append(t.to(device) if device is not None else (t.pin_memory() if pinned else t))
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1908_05834_gb300 import build as cuda_build
    if rank == 0 or not os.path.exists(cuda_build.LIB):
        cuda_build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    from paper_1908_05834_gb300 import bchar, inputs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = inputs.workload(args.workload, n=args.n)
    nc = wl.nc
    nsteps = args.warmup + args.steps
    faces_dev = [_face_tensors(wl, st, dev) for st in range(nsteps)]
    extra = {} if args.qp_tol is None else {"qp_tol": args.qp_tol}
    if args.qp_max_refine is not None:
        extra["qp_max_refine"] = args.qp_max_refine
    opts = bchar.default_options(precision=bchar.FP32_SPLIT if wl.precision == "fp32split" else bchar.FP64, **extra)
    mesh = bchar.Mesh(wl.coords, wl.phi, opts)
    cdt = torch.float32 if wl.c_dtype == "f32" else torch.float64
    c = torch.tensor(wl.c0, dtype=cdt, device=dev)
    out = torch.empty_like(c)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def one(st):
        nonlocal c, out
        mesh.set_velocity(faces_dev[st])
        info = mesh.step(wl.dt, c, out)
        c, out = out, c
        return info

    for st in range(args.warmup):
        one(st)
    torch.cuda.synchronize()
    c_at_timed = c.cpu()  # the end-to-end run repeats the timed steps from here
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    sampler = ClockSampler(local_rank)
    if not args.profile:
        sampler.start()
    times, infos = [], []
    for k in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos.append(one(args.warmup + k))
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total = max_over_ranks(sum(times), dev)
    value = whole_job_rate(nc, args.steps, world, total)
    last = infos[-1]
    nnz = last["nnz"]
    cb = 4 if wl.c_dtype == "f32" else 8

    # kernel timings: CUDA events around graph replays of each stage's kernels on
    # the handle's stream, on the last step's data
    torch.cuda.nvtx.range_push("stage_timing")
    ms = {"update": mesh.time_stage(bchar.STAGE_UPDATE, 50), "scaling": mesh.time_stage(bchar.STAGE_SCALING, 20),
          "cg_matvec": mesh.time_stage(bchar.STAGE_CG_MATVEC, 50),
          "assemble": mesh.time_stage(bchar.STAGE_ASSEMBLE, 3), "track": mesh.time_stage(bchar.STAGE_TRACK, 3)}
    if last["amg_levels"] > 0:
        ms["smooth"] = mesh.time_stage(bchar.STAGE_SMOOTH, 50)
        ms["vcycle"] = mesh.time_stage(bchar.STAGE_VCYCLE, 20)
    torch.cuda.nvtx.range_pop()
    cg_mean = statistics.mean(i["cg_iters"] for i in infos)
    # launches per step of each streaming kernel: the update once, the scalings
    # N = 10 times (a column and a row pass each), the matvec once per CG
    # iteration, and the finest level's post-smoothing sweep once per V-cycle
    # (one V-cycle per CG iteration)
    per_step = {"update": 1, "scaling": opts.n_scale, "cg_matvec": cg_mean, "smooth": cg_mean}
    hbm, peak_kind = _peaks()
    step_ms = 1e3 * total / args.steps
    kernels = {}
    names = {"update": "k_spmv", "scaling": "k_scale_tiles", "cg_matvec": "k_cg_matvec",
             "smooth": "k_jacobi<double> (finest multigrid level)"}
    for stage in ("update", "scaling", "cg_matvec", "smooth"):
        if stage not in ms:
            continue
        byt = algorithmic_bytes(stage, nc, nnz, cb)
        gbs = byt / (ms[stage] * 1e-3) / 1e9
        kernels[stage] = {"kernel": names[stage], "algorithmic_bytes_per_launch": byt,
                          "mean_launch_ms": round(ms[stage], 5), "achieved": round(gbs, 1),
                          "frac": round(gbs / hbm, 4), "launches_per_step": round(per_step[stage], 1),
                          "share_of_step": round(ms[stage] * per_step[stage] / step_ms, 4)}
    # the roofline kernel: the largest share of the step among the kernels of the
    # method's own stages (the update, the scalings, the minimisation's product);
    # the multigrid smoother, the preconditioner's kernel, is listed beside them
    dom = max(("update", "scaling", "cg_matvec"), key=lambda k: kernels[k]["share_of_step"])
    K = kernels[dom]
    traffic, traffic_line = measured_traffic(K["kernel"], args.workload)
    roofline = {"bound": "hbm", "kernel": K["kernel"], "stage": dom, "achieved": K["achieved"], "peak": hbm,
                "unit": "GB/s", "frac": K["frac"], "traffic": traffic,
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch: " + traffic_line)
                if traffic else "no ncu capture of the current kernel source",
                "peak_source": f"{peak_kind} hbm_gbs (burst copy)",
                "algorithmic_bytes_per_launch": K["algorithmic_bytes_per_launch"],
                "mean_launch_ms": K["mean_launch_ms"], "share_of_step": K["share_of_step"],
                "all_streaming_kernels": kernels}

    e2e = None if args.profile else run_e2e(args, mesh, wl, bchar, torch, dev, c_at_timed)

    batched = served = None
    if world == 1 and not args.no_serve and not args.profile:
        batched = run_batched(args, torch, bchar, inputs)
        served = run_served(args, torch, bchar, inputs)

    step_stage_ms = {k: round(statistics.mean(i["ms_stage"][k] for i in infos), 3) for k in infos[0]["ms_stage"]}
    result = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded analytic fields and meshes)",
        "config": {"workload": f"{args.workload}: {inputs.describe(args.workload, args.n)}",
                   "cells": nc, "parallelism": f"replicas x{world}",
                   "l2": "flushed (256 MB write) between steps; inputs also exceed L2",
                   "qp_tol": opts.qp_tol, "qp_max_refine": opts.qp_max_refine, "qp_note": "the bounded minimisation is solved to the library default "
                   "(scaled constraint residual <= qp_tol, mean complementarity <= 1e-12), the tolerance the "
                   "parity tests use; qp_converged counts the timed steps that met it"},
        "gpu_launches": int(sum(i["kernel_launches"] for i in infos)),
        "roofline": roofline,
        "stage_ms": {k: round(v, 4) for k, v in ms.items()},
        "step_stage_ms": step_stage_ms,
        "step_stats": {"ip_iters": [i["ip_iters"] for i in infos], "cg_iters": [i["cg_iters"] for i in infos],
                       "qp_converged": sum(i["qp_converged"] for i in infos),
                       "kkt_rel_max": max(i["kkt_rel"] for i in infos),
                       "max_rel_row_res_max": max(i["max_rel_row_res"] for i in infos),
                       "max_rel_col_res_max": max(i["max_rel_col_res"] for i in infos),
                       "n_at_bounds": [i["n_at_bounds"] for i in infos],
                       "amg_levels": last["amg_levels"], "amg_coarsest": last["amg_coarsest"], "nnz": nnz,
                       "row_cap": last["row_cap"], "spill_rows": last["spill_rows"], "substeps": last["substeps"],
                       "max_rel_mass_change": max(abs(i["mass_after"] - i["mass_before"]) / i["mass_before"]
                                                  for i in infos)},
        "clocks": clocks,
        "e2e": e2e,
    }
    if batched is not None:
        result["batched"] = batched
    if served is not None:
        result["served"] = served
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline and not args.profile:
            result["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(result), flush=True)
    mesh.close()


def run_e2e(args, mesh, wl, bchar, torch, dev, c_start):
    """The same steps as the device-timed run, through the C ABI with HOST
    buffers: every step passes the step's face velocities from pinned host
    memory (the library copies them), copies c to the device and reads the new
    c back; the clock (host, around the whole loop) includes all of it."""
    k0, k = args.warmup, args.steps
    faces_host = [_face_tensors(wl, k0 + st, pinned=True) for st in range(k)]
    c_host = c_start.clone().pin_memory()
    back = torch.empty_like(c_host).pin_memory()
    c_dev = torch.empty(wl.nc, dtype=c_host.dtype, device=dev)
    out = torch.empty_like(c_dev)
    h2d = sum(f.numel() * f.element_size() for f in faces_host[0]) + c_host.numel() * c_host.element_size()
    d2h = back.numel() * back.element_size()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for st in range(k):
        mesh.set_velocity([f.numpy() for f in faces_host[st]])
        c_dev.copy_(c_host, non_blocking=True)
        mesh.step(wl.dt, c_dev, out)
        back.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        c_host.copy_(back)
    t = time.perf_counter() - t0
    return {"value": round(wl.nc * k / t, 1), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": k, "step_indices": [k0, k0 + k - 1]}


def _serving_sample(inputs, count, max_cells, steps):
    """The first `count` requests of the serving stream with at most max_cells
    cells, each cut to `steps` steps (a bounded sample of the stream)."""
    picked = []
    for r in inputs.serving_requests(512):
        if r.nc <= max_cells:
            picked.append(dataclasses.replace(r, steps=min(r.steps, steps)))
        if len(picked) == count:
            break
    return picked


def _serving_options(bchar):
    return bchar.default_options(precision=bchar.FP32_SPLIT)


def run_batched(args, torch, bchar, inputs):
    """Plain vs batched stepping of a sample of the serving stream (uneven
    sizes): plain = one bchar_step after another; batched = bchar_step_batch
    of all instances per step.  Host wall clock around whole steps (every
    instance's step has finished when the call returns)."""
    reqs = _serving_sample(inputs, args.batch_count, args.serve_max_cells, args.batch_steps + 1)
    prepared = [r.materialize() for r in reqs]
    opts = _serving_options(bchar)

    def make():
        hs = []
        for (coords, phi, faces, c0) in prepared:
            st = torch.cuda.Stream()
            m = bchar.Mesh(coords, phi, opts, stream=st.cuda_stream)
            fd = [torch.from_numpy(np.ascontiguousarray(f).reshape(-1)).cuda() for f in faces]
            c = torch.tensor(c0, dtype=torch.float64, device="cuda")
            hs.append([m, fd, c, torch.empty_like(c)])
        torch.cuda.synchronize()
        return hs

    def plain_step(hs, k):
        for r, h in zip(reqs, hs):
            h[0].set_velocity(h[1], scale=r.time_factor(k))
            h[0].step(r.dt, h[2], h[3])
            h[2], h[3] = h[3], h[2]

    def batch_step(hs, k):
        for r, h in zip(reqs, hs):
            h[0].set_velocity(h[1], scale=r.time_factor(k))
        bchar.step_batch([h[0] for h in hs], [r.dt for r in reqs], [h[2] for h in hs], [h[3] for h in hs])
        for h in hs:
            h[2], h[3] = h[3], h[2]

    out, finals = {}, {}
    for mode, fn in (("plain", plain_step), ("batched", batch_step)):
        hs = make()
        fn(hs, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(1, 1 + args.batch_steps):
            fn(hs, k)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        out[mode] = round(sum(r.nc for r in reqs) * args.batch_steps / t, 1)
        finals[mode] = [h[2].cpu() for h in hs]
        for h in hs:
            h[0].close()
    same = all(torch.equal(a, b) for a, b in zip(finals["plain"], finals["batched"]))
    return {"plain": out["plain"], "batched": out["batched"], "unit": UNIT,
            "speedup": round(out["batched"] / out["plain"], 3), "bitwise_equal": same,
            "instances": len(reqs), "steps": args.batch_steps, "cells": [r.nc for r in reqs],
            "sample": f"the first {len(reqs)} requests of the serving stream (seed 4004) with at most "
                      f"{args.serve_max_cells} cells, {args.batch_steps} timed steps after 1 warm-up step, "
                      f"FP32 split, library-default minimisation tolerance"}


def run_served(args, torch, bchar, inputs):
    """A sample of the serving stream (Poisson arrivals, mean gap 2 ms, 60 % 2D /
    40 % 3D) through the serving loop: 120 GB admission budget, --serve-slots
    concurrent requests.  The payloads (mesh, phi, base field, c0) are built
    before the clock starts; latency = finish - arrival, including queueing and
    the uploads."""
    from paper_1908_05834_gb300 import serve
    reqs = _serving_sample(inputs, args.serve_requests, args.serve_max_cells, args.serve_steps)
    t0 = time.perf_counter()
    prepared = {r.rid: r.materialize() for r in reqs}
    prep_s = time.perf_counter() - t0
    opts = _serving_options(bchar)
    srv = serve.Server(serve.GpuExecutor(prepared, opts, torch.cuda.current_device()),
                       serve.estimator_for(prepared, opts), budget_bytes=120e9, max_active=args.serve_slots)
    res = srv.run(reqs)
    s = serve.summarize(res)
    s.update({"unit": UNIT, "budget_gb": 120, "slots": args.serve_slots,
              "peak_admitted_gb": round(srv.peak_used / 1e9, 2), "peak_active": srv.peak_active,
              "max_peak_bytes_over_estimate": round(max((r.peak_bytes / r.est_bytes) for r in res
                                                        if r.status == "ok"), 3),
              "footprint_overruns": len(srv.overruns),
              "prep_s": round(prep_s, 1),
              "sample": f"the first {len(reqs)} requests of the 512-request serving stream (seed 4004) with at "
                        f"most {args.serve_max_cells} cells, each cut to {args.serve_steps} steps, FP32 split, "
                        f"library-default minimisation tolerance"})
    return s


# ---------------------------------------------------------------- the oracle on the host cores

_W = {}


_ONE_THREAD = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _oracle_worker_init(n):
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1908_05834_gb300 import inputs
    wl = inputs.workload(WORKLOAD, n=n)
    _W["wl"] = wl
    _W["mesh"] = oracle.Mesh(wl.coords, wl.phi)
    _W["c"] = wl.c0.astype(np.float64)


def _oracle_worker_step(k):
    import oracle
    wl = _W["wl"]
    t = time.perf_counter()
    r = oracle.step(_W["mesh"], wl.faces(k % wl.steps), wl.dt, _W["c"])
    _W["c"] = r["c"]
    return time.perf_counter() - t


class OraclePool:
    """One oracle process per host core (spawned), each stepping its own copy
    of the bounded sample: the recipe at ORACLE_SAMPLE_N^d cells."""

    def __init__(self, procs: int | None = None):
        import oracle
        oracle.build_oracle()  # once, before the workers load it
        self.procs = procs or len(os.sched_getaffinity(0))
        # one BLAS thread per process (the processes already cover the cores): the
        # spawned interpreters read these when they first import numpy
        saved = {v: os.environ.get(v) for v in _ONE_THREAD}
        os.environ.update({v: "1" for v in _ONE_THREAD})
        try:
            self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_worker_init,
                                                     initargs=(ORACLE_SAMPLE_N,))
        finally:
            for v, old in saved.items():
                if old is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = old
        from paper_1908_05834_gb300 import inputs
        self.cells = inputs.workload(WORKLOAD, n=ORACLE_SAMPLE_N).nc

    def step(self, k: int) -> float:
        """Step k on every process; returns the wall time."""
        t = time.perf_counter()
        self.pool.map(_oracle_worker_step, [k] * self.procs, chunksize=1)
        return time.perf_counter() - t

    def close(self):
        self.pool.close()
        self.pool.join()

    def sample_text(self, steps: int, seconds: float) -> str:
        return (f"{self.procs} processes (one per host core, {cpu_model()}), each stepping its own copy of the "
                f"same recipe at {ORACLE_SAMPLE_N}x{ORACLE_SAMPLE_N} ({self.cells} cells) for {steps} steps, "
                f"{seconds:.1f} s wall; serial C + numpy/scipy (SuperLU) per process")


def cpu_baseline(seconds: float):
    pool = OraclePool()
    try:
        pool.step(0)  # warm-up (imports, first factorisation)
        t, k = 0.0, 0
        while t < seconds and k < 20:
            t += pool.step(1 + k)
            k += 1
    finally:
        pool.close()
    rate = pool.cells * pool.procs * k / t
    return {"value": round(rate, 1), "unit": UNIT, "cores": pool.procs, "kind": "oracle",
            "sample": pool.sample_text(k, t)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    pool = OraclePool()
    try:
        for st in range(args.warmup):
            pool.step(st)
        t = 0.0
        for k in range(args.steps):
            t += pool.step(args.warmup + k)
    finally:
        pool.close()
    value = pool.cells * pool.procs * args.steps / t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded analytic fields and meshes)",
        "config": {"workload": f"{WORKLOAD} recipe, oracle sample at {ORACLE_SAMPLE_N}^2 per process",
                   "cells": pool.cells * pool.procs},
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                         "sample": pool.sample_text(args.steps, t)},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--n", type=int, default=None, help="cells per axis (same recipe; for small profiling runs)")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--qp-tol", type=float, default=None, help="default: the library's default")
    p.add_argument("--qp-max-refine", type=int, default=None,
                   help="cap on interior-point iterations (default: the library's); for short profiling runs")
    p.add_argument("--no-serve", action="store_true", help="skip the batched and served measurements")
    p.add_argument("--batch-count", type=int, default=8)
    p.add_argument("--batch-steps", type=int, default=2)
    p.add_argument("--serve-requests", type=int, default=12)
    p.add_argument("--serve-steps", type=int, default=3)
    p.add_argument("--serve-slots", type=int, default=12)
    p.add_argument("--serve-max-cells", type=int, default=150000)
    p.add_argument("--profile", action="store_true",
                   help="a run to capture under a profiler: the steps and the stage replays only (no clock "
                        "sampling subprocess, no end-to-end, serving or CPU runs); its line is not a bench result")
    args = p.parse_args()
    rank, world, local_rank = _env_rank()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
