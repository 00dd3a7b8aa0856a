"""Benchmark: B-char cell-steps/s on the 1024x1024 single-vortex workload.

One "step" is one time step of the whole hot path on one GPU: setting the
step's velocity (with its checks) and bchar_step (tracking, intersections,
scalings, minimisation, weights, update), through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own replica of the workload on its
own GPU (the method is single-GPU; replicas only) and rank 0 prints one JSON
line with the whole-job rate.  --impl reference times the FP64 CPU oracle on
the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
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
ORACLE_SAMPLE_N = 128  # cells per axis of the oracle's bounded sample (same recipe)


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


def algorithmic_bytes(stage: str, nc: int, nnz: int) -> int:
    """Bytes one launch of a stage must move at minimum (the per-unit figures
    of the design notes times the units of one launch)."""
    if stage == "cg_matvec":
        # per entry, once through the row view and once through the column
        # view: column/row index 4 B + a^2 8 B; per node (2 nc): pointer 8 B,
        # diagonal 8 B, p read 8 B, q write 8 B
        return nnz * 2 * (4 + 8) + 2 * nc * (8 + 8 + 8 + 8)
    if stage == "smooth":
        # one FP32 damped-Jacobi sweep of the finest multigrid level: 2 nc
        # nodes, 2 nnz off-diagonal entries (value 4 B + column 4 B); per node
        # pointer 8 B, x, b, diagonal read and x_out written (4 B each)
        return 2 * nnz * (4 + 4) + 2 * nc * (8 + 4 * 4)
    if stage == "update":
        # per entry: column 4 B + weight 8 B; per cell: row pointer 8 B,
        # c_in 8 B, c_out 8 B, |K|_phi 8 B
        return nnz * (4 + 8) + nc * (8 + 8 + 8 + 8)
    raise KeyError(stage)


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
    faces_dev = []
    for st in range(nsteps):
        f = wl.faces(st % wl.steps)
        faces_dev.append([torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to(dev) for a in f])
    opts = bchar.default_options(precision=bchar.FP32_SPLIT if wl.precision == "fp32split" else bchar.FP64,
                                 qp_max_iter=args.qp_max_iter, qp_tol=args.qp_tol)
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
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    sampler = ClockSampler(local_rank)
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

    # dominant kernel: live CUDA-event timing of the stages on the last step's data
    last = infos[-1]
    # the NVTX range lets a profiler select these replays (ncu --nvtx --nvtx-include stage_timing/)
    torch.cuda.nvtx.range_push("stage_timing")
    stage_ms = {
        "smooth": mesh.time_stage(bchar.STAGE_SMOOTH, 50),
        "cg_matvec": mesh.time_stage(bchar.STAGE_CG_MATVEC, 50),
        "update": mesh.time_stage(bchar.STAGE_UPDATE, 50),
        "assemble": mesh.time_stage(bchar.STAGE_ASSEMBLE, 5),
        "track": mesh.time_stage(bchar.STAGE_TRACK, 5),
    }
    torch.cuda.nvtx.range_pop()
    cg_mean = statistics.mean(i["cg_iters"] for i in infos)
    step_stage_ms = {k: round(statistics.mean(i["ms_stage"][k] for i in infos), 3) for k in infos[0]["ms_stage"]}
    per_step_ms = {
        "smooth_level0": stage_ms["smooth"] * 2 * cg_mean,  # the finest level's two passes per V-cycle
        "cg_matvec": stage_ms["cg_matvec"] * cg_mean,
        "update": stage_ms["update"],
        "assemble": stage_ms["assemble"],
        "track": stage_ms["track"],
    }
    hbm, peak_kind = _peaks()
    sm_bytes = algorithmic_bytes("smooth", nc, last["nnz"])
    achieved = sm_bytes / (stage_ms["smooth"] * 1e-3) / 1e9
    mv_bytes = algorithmic_bytes("cg_matvec", nc, last["nnz"])
    # DRAM bytes of one finest-level sweep from an ncu capture of the same kernel
    # on the 512x512 case of this recipe (profiles/k_jacobi_vortex2d_512.md:
    # 23.92 MB read, no write reaching DRAM), scaled by cells to this launch
    traffic = round(23.921408e6 / (512 * 512) * nc) if args.workload == WORKLOAD else None
    roofline = {"bound": "hbm", "kernel": "k_jacobi<float> (finest multigrid level, post-smoothing)",
                "achieved": round(achieved, 1),
                "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": traffic,
                "traffic_note": "dram read+write per launch, ncu capture at 512x512 scaled by cells" if traffic else None,
                "peak_source": f"{peak_kind} hbm_gbs (burst copy)", "algorithmic_bytes_per_launch": sm_bytes,
                "mean_launch_ms": round(stage_ms["smooth"], 5),
                "k_cg_matvec": {"achieved": round(mv_bytes / (stage_ms["cg_matvec"] * 1e-3) / 1e9, 1),
                                "frac": round(mv_bytes / (stage_ms["cg_matvec"] * 1e-3) / 1e9 / hbm, 4),
                                "algorithmic_bytes_per_launch": mv_bytes,
                                "mean_launch_ms": round(stage_ms["cg_matvec"], 5)}}

    # end to end through the public API with host buffers
    e2e = run_e2e(args, mesh, wl, bchar, torch, dev)

    # plain vs batched, and the serving loop (one GPU; replicas at N > 1 are not re-measured)
    batched = served = None
    if world == 1 and not args.no_serve:
        batched = run_batched(args, torch, bchar, inputs)
        served = run_served(args, torch, bchar, inputs)

    result = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded analytic fields and meshes)",
        "config": {"workload": f"{args.workload}: {inputs.describe(args.workload, args.n)}",
                   "cells": nc, "cells_per_axis": len(wl.coords[0]) - 1, "parallelism": f"replicas x{world}", "l2": "flushed (256 MB write) between steps",
                   "qp_tol": args.qp_tol, "qp_max_iter": args.qp_max_iter,
                   "qp_note": "the minimisation is solved to qp_tol (relative L1 optimality residual); global mass "
                              "is exact regardless (final column scaling); qp_converged counts the steps that "
                              "reached qp_tol within qp_max_iter"},
        "gpu_launches": int(statistics.mean(i["kernel_launches"] for i in infos) * args.steps) + 0,
        "roofline": roofline,
        "stage_ms_per_step": {k: round(v, 3) for k, v in per_step_ms.items()},
        "step_stage_ms": step_stage_ms,
        "step_stats": {"cg_iters_mean": statistics.mean(i["cg_iters"] for i in infos),
                       "qp_converged": sum(i["qp_converged"] for i in infos),
                       "kkt_rel_max": max(i["kkt_rel"] for i in infos),
                       "max_rel_row_res_max": max(i["max_rel_row_res"] for i in infos),
                       "amg_levels": last["amg_levels"], "amg_coarsest": last["amg_coarsest"], "nnz": last["nnz"],
                       "row_cap": last["row_cap"],
                       "substeps": last["substeps"],
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
        if world == 1 and not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(result), flush=True)
    mesh.close()


def run_e2e(args, mesh, wl, bchar, torch, dev):
    """Same metric through the C ABI with HOST buffers: every step copies the
    step's face velocities and c to the device and reads c back."""
    k = max(1, min(args.steps, 2))
    faces_host = [[torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).pin_memory() for a in wl.faces(st % wl.steps)]
                  for st in range(k)]
    cdt = torch.float32 if wl.c_dtype == "f32" else torch.float64
    c_host = torch.tensor(wl.c0, dtype=cdt).pin_memory()
    back = torch.empty_like(c_host).pin_memory()
    c_dev = torch.empty(wl.nc, dtype=cdt, device=dev)
    out = torch.empty_like(c_dev)
    h2d = sum(f.numel() * 8 for f in faces_host[0]) + c_host.numel() * c_host.element_size()
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
            "d2h_bytes_per_step": int(d2h), "steps": k}


def _serving_options(bchar, args):
    return bchar.default_options(precision=bchar.FP32_SPLIT, qp_tol=args.qp_tol, qp_max_iter=args.qp_max_iter)


def run_batched(args, torch, bchar, inputs):
    """Plain vs batched stepping of the first --batch-count meshes of the
    serving stream (uneven sizes), --batch-steps steps each after one warm-up
    step: plain = one bchar_step after another; batched = bchar_step_batch of
    all instances per step.  Host wall clock around whole steps (every
    instance's step has finished when the call returns)."""
    reqs = inputs.serving_requests(args.batch_count)
    prepared = [r.materialize() for r in reqs]
    opts = _serving_options(bchar, args)

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

    out = {}
    finals = {}
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
            "instances": len(reqs), "steps": args.batch_steps,
            "cells": [r.nc for r in reqs],
            "sample": f"meshes of the first {len(reqs)} requests of the serving stream (seed 4004), "
                      f"{args.batch_steps} timed steps after 1 warm-up step, FP32 split, qp_tol {args.qp_tol}"}


def run_served(args, torch, bchar, inputs):
    """The first --serve-requests requests of the serving stream (Poisson
    arrivals, mean gap 2 ms, 60 % 2D / 40 % 3D, 10-100 steps) through the
    serving loop: 120 GB admission budget, --serve-slots concurrent requests.
    The payloads (mesh, phi, base field, c0) are built before the clock
    starts; latency = finish - arrival, including queueing and the uploads."""
    from paper_1908_05834_gb300 import serve
    reqs = inputs.serving_requests(args.serve_requests)
    t0 = time.perf_counter()
    prepared = {r.rid: r.materialize() for r in reqs}
    prep_s = time.perf_counter() - t0
    opts = _serving_options(bchar, args)
    srv = serve.Server(serve.GpuExecutor(prepared, opts, torch.cuda.current_device()),
                       serve.estimator_for(prepared, opts), budget_bytes=120e9, max_active=args.serve_slots)
    res = srv.run(reqs)
    s = serve.summarize(res)
    s.update({"unit": UNIT, "budget_gb": 120, "slots": args.serve_slots,
              "peak_admitted_gb": round(srv.peak_used / 1e9, 2), "peak_active": srv.peak_active,
              "max_peak_bytes_over_estimate": round(max((r.peak_bytes / r.est_bytes) for r in res
                                                        if r.status == "ok"), 3),
              "footprint_overruns": len(srv.overruns),  # requests charged above their estimate
              "prep_s": round(prep_s, 1),
              "sample": f"first {len(reqs)} of the 512-request serving stream (seed 4004), full step counts, "
                        f"FP32 split, qp_tol {args.qp_tol}"})
    return s


def oracle_sample_step_rate(seconds: float):
    """The FP64 CPU oracle as it stands, timed on this host, on a bounded
    sample of the workload: the same recipe at ORACLE_SAMPLE_N^2 cells,
    consecutive steps until about `seconds` of CPU time."""
    import oracle
    from paper_1908_05834_gb300 import inputs
    wl = inputs.workload(WORKLOAD, n=ORACLE_SAMPLE_N)
    mesh = oracle.Mesh(wl.coords, wl.phi)
    oracle.build_oracle()
    c = wl.c0.astype(np.float64)
    t0 = time.perf_counter()
    steps = 0
    while True:
        r = oracle.step(mesh, wl.faces(steps % wl.steps), wl.dt, c)
        c = r["c"]
        steps += 1
        if time.perf_counter() - t0 >= seconds or steps >= 50:
            break
    t = time.perf_counter() - t0
    return wl.nc * steps / t, steps, t, wl.nc


def cpu_baseline(seconds: float):
    rate, steps, t, nc = oracle_sample_step_rate(seconds)
    return {"value": round(rate, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} consecutive steps of the same recipe at {ORACLE_SAMPLE_N}x{ORACLE_SAMPLE_N} "
                      f"({nc} cells), {t:.1f} s, serial C + numpy/scipy (SuperLU)"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    # each step of --steps/--warmup is one oracle step on the bounded sample
    import oracle
    from paper_1908_05834_gb300 import inputs
    wl = inputs.workload(WORKLOAD, n=ORACLE_SAMPLE_N)
    mesh = oracle.Mesh(wl.coords, wl.phi)
    oracle.build_oracle()
    c = wl.c0.astype(np.float64)
    for st in range(args.warmup):
        c = oracle.step(mesh, wl.faces(st % wl.steps), wl.dt, c)["c"]
    t0 = time.perf_counter()
    for k in range(args.steps):
        c = oracle.step(mesh, wl.faces((args.warmup + k) % wl.steps), wl.dt, c)["c"]
    t = time.perf_counter() - t0
    value = wl.nc * args.steps / t
    sample = (f"{args.steps} steps of the same recipe at {ORACLE_SAMPLE_N}x{ORACLE_SAMPLE_N} ({wl.nc} cells), "
              f"serial C + numpy/scipy (SuperLU)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded analytic fields and meshes)",
        "config": {"workload": f"{WORKLOAD} recipe, oracle sample at {ORACLE_SAMPLE_N}^2", "cells": wl.nc},
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--qp-max-iter", type=int, default=30000)
    p.add_argument("--qp-tol", type=float, default=1e-5)
    p.add_argument("--n", type=int, default=None, help="cells per axis (same recipe; for small profiling runs)")
    p.add_argument("--no-serve", action="store_true", help="skip the batched and served measurements")
    p.add_argument("--batch-count", type=int, default=16)
    p.add_argument("--batch-steps", type=int, default=3)
    p.add_argument("--serve-requests", type=int, default=32)
    p.add_argument("--serve-slots", type=int, default=32)
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
