"""Serving loop: a stream of independent transport requests on one GPU.

Each request is a small B-char problem (mesh, porosity, a velocity field
u(x) g(t), an initial concentration, dt and a number of steps) that arrives at
some time and wants its final concentration back.  The server keeps every
admitted request's mesh, weights and concentration resident on the device and
runs the requests concurrently, each from its own host thread on its own CUDA
stream, so that their kernels and host round trips overlap (continuous
batching: a request starts as soon as a slot and memory are free, and a
finishing request frees both at once).

Admission is first-come first-served: the oldest waiting request is admitted
when it has arrived, fewer than ``max_active`` requests run, and its device
footprint estimate (``bchar_estimate_device_bytes``) fits in what is left of
the memory budget; later requests wait behind it (no overtaking, so no
starvation).  A request whose estimate exceeds the whole budget is rejected.
A running request reports the device memory it holds after every step; when
that exceeds its estimate (a step whose rows outgrow the row slab's initial
width holds more than the estimate), the larger figure is charged against the
budget from then on, so later admissions wait instead of over-committing the
device.

Every step runs in the library's kernels (``bchar.Mesh.step``); this module
only schedules.  The scheduler itself takes the executor and the estimator as
arguments, so its rules are testable without a GPU.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field
from typing import Any, Callable

import numpy as np


@dataclass
class Result:
    rid: int
    arrival_s: float          # offsets from the start of the run
    admitted_s: float
    finished_s: float
    cells: int
    steps: int
    est_bytes: int
    status: str = "ok"        # "ok", "rejected: ...", or the error text
    c: np.ndarray | None = None
    peak_bytes: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def latency_s(self) -> float:
        return self.finished_s - self.arrival_s


class Server:
    """First-come first-served admission under a device-memory budget and a
    limit on concurrent requests; one host thread per running request.

    executor(request, report) -> dict with at least "c" (final concentration,
    host) and optionally "peak_bytes"; it may raise, which fails that request
    only.  report(bytes) may be called any number of times while it runs, with
    the device memory the request holds.  estimator(request) -> int bytes.
    clock() -> seconds."""

    def __init__(self, executor: Callable[[Any], dict], estimator: Callable[[Any], int],
                 budget_bytes: float = 120e9, max_active: int = 32, clock: Callable[[], float] = time.perf_counter):
        if max_active < 1 or budget_bytes <= 0:
            raise ValueError("max_active >= 1 and budget_bytes > 0 required")
        self.executor = executor
        self.estimator = estimator
        self.budget = float(budget_bytes)
        self.max_active = int(max_active)
        self.clock = clock
        self.peak_used = 0.0          # largest sum of admitted estimates
        self.peak_active = 0
        self.admission_log: list[tuple[float, int, float]] = []  # (time, rid, bytes in use after admission)
        self.overruns: list[tuple[float, int, int, int]] = []     # (time, rid, estimate, reported bytes)

    def run(self, requests) -> list[Result]:
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival_s, r.rid)))
        cond = threading.Condition()
        results: dict[int, Result] = {}
        active: dict[int, threading.Thread] = {}
        charged: dict[int, float] = {}  # bytes each running request holds against the budget
        used = [0.0]
        t0 = self.clock()

        def now() -> float:
            return self.clock() - t0

        def reporter(rid, est):
            def report(nbytes):
                with cond:
                    extra = float(nbytes) - charged[rid]
                    if extra > 0:
                        if charged[rid] == est:
                            self.overruns.append((now(), rid, est, int(nbytes)))
                        charged[rid] = float(nbytes)
                        used[0] += extra
                        self.peak_used = max(self.peak_used, used[0])
            return report

        def worker(req, est, admitted):
            try:
                out = self.executor(req, reporter(req.rid, est))
                res = Result(req.rid, req.arrival_s, admitted, now(), req.nc, req.steps, est, "ok", out.get("c"),
                             int(out.get("peak_bytes", 0)), {k: v for k, v in out.items() if k not in ("c",)})
            except Exception as e:  # the request fails, the server goes on
                res = Result(req.rid, req.arrival_s, admitted, now(), req.nc, req.steps, est, f"error: {e}")
            with cond:
                used[0] -= charged.pop(req.rid)
                del active[req.rid]
                results[req.rid] = res
                cond.notify_all()

        with cond:
            while pending or active:
                # admit in order while the head fits
                while pending:
                    req = pending[0]
                    t = now()
                    if req.arrival_s > t:
                        break
                    est = int(self.estimator(req))
                    if est > self.budget:
                        pending.popleft()
                        results[req.rid] = Result(req.rid, req.arrival_s, t, t, req.nc, req.steps, est,
                                                  "rejected: estimate exceeds the memory budget")
                        continue
                    if len(active) >= self.max_active or used[0] + est > self.budget:
                        break
                    pending.popleft()
                    used[0] += est
                    charged[req.rid] = float(est)
                    self.peak_used = max(self.peak_used, used[0])
                    self.admission_log.append((t, req.rid, used[0]))
                    th = threading.Thread(target=worker, args=(req, est, t), daemon=True)
                    active[req.rid] = th
                    self.peak_active = max(self.peak_active, len(active))
                    th.start()
                # sleep until the head arrives or a request finishes
                timeout = None
                if pending and pending[0].arrival_s > now():
                    timeout = pending[0].arrival_s - now()
                if pending or active:
                    cond.wait(timeout)
        return [results[r.rid] for r in sorted(requests, key=lambda r: r.rid)]


def summarize(results: list[Result]) -> dict:
    """Throughput (cell-steps/s over the makespan) and latency percentiles of the finished requests."""
    ok = [r for r in results if r.status == "ok"]
    if not ok:
        return {"requests": len(results), "ok": 0}
    lat = np.array([r.latency_s for r in ok]) * 1e3
    start = min(r.arrival_s for r in ok)
    end = max(r.finished_s for r in ok)
    cell_steps = sum(r.cells * r.steps for r in ok)
    out = {"requests": len(results), "ok": len(ok), "cell_steps": int(cell_steps),
           "makespan_s": round(end - start, 4), "cell_steps_per_s": round(cell_steps / (end - start), 1),
           "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
           "max_ms": round(float(lat.max()), 3)}
    stages: dict[str, float] = {}
    for r in ok:
        for name, ms in r.extra.get("stage_ms", {}).items():
            stages[name] = stages.get(name, 0.0) + ms
    if stages:  # summed over requests (concurrent requests overlap, so the sum exceeds the makespan)
        out["stage_ms_sum"] = {k: round(v, 1) for k, v in stages.items()}
    return out


# ---------------------------------------------------------------- the GPU executor

class GpuExecutor:
    """Runs one request through the C ABI on its own CUDA stream: create the
    mesh, upload the base face velocities and c0 once, then per step
    ``bchar_set_velocity_scaled`` (factor g(t) on the device) and
    ``bchar_step``; copy the final c back and free the handle.

    ``prepared`` maps rid -> (coords, phi, faces, c0) host arrays (the client's
    payload, built before the run); ``options`` is a bchar.Options."""

    def __init__(self, prepared: dict, options, device: int = 0):
        self.prepared = prepared
        self.options = options
        self.device = device

    def __call__(self, req, report=None) -> dict:
        import torch
        from . import bchar
        torch.cuda.set_device(self.device)
        coords, phi, faces, c0 = self.prepared[req.rid]
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            mesh = bchar.Mesh(coords, phi, self.options, stream=stream.cuda_stream)
            try:
                fdev = [torch.from_numpy(np.ascontiguousarray(f).reshape(-1)).to("cuda") for f in faces]
                c = torch.from_numpy(np.ascontiguousarray(c0, dtype=np.float64)).to("cuda")
                out = torch.empty_like(c)
                iters = 0
                stage_ms: dict[str, float] = {}
                for k in range(req.steps):
                    mesh.set_velocity(fdev, scale=req.time_factor(k))
                    info = mesh.step(req.dt, c, out)
                    iters += info["cg_iters"]
                    for name, ms in info["ms_stage"].items():
                        stage_ms[name] = stage_ms.get(name, 0.0) + ms
                    c, out = out, c
                    if report is not None:
                        report(mesh.device_bytes()[1])
                host = c.cpu().numpy()
                peak = mesh.device_bytes()[1]
            finally:
                mesh.close()
        return {"c": host, "peak_bytes": peak, "cg_iters": iters, "stage_ms": stage_ms}


def estimator_for(prepared: dict, options) -> Callable[[Any], int]:
    from . import bchar

    def est(req) -> int:
        return bchar.estimate_device_bytes(prepared[req.rid][0], options)
    return est
