"""Host-side rules of the serving loop (no GPU): first-come first-served
admission, the memory budget, the limit on running requests, rejection and
failure isolation.  The executor is a fake that sleeps."""
import sys
import threading
import time
from dataclasses import dataclass

import pytest

from paper_1908_05834_gb300 import serve
from paper_1908_05834_gb300.inputs import serving_requests


@dataclass
class Req:
    rid: int
    arrival_s: float
    nc: int
    steps: int = 1
    work_s: float = 0.02
    fail: bool = False
    report_bytes: int | None = None  # device memory the request reports once it runs


def fake_executor(running: list, lock: threading.Lock):
    def run(req, report):
        with lock:
            running.append(req.rid)
        if req.report_bytes is not None:
            report(req.report_bytes)
        time.sleep(req.work_s)
        with lock:
            running.remove(req.rid)
        if req.fail:
            raise RuntimeError("planted failure")
        return {"c": [req.rid], "peak_bytes": req.nc}
    return run


def by_cells(req):
    return req.nc


def test_all_requests_answered_in_rid_order():
    reqs = [Req(i, 0.001 * i, 100 + i) for i in range(12)]
    srv = serve.Server(fake_executor([], threading.Lock()), by_cells, budget_bytes=1e9, max_active=4)
    res = srv.run(reqs)
    assert [r.rid for r in res] == list(range(12))
    assert all(r.status == "ok" and r.c == [r.rid] for r in res)
    assert all(r.finished_s >= r.admitted_s >= r.arrival_s - 1e-9 for r in res)


def test_budget_and_slot_limits_hold():
    running, lock = [], threading.Lock()
    reqs = [Req(i, 0.0, nc) for i, nc in enumerate([40, 30, 30, 50, 10, 20, 60, 5, 25, 35])]
    srv = serve.Server(fake_executor(running, lock), by_cells, budget_bytes=100, max_active=3)
    res = srv.run(reqs)
    assert all(r.status == "ok" for r in res)
    assert srv.peak_used <= 100
    assert all(used <= 100 for _, _, used in srv.admission_log)
    assert srv.peak_active <= 3


def test_first_come_first_served():
    reqs = [Req(i, 0.002 * i, 10 + (i % 3) * 40) for i in range(10)]
    srv = serve.Server(fake_executor([], threading.Lock()), by_cells, budget_bytes=100, max_active=2)
    srv.run(reqs)
    order = [rid for _, rid, _ in srv.admission_log]
    assert order == sorted(order)  # admitted in arrival order: nobody overtakes


def test_continuous_batching_fills_freed_slots():
    # a long request and many short ones arriving together: the short ones
    # flow through the other slot while the long one runs
    reqs = [Req(0, 0.0, 1, work_s=0.3)] + [Req(i, 0.0, 1, work_s=0.02) for i in range(1, 9)]
    srv = serve.Server(fake_executor([], threading.Lock()), by_cells, budget_bytes=1e9, max_active=2)
    res = srv.run(reqs)
    assert srv.peak_active == 2
    long_done = res[0].finished_s
    assert sum(r.finished_s < long_done for r in res[1:]) >= 6


def test_oversize_rejected_and_failure_isolated():
    reqs = [Req(0, 0.0, 500), Req(1, 0.0, 10, fail=True), Req(2, 0.0, 10)]
    srv = serve.Server(fake_executor([], threading.Lock()), by_cells, budget_bytes=100, max_active=2)
    res = srv.run(reqs)
    assert res[0].status.startswith("rejected")
    assert res[1].status.startswith("error") and "planted" in res[1].status
    assert res[2].status == "ok"


def test_reported_footprint_above_the_estimate_delays_admission():
    # request 0 is estimated at 30 but holds 90 once it runs: request 1 (30)
    # would fit beside the estimate (60 <= 100) but not beside the 90
    reqs = [Req(0, 0.0, 30, work_s=0.25, report_bytes=90), Req(1, 0.05, 30, work_s=0.0)]
    srv = serve.Server(fake_executor([], threading.Lock()), by_cells, budget_bytes=100, max_active=4)
    res = srv.run(reqs)
    assert all(r.status == "ok" for r in res)
    assert res[1].admitted_s >= res[0].finished_s - 1e-3
    assert [(rid, est, got) for _, rid, est, got in srv.overruns] == [(0, 30, 90)]
    assert srv.peak_used == 90


def test_reported_footprint_below_the_estimate_keeps_the_estimate():
    # the estimate stays charged when a request reports less (it may still grow)
    reqs = [Req(0, 0.0, 30, work_s=0.25, report_bytes=10), Req(1, 0.05, 40, work_s=0.0)]
    srv = serve.Server(fake_executor([], threading.Lock()), by_cells, budget_bytes=60, max_active=4)
    res = srv.run(reqs)
    assert res[1].admitted_s >= res[0].finished_s - 1e-3
    assert srv.overruns == [] and srv.peak_used == 40


def test_waits_for_arrivals():
    reqs = [Req(0, 0.0, 1, work_s=0.0), Req(1, 0.15, 1, work_s=0.0)]
    srv = serve.Server(fake_executor([], threading.Lock()), by_cells, budget_bytes=10, max_active=4)
    res = srv.run(reqs)
    assert res[1].admitted_s >= 0.15 - 1e-3


def test_summary_percentiles():
    res = [serve.Result(i, 0.0, 0.0, 0.001 * (i + 1), 100, 2, 1) for i in range(100)]
    s = serve.summarize(res)
    assert s["ok"] == 100 and s["cell_steps"] == 100 * 100 * 2
    assert abs(s["p50_ms"] - 50.5) < 1e-6 and abs(s["p99_ms"] - 99.01) < 1e-6


def test_serving_stream_recipe():
    rs = serving_requests(512)
    assert len(rs) == 512
    two = [r for r in rs if r.dim == 2]
    three = [r for r in rs if r.dim == 3]
    assert 0.5 < len(two) / 512 < 0.7
    assert all(64 <= r.n <= 1024 for r in two) and all(32 <= r.n <= 160 for r in three)
    assert all(10 <= r.steps <= 100 and 0.5 <= r.amplitude <= 2 and 0.5 <= r.cfl <= 4 for r in rs)
    gaps = [b.arrival_s - a.arrival_s for a, b in zip(rs, rs[1:])]
    assert all(g >= 0 for g in gaps) and 0.0015 < sum(gaps) / len(gaps) < 0.0025
    # dt from the CFL: A U_max dt / (h phi_min) = CFL
    for r in rs[:20]:
        umax, phimin = (1.0, 1.0) if r.dim == 2 else (2.0, 0.1)
        assert r.amplitude * umax * r.dt * r.n / phimin == pytest.approx(r.cfl, rel=1e-12)
    assert serving_requests(8) == serving_requests(8)  # seeded


def test_serving_request_payloads():
    """The arrays of a 2D and a 3D request: RT0 face counts, porosity ranges,
    c0 in [0, 1], the scaled time factor and a divergence-free base field."""
    import math
    import numpy as np
    rs = serving_requests(64)
    r2 = next(r for r in rs if r.dim == 2 and r.n <= 200)
    r3 = next(r for r in rs if r.dim == 3 and r.n <= 48)
    for r in (r2, r3):
        coords, phi, faces, c0 = r.materialize()
        n = r.n
        assert len(coords) == r.dim and all(len(c) == n + 1 for c in coords)
        assert phi.shape == (n ** r.dim,) and c0.shape == (n ** r.dim,)
        assert np.all((c0 >= 0) & (c0 <= 1)) and c0.max() == 1.0
        for a, f in enumerate(faces):
            assert f.size == (n + 1) * n ** (r.dim - 1)
        if r.dim == 2:
            assert np.all(phi == 1.0)
        else:
            assert phi.min() >= 0.1 and phi.max() <= 0.3
        # RT0 face fluxes of the separable field: zero net flux per cell
        h = 1.0 / n
        div = sum(np.diff(f, axis=r.dim - 1 - a) * h ** (r.dim - 1) for a, f in enumerate(faces))
        assert np.abs(div).max() <= 1e-12 * max(np.abs(f).max() for f in faces)
        t = (0.5) * r.dt
        assert r.time_factor(0) == pytest.approx(r.amplitude * math.cos(math.pi * t / r.T), rel=1e-14)


@pytest.mark.parametrize("name", ["vortex2d_32", "vortex2d_1024", "deform3d_128", "deform3d_256"])
def test_workload_descriptions_follow_the_recipes(name):
    """The one-line description a measurement records names the recipe the
    workload actually builds: its size, time step, storage and precision."""
    import numpy as np
    from paper_1908_05834_gb300 import inputs
    assert name in inputs.WORKLOADS
    n = 6
    wl = inputs.workload(name, n=n)
    text = inputs.describe(name, n)
    size = f"{n}x{n}" if wl.dim == 2 else f"{n}^3"
    assert text.startswith(size) or text.startswith(f"uniform {size}")
    assert f"dt={wl.dt:g}" in text
    assert ("stored in FP32" in text) == (wl.c_dtype == "f32")
    assert ("FP32 tracking" in text) == (wl.precision == "fp32split")
    assert ("stretched" in text) == (len(set(np.round(np.diff(wl.coords[0]), 12))) > 1)
    assert ("steady" in text) == (wl.T is None)
    d = int(name.split("_")[1])  # the default size is in the name
    assert (f"{d}x{d}" if wl.dim == 2 else f"{d}^3") in inputs.describe(name)


def test_gpu_executor_host_logic_with_a_fake_mesh(monkeypatch):
    """GpuExecutor's bookkeeping without a GPU: one report per step of the
    handle's device bytes (charged by the server above the estimate), the CG
    iterations and stage times summed over the steps, the peak returned, the
    final c copied back.  The CUDA calls and the mesh are replaced by fakes."""
    import contextlib
    import types

    import numpy as np
    import torch

    from paper_1908_05834_gb300 import inputs

    class FakeStream:
        cuda_stream = 0

    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    to = torch.Tensor.to
    # a device copy: a new tensor, like a real upload
    monkeypatch.setattr(torch.Tensor, "to", lambda self, *a, **k: self.clone() if a[:1] == ("cuda",) else to(self, *a, **k))

    class FakeMesh:
        def __init__(self, coords, phi, opts, stream=None):
            self.bytes = 100

        def set_velocity(self, faces, scale=1.0):
            pass

        def step(self, dt, c, out):
            out.copy_(c * 0.5)
            self.bytes += 50
            return {"cg_iters": 3, "ms_stage": {"total": 1.5}}

        def device_bytes(self):
            return self.bytes, self.bytes

        def close(self):
            pass

    fake = types.SimpleNamespace(Mesh=FakeMesh, estimate_device_bytes=lambda coords, opts: 120)
    import paper_1908_05834_gb300 as pkg
    monkeypatch.setitem(sys.modules, "paper_1908_05834_gb300.bchar", fake)
    monkeypatch.setattr(pkg, "bchar", fake, raising=False)

    req = inputs.ServeRequest(rid=0, arrival_s=0.0, dim=2, n=16, amplitude=1.0, cfl=1.0, steps=3, phi_seed=1)
    prepared = {0: req.materialize()}
    srv = serve.Server(serve.GpuExecutor(prepared, None), serve.estimator_for(prepared, None),
                       budget_bytes=1e9, max_active=2)
    (res,) = srv.run([req])
    assert res.status == "ok" and res.est_bytes == 120 and res.peak_bytes == 250
    assert res.extra["cg_iters"] == 9 and res.extra["stage_ms"] == {"total": 4.5}
    assert np.allclose(res.c, prepared[0][3] * 0.125)
    assert [(rid, est, got) for _, rid, est, got in srv.overruns] == [(0, 120, 150)]
    assert srv.peak_used == 250
