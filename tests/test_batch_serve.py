"""Batching and serving on the GPU, through the C ABI.

* bchar_step_batch gives, per instance, bitwise the result of a plain
  bchar_step (each instance runs the same kernels in the same order).
* bchar_set_velocity_scaled(s) equals bchar_set_velocity of the host-scaled
  field (one correctly rounded FP64 product either way).
* bchar_device_bytes stays within bchar_estimate_device_bytes.
* A request served in a mix of concurrent requests returns bitwise what it
  returns alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1908_05834_gb300 import bchar, inputs, serve  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [("vortex2d_1024", 40, bchar.FP32_SPLIT), ("vortex2d_32", 33, bchar.FP64), ("deform3d_128", 12, bchar.FP32_SPLIT)]


def _options(precision):
    return bchar.default_options(precision=precision, qp_tol=1e-10)


def _handle(wl, precision):
    stream = torch.cuda.Stream()
    m = bchar.Mesh(wl.coords, wl.phi, _options(precision), stream=stream.cuda_stream)
    return m, stream


def test_batch_equals_plain_bitwise():
    wls = [inputs.workload(name, n=n) for name, n, _ in CASES]
    plain = [_handle(wl, p) for wl, (_, _, p) in zip(wls, CASES)]
    batch = [_handle(wl, p) for wl, (_, _, p) in zip(wls, CASES)]
    cs_p = [torch.tensor(wl.c0, dtype=torch.float64, device="cuda") for wl in wls]
    cs_b = [c.clone() for c in cs_p]
    out_p = [torch.empty_like(c) for c in cs_p]
    out_b = [torch.empty_like(c) for c in cs_b]
    torch.cuda.synchronize()
    for step in range(2):
        infos_p = []
        for i, (wl, (m, s)) in enumerate(zip(wls, plain)):
            m.set_velocity(wl.faces(step))
            infos_p.append(m.step(wl.dt, cs_p[i], out_p[i]))
            s.synchronize()
        for wl, (m, _) in zip(wls, batch):
            m.set_velocity(wl.faces(step))
        infos_b, sts = bchar.step_batch([m for m, _ in batch], [wl.dt for wl in wls], cs_b, out_b)
        assert sts == [0, 0, 0]
        torch.cuda.synchronize()
        for i in range(3):
            assert torch.equal(out_p[i], out_b[i]), f"instance {i} differs at step {step}"
            for key in ("nnz", "cg_iters", "mass_after", "kkt_rel"):
                assert infos_p[i][key] == infos_b[i][key]
        cs_p, out_p = out_p, cs_p
        cs_b, out_b = out_b, cs_b
    for m, _ in plain + batch:
        m.close()


def test_batch_rejects_duplicates():
    wl = inputs.workload("vortex2d_32", n=16)
    m, _ = _handle(wl, bchar.FP64)
    c = torch.tensor(wl.c0, dtype=torch.float64, device="cuda")
    o = torch.empty_like(c)
    with pytest.raises(bchar.BcharError) as e:
        bchar.step_batch([m, m], [wl.dt, wl.dt], [c, c], [o, o])
    assert e.value.name == "INVALID_ARG"
    m.close()


def test_scaled_velocity_equals_scaled_field():
    wl = inputs.workload("vortex2d_1024", n=36)
    s = 0.6180339887498949
    outs = []
    for scaled_on_device in (True, False):
        m, stream = _handle(wl, bchar.FP32_SPLIT)
        if scaled_on_device:
            m.set_velocity(wl.faces(0), scale=s)
        else:
            m.set_velocity([f * s for f in wl.faces(0)])
        c = torch.tensor(wl.c0, dtype=torch.float64, device="cuda")
        o = torch.empty_like(c)
        m.step(wl.dt, c, o)
        stream.synchronize()
        outs.append(o.cpu())
        m.close()
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("name,n,precision", [("vortex2d_1024", 64, bchar.FP32_SPLIT), ("vortex2d_32", 48, bchar.FP64),
                                              ("deform3d_128", 16, bchar.FP32_SPLIT)])
def test_footprint_within_estimate(name, n, precision):
    wl = inputs.workload(name, n=n)
    est = bchar.estimate_device_bytes(wl.coords, _options(precision))
    m, stream = _handle(wl, precision)
    c = torch.tensor(wl.c0, dtype=torch.float64, device="cuda")
    o = torch.empty_like(c)
    for step in range(2):
        m.set_velocity(wl.faces(step))
        m.step(wl.dt, c, o)
        c, o = o, c
    stream.synchronize()
    now, peak = m.device_bytes()
    assert 0 < now <= peak <= est, (now, peak, est)
    m.close()


def _small_requests():
    spec = [(2, 48, 4), (3, 12, 3), (2, 64, 3), (3, 16, 2), (2, 40, 4), (3, 10, 3)]
    reqs = []
    for rid, (dim, n, steps) in enumerate(spec):
        reqs.append(inputs.ServeRequest(rid=rid, arrival_s=0.0, dim=dim, n=n, amplitude=0.5 + 0.25 * rid,
                                        cfl=1.0 + 0.5 * rid, steps=steps, phi_seed=100 + rid))
    return reqs


def test_served_alone_equals_in_mix():
    reqs = _small_requests()
    prepared = {r.rid: r.materialize() for r in reqs}
    opts = _options(bchar.FP32_SPLIT)
    ex = serve.GpuExecutor(prepared, opts)
    est = serve.estimator_for(prepared, opts)
    mix = serve.Server(ex, est, budget_bytes=120e9, max_active=len(reqs)).run(reqs)
    alone = serve.Server(ex, est, budget_bytes=120e9, max_active=1).run(reqs)
    for a, b in zip(mix, alone):
        assert a.status == "ok" and b.status == "ok", (a.status, b.status)
        assert np.array_equal(a.c, b.c), f"request {a.rid} differs in the mix"
        assert a.peak_bytes <= a.est_bytes
    s = serve.summarize(mix)
    assert s["ok"] == len(reqs) and s["p99_ms"] >= s["p50_ms"] > 0
    # mass is conserved by every served request (phi = 1 in 2D; porous in 3D)
    for r in reqs:
        coords, phi, _, c0 = prepared[r.rid]
        vol = np.prod(np.meshgrid(*[np.diff(c) for c in reversed(coords)], indexing="ij"), axis=0).reshape(-1)
        m0 = float(np.sum(vol * phi * c0))
        m1 = float(np.sum(vol * phi * mix[r.rid].c))
        assert abs(m1 - m0) <= 1e-12 * m0
