"""bchar_mass_noalloc: the porous mass without any device allocation.

It is for callers that cannot allocate device memory where they need the
value (a fixed memory budget, a framework's own pool, or no implicit
synchronisation allowed mid-step).  Checked through the C ABI against the
masses bchar_step reports for the same c, on two calls in a row (the scratch
array is shared and keeps the previous call's contents), in FP64 and FP32,
and the size limit.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1908_05834_gb300 import inputs

pytestmark = pytest.mark.gpu

MASS_TOL = 1e-12  # the relative mass tolerance of the other GPU tests


def _volphi(wl):
    w = [np.diff(c) for c in wl.coords]
    vol = np.multiply.outer(w[1], w[0]) if wl.dim == 2 else np.multiply.outer(np.multiply.outer(w[2], w[1]), w[0])
    return np.ascontiguousarray(vol.reshape(-1) * wl.phi)


@pytest.mark.parametrize("name,n", [("vortex2d_1024", 45), ("deform3d_128", 12)])
def test_mass_noalloc_matches_step_masses(name, n):
    import torch
    from paper_1908_05834_gb300 import build
    build.build()
    from paper_1908_05834_gb300 import bchar
    wl = inputs.workload(name, n=n)
    mesh = bchar.Mesh(wl.coords, wl.phi)
    mesh.set_velocity(wl.faces(2))
    c_in = torch.tensor(wl.c0, dtype=torch.float64, device="cuda")
    c_out = torch.empty_like(c_in)
    info = mesh.step(wl.dt, c_in, c_out)
    vp = torch.tensor(_volphi(wl), device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for c, want in [(c_in, info["mass_before"]), (c_out, info["mass_after"])] * 2:  # two calls in a row each
        out.fill_(np.nan)
        st = bchar.bchar_mass_noalloc(vp.data_ptr(), c.data_ptr(), bchar.C_F64, wl.nc, out.data_ptr(), stream)
        assert st == bchar.BCHAR_OK
        torch.cuda.synchronize()
        assert abs(out.item() - want) <= MASS_TOL * abs(want)
    c32 = c_out.to(torch.float32)
    st = bchar.bchar_mass_noalloc(vp.data_ptr(), c32.data_ptr(), bchar.C_F32, wl.nc, out.data_ptr(), stream)
    assert st == bchar.BCHAR_OK
    torch.cuda.synchronize()
    want32 = float(np.sum(_volphi(wl) * c32.cpu().numpy().astype(np.float64)))
    assert abs(out.item() - want32) <= MASS_TOL * abs(want32)
    mesh.close()


def test_mass_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1908_05834_gb300 import build
    build.build()
    from paper_1908_05834_gb300 import bchar
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    # the pointers are never read when the size is refused
    assert bchar.bchar_mass_noalloc(x.data_ptr(), x.data_ptr(), bchar.C_F64, (1 << 24) + 1, out.data_ptr(),
                                    stream) == 8  # BCHAR_ERR_CAPACITY
    assert bchar.bchar_mass_noalloc(x.data_ptr(), x.data_ptr(), bchar.C_F64, 0, out.data_ptr(), stream) == 1
    assert bchar.bchar_mass_noalloc(x.data_ptr(), x.data_ptr(), bchar.C_F64, 4, out.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    assert out.item() == 4.0
