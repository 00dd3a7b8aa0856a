"""GPU path vs the FP64 CPU oracle, element by element, through the C ABI.

Sizes are chosen so the oracle finishes in seconds while the GPU kernels
still see several blocks/warps and ragged tails (cell counts that are not
multiples of 32), plus sampled rows and invariants at the full workload sizes.

Tolerances (from the arithmetic):
  * FP64 mode: tracked points and A^(0), A^(N) differ from the oracle only by
    rounding order (~1e-15 relative); 1e-10 is used.  Final weights and c
    also depend on how far each side solved the bound-constrained
    minimisation (both by interior-point iterations to their stopping rule,
    the GPU with conjugate-gradient solves of its normal equations): the bar
    is 1e-5 of the row maximum for W and 1e-5 relative L1 for c.
  * FP32-split mode: tracking and intersections in FP32 (6e-8 relative per
    operation, ~1e-6 of a ball radius after the RK4 substeps); a stage point
    that lands within rounding of a face can take the neighbouring cell's
    field, so a few rows may differ by more.  Bar: c within 1e-5 relative L1,
    99.9 % of rows of A^(0) within 1e-4 of the row maximum; the measured
    maximum is reported.
  * Mass: |M^{n+1} - M^n| <= 1e-12 M^n on the GPU in both modes.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1908_05834_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1908_05834_gb300 import build
    build.build()
    from paper_1908_05834_gb300 import bchar
    return bchar


def _case(name):
    if name == "uniform2d":
        wl = inputs.workload("vortex2d_32", n=37)
    elif name == "stretched2d":
        wl = inputs.workload("vortex2d_1024", n=45)
    elif name == "porous3d":
        # an even count, as in the full workload: with an odd count the field's
        # symmetry puts faces of exactly zero normal velocity under the balls'
        # axis points, where every start is a face tie
        wl = inputs.workload("deform3d_128", n=12)
    elif name == "stretched3d":
        # 8^3: the paper's problem is feasible here (an LP decides, see the oracle tests)
        wl = inputs.workload("deform3d_256", n=8)
    elif name == "stretched3d_infeasible":
        # 9^3: the doubling cap makes the paper's problem infeasible; both sides
        # return the unique minimiser of the same elastic penalty (least total violation)
        wl = inputs.workload("deform3d_256", n=9)
    else:
        raise KeyError(name)
    return wl


def _gpu_step(bc, wl, faces, c, precision=0, **opt):
    import torch
    o = bc.default_options(precision=precision, **opt)
    mesh = bc.Mesh(wl.coords, wl.phi, o)
    mesh.set_velocity(faces)
    dt = torch.float32 if np.asarray(c).dtype == np.float32 else torch.float64
    c_in = torch.tensor(np.asarray(c), dtype=dt, device="cuda")
    c_out = torch.empty_like(c_in)
    info = mesh.step(wl.dt, c_in, c_out)
    return mesh, info, c_out.cpu().numpy()


def _csr(mesh, which):
    rp, cols, vals = mesh.export_matrix(which)
    return sp.csr_matrix((vals, cols, rp), shape=(mesh.nc, mesh.nc))


def _row_rel_err(A, B):
    """max over rows of max |A - B| / max |B| in the row (absent entries = 0)."""
    D = (A - B).tocsr()
    Bm = abs(B).max(axis=1).toarray().ravel()
    Dm = abs(D).max(axis=1).toarray().ravel()
    return Dm / np.where(Bm > 0, Bm, 1.0)


CASES = ["uniform2d", "stretched2d", "porous3d", "stretched3d", "stretched3d_infeasible"]


@pytest.mark.parametrize("name", CASES)
def test_tracked_balls_match_oracle_fp64(bc, name):
    wl = _case(name)
    faces = wl.faces(3)
    mesh, info, _ = _gpu_step(bc, wl, faces, wl.c0.astype(np.float64))
    pos, rh, off = mesh.export_tracked()
    om = oracle.Mesh(wl.coords, wl.phi)
    s = oracle.substep_count(om, faces, wl.dt)
    assert info["substeps"] == s
    ooff, ocen, orh = oracle.track_balls(om, faces, wl.dt, s, np.arange(om.nc))
    assert np.array_equal(off, ooff)
    h = min(float(np.min(np.diff(c))) for c in wl.coords)
    err = np.maximum(np.max(np.abs(pos - ocen), axis=1), np.abs(rh - orh))
    ok = err <= 1e-10 * h
    print(f"\n{name}: {np.sum(~ok)} of {ok.size} balls differ (face ties); max err elsewhere {err[ok].max():.1e}")
    assert np.mean(ok) >= 0.995
    if wl.phi.min() == wl.phi.max():
        assert ok.all()  # constant porosity: no tie changes the path beyond rounding
    mesh.close()


@pytest.mark.parametrize("name", CASES)
def test_matrices_match_oracle_fp64(bc, name):
    wl = _case(name)
    faces = wl.faces(3)
    c = wl.c0.astype(np.float64)
    mesh, info, c_gpu = _gpu_step(bc, wl, faces, c)
    ref = oracle.step(oracle.Mesh(wl.coords, wl.phi), faces, wl.dt, c)
    A0, AN, A = _csr(mesh, 0), _csr(mesh, 1), _csr(mesh, 2)
    e0 = _row_rel_err(A0, ref["A0"])
    ok = e0 <= 1e-10
    print(f"\n{name}: A0 rows off by face ties {np.sum(~ok)}/{ok.size}; max elsewhere {e0[ok].max():.1e}; "
          f"interior-point iters {info['ip_iters']} (oracle {ref['iterations']}), cg iters {info['cg_iters']}, "
          f"constraint residual {info['kkt_rel']:.1e}, at bounds {info['n_at_bounds']} (oracle {ref['n_at_bounds']})")
    assert info["qp_converged"]
    assert np.mean(ok) >= 0.99
    if wl.phi.min() == wl.phi.max():
        assert ok.all()
        assert info["void_balls"] == ref["void_balls"] and info["empty_cols"] == ref["empty_cols"]
        assert np.max(_row_rel_err(AN, ref["AN"])) <= 1e-9
    # final weights: the bar is 1e-5 of the row maximum
    vp = oracle.Mesh(wl.coords, wl.phi).volphi()
    W = sp.diags(1.0 / vp) @ A
    assert np.max(_row_rel_err(W.tocsr(), ref["W"])) <= 1e-5
    err = np.abs(c_gpu - ref["c"]).sum() / np.abs(ref["c"]).sum()
    assert err <= 1e-5
    assert abs(info["mass_after"] - info["mass_before"]) <= 1e-12 * info["mass_before"]
    assert info["max_rel_col_res"] <= 1e-13
    mesh.close()


@pytest.mark.parametrize("name,n", [("vortex2d_1024", 24), ("deform3d_128", 8)])
def test_three_balls_per_axis_matches_oracle(bc, name, n):
    """More balls per cell (Sec 4 conclusion on the number of balls): n_b = 3
    per axis (9 balls per square cell in 2D, 27 per cube in 3D) on a stretched
    2D and a porous 3D case, GPU against the oracle with the same packing."""
    wl = inputs.workload(name, n=n)
    faces = wl.faces(2)
    c = wl.c0.astype(np.float64)
    mesh, info, c_gpu = _gpu_step(bc, wl, faces, c, balls_per_axis=3)
    om = oracle.Mesh(wl.coords, wl.phi, nb=3)
    ref = oracle.step(om, faces, wl.dt, c)
    assert mesh.nballs == int(ref["ball_offset"][-1]) >= 9 * om.nc
    e0 = _row_rel_err(_csr(mesh, 0), ref["A0"])
    print(f"\n{name} n_b = 3: {mesh.nballs} balls, A0 rows off by face ties {np.sum(e0 > 1e-10)}/{e0.size}")
    assert np.mean(e0 <= 1e-10) >= 0.99
    assert info["qp_converged"]
    W = sp.diags(1.0 / om.volphi()) @ _csr(mesh, 2)
    assert np.max(_row_rel_err(W.tocsr(), ref["W"])) <= 1e-5
    err = np.abs(c_gpu - ref["c"]).sum() / np.abs(ref["c"]).sum()
    assert err <= 1e-5
    assert abs(info["mass_after"] - info["mass_before"]) <= 1e-12 * info["mass_before"]
    mesh.close()


def test_multilevel_preconditioner_case_matches_oracle(bc):
    """A 96x96 stretched vortex: 18 432 constraint nodes, so the multigrid's
    finest levels exceed one block and run the multi-block V-cycle kernels
    (the smaller cases are cycled by one block alone).  The final weights and
    c match the oracle as on the small cases."""
    wl = inputs.workload("vortex2d_1024", n=96)
    faces = wl.faces(3)
    c = wl.c0.astype(np.float64)
    mesh, info, c_gpu = _gpu_step(bc, wl, faces, c)
    ref = oracle.step(oracle.Mesh(wl.coords, wl.phi), faces, wl.dt, c)
    print(f"\n96^2: levels {info['amg_levels']}, coarsest {info['amg_coarsest']}, interior-point iters "
          f"{info['ip_iters']}, cg iters {info['cg_iters']}")
    assert info["qp_converged"]
    assert info["amg_levels"] >= 3 and 2 * wl.nc > 4096
    vp = oracle.Mesh(wl.coords, wl.phi).volphi()
    W = sp.diags(1.0 / vp) @ _csr(mesh, 2)
    assert np.max(_row_rel_err(W.tocsr(), ref["W"])) <= 1e-5
    err = np.abs(c_gpu - ref["c"]).sum() / np.abs(ref["c"]).sum()
    assert err <= 1e-5
    assert abs(info["mass_after"] - info["mass_before"]) <= 1e-12 * info["mass_before"]
    mesh.close()


@pytest.mark.parametrize("name,width", [("stretched2d", 2), ("porous3d", 8)])
def test_rows_wider_than_the_slab_go_to_the_spill_area(bc, name, width):
    """A slab narrower than most rows: those rows are assembled a second time
    into the spill area, and the step is bitwise the one with the default slab
    (and so still matches the oracle)."""
    wl = _case(name)
    faces = wl.faces(2)
    c = wl.c0.astype(np.float64)
    m1, i1, c1 = _gpu_step(bc, wl, faces, c)
    m2, i2, c2 = _gpu_step(bc, wl, faces, c, slab_width=width)
    assert i1["spill_rows"] == 0 and i2["spill_rows"] > 0
    assert i2["max_row_len"] == i1["max_row_len"] > width
    assert np.array_equal(c1, c2)
    for which in (0, 2):
        r1, r2 = m1.export_matrix(which), m2.export_matrix(which)
        assert all(np.array_equal(x, y) for x, y in zip(r1, r2))
    m1.close()
    m2.close()


def test_vortex32_full_run_fp64(bc):
    """The 32x32 steady vortex, all 20 steps, GPU and oracle side by side."""
    import torch
    wl = inputs.workload("vortex2d_32")
    om = oracle.Mesh(wl.coords, wl.phi)
    mesh = bc.Mesh(wl.coords, wl.phi, bc.default_options())
    c_ref = wl.c0.astype(np.float64)
    c_gpu = torch.tensor(c_ref, device="cuda")
    out = torch.empty_like(c_gpu)
    m0 = oracle.total_mass(om, c_ref)
    for st in range(wl.steps):
        faces = wl.faces(st)
        mesh.set_velocity(faces)
        info = mesh.step(wl.dt, c_gpu, out)
        c_gpu, out = out, c_gpu
        c_ref = oracle.step(om, faces, wl.dt, c_ref)["c"]
        g = c_gpu.cpu().numpy()
        assert np.abs(g - c_ref).sum() / np.abs(c_ref).sum() <= 1e-5, st
        assert abs(info["mass_after"] - info["mass_before"]) <= 1e-12 * m0
    mesh.close()


def test_stretched2d_steps_match_oracle(bc):
    """Consecutive steps of the stretched 2D recipe on one handle (the
    multigrid hierarchy and every buffer reused between steps): each step
    matches the oracle's."""
    import torch
    wl = _case("stretched2d")
    om = oracle.Mesh(wl.coords, wl.phi)
    mesh = bc.Mesh(wl.coords, wl.phi, bc.default_options())
    c_ref = wl.c0.astype(np.float64)
    c_gpu = torch.tensor(c_ref, device="cuda")
    out = torch.empty_like(c_gpu)
    for st in range(3):
        faces = wl.faces(st)
        mesh.set_velocity(faces)
        info = mesh.step(wl.dt, c_gpu, out)
        c_gpu, out = out, c_gpu
        c_ref = oracle.step(om, faces, wl.dt, c_ref)["c"]
        g = c_gpu.cpu().numpy()
        assert info["qp_converged"]
        assert np.abs(g - c_ref).sum() / np.abs(c_ref).sum() <= 1e-5, st
    mesh.close()


def test_porous3d_steps_match_oracle(bc):
    """Consecutive 3D steps on one handle: every step matches the oracle."""
    import torch
    wl = _case("porous3d")
    om = oracle.Mesh(wl.coords, wl.phi)
    mesh = bc.Mesh(wl.coords, wl.phi, bc.default_options())
    c_ref = wl.c0.astype(np.float64)
    c_gpu = torch.tensor(c_ref, device="cuda")
    out = torch.empty_like(c_gpu)
    m0 = oracle.total_mass(om, c_ref)
    for st in range(3):
        faces = wl.faces(st)
        mesh.set_velocity(faces)
        info = mesh.step(wl.dt, c_gpu, out)
        c_gpu, out = out, c_gpu
        c_ref = oracle.step(om, faces, wl.dt, c_ref)["c"]
        g = c_gpu.cpu().numpy()
        assert np.abs(g - c_ref).sum() / np.abs(c_ref).sum() <= 1e-5, st
        assert abs(info["mass_after"] - info["mass_before"]) <= 1e-12 * m0
    mesh.close()


def test_iteration_cap_ends_the_minimisation_and_keeps_bounds_and_mass(bc):
    """With the interior-point iterations capped below what the stopping rule
    needs, the step reports qp_converged = 0, yet every 1 + x is inside the
    bounds (the iterates are interior), the weights are non-negative and the
    global mass is conserved (final column scaling)."""
    import torch
    wl = _case("stretched2d")
    o = bc.default_options(qp_max_refine=4)
    mesh = bc.Mesh(wl.coords, wl.phi, o)
    c = torch.tensor(wl.c0, dtype=torch.float64, device="cuda")
    out = torch.empty_like(c)
    mesh.set_velocity(wl.faces(0))
    info = mesh.step(wl.dt, c, out)
    assert not info["qp_converged"] and info["ip_iters"] == 4
    rp, cols, vals = mesh.export_matrix(2)
    assert vals.min() >= 0.0
    assert abs(info["mass_after"] - info["mass_before"]) <= 1e-12 * info["mass_before"]
    mesh.close()


@pytest.mark.parametrize("name", ["stretched2d", "porous3d"])
def test_fp32_split_error_budget(bc, name):
    wl = _case(name)
    faces = wl.faces(3)
    c = wl.c0.astype(np.float64)
    mesh, info, c_gpu = _gpu_step(bc, wl, faces, c, precision=bc.FP32_SPLIT)
    ref = oracle.step(oracle.Mesh(wl.coords, wl.phi), faces, wl.dt, c)
    e0 = _row_rel_err(_csr(mesh, 0), ref["A0"])
    frac_ok = np.mean(e0 <= 1e-4)
    err_c = np.abs(c_gpu - ref["c"]).sum() / np.abs(ref["c"]).sum()
    print(f"\n{name} FP32 split: A0 max row err {e0.max():.2e}, rows within 1e-4: {frac_ok:.4%}, c L1 {err_c:.2e}")
    assert frac_ok >= 0.999
    assert err_c <= 1e-5
    assert abs(info["mass_after"] - info["mass_before"]) <= 1e-12 * info["mass_before"]
    mesh.close()


FULL_SIZE_IP_ITERS = 25  # interior-point iterations of the 256^3 step


@pytest.mark.parametrize("name,precision", [("vortex2d_1024", 1), ("deform3d_128", 1), ("deform3d_256", 1)])
def test_full_size_sampled_rows(bc, name, precision):
    """Full workload size, one step in the benchmarked configuration: sampled
    rows of A^(0) recomputed one by one by the oracle, plus invariants.  The
    256^3 workload keeps c in FP32 (its stored mass is checked too); its
    matrix is read row by row from the exported arrays (no sparse copy).

    The minimisation is solved to the default tolerance (as benchmarked)
    on the 1024^2 and 128^3 workloads.  On 256^3 a converged solve takes
    minutes, so there it stops after FULL_SIZE_IP_ITERS iterations and
    qp_converged is not asserted; every other invariant (bounds, exact column
    masses, exact global mass) holds at any iterate."""
    if name == "deform3d_256" and os.environ.get("BCHAR_FULL_256") != "1":
        # its 25 capped interior-point iterations alone ran past 15 minutes on one GB300
        pytest.skip("one 256^3 step takes more than 15 minutes (minimisation); set BCHAR_FULL_256=1 to run it")
    wl = inputs.workload(name)
    faces = wl.faces(0)
    c = wl.c0 if wl.c_dtype == "f32" else wl.c0.astype(np.float64)
    cap = {"qp_max_refine": FULL_SIZE_IP_ITERS} if name == "deform3d_256" else {}
    mesh, info, c_gpu = _gpu_step(bc, wl, faces, c, precision=precision, **cap)
    om = oracle.Mesh(wl.coords, wl.phi)
    rng = np.random.Generator(np.random.PCG64(99))
    rows = np.sort(rng.choice(om.nc, size=48, replace=False))
    s = oracle.substep_count(om, faces, wl.dt)
    assert info["substeps"] == s
    off, cen, rh = oracle.track_balls(om, faces, wl.dt, s, rows)
    rl, cols, vals, _ = oracle.assemble_rows(om, faces, off, cen, rh, rows)
    rp, gcol, gval = mesh.export_matrix(0)
    start = 0
    bad = 0
    for r, n in zip(rows, rl):
        want = dict(zip(cols[start:start + n], vals[start:start + n]))
        start += n
        gotd = dict(zip(gcol[rp[r]:rp[r + 1]], gval[rp[r]:rp[r + 1]]))
        keys = set(want) | set(gotd)
        mx = max(want.values())
        e = max(abs(gotd.get(k, 0.0) - want.get(k, 0.0)) for k in keys) / mx
        bad += e > 1e-4
    assert bad <= 1  # a stage point within FP32 rounding of a face may flip one row
    vp = om.volphi()
    assert np.all(np.diff(rp) > 0)  # every row carries its cell's mass
    rowsum = np.add.reduceat(gval, rp[:-1])
    # eq. ball_int: every row sums to |K|_phi (FP32 fractions: 1e-5), except the
    # rows that received seeds for empty columns, whose extra entries a_ij =
    # |M_j|_phi are the only entry of their column
    rel = np.abs(rowsum - vp) / vp
    off_rows = np.flatnonzero(rel > 1e-5)
    print(f"\n{name}: nnz {rp[-1]}, empty columns seeded {info['empty_cols']}, void balls {info['void_balls']}, "
          f"rows off the identity {off_rows.size}, max elsewhere {np.delete(rel, off_rows).max():.1e}")
    assert off_rows.size <= info["empty_cols"]
    if off_rows.size:
        colcnt = np.bincount(gcol, minlength=om.nc)
        for r in off_rows:
            cs, vs = gcol[rp[r]:rp[r + 1]], gval[rp[r]:rp[r + 1]]
            seeded = (colcnt[cs] == 1) & (vs == vp[cs])
            assert seeded.any()
            assert abs(rowsum[r] - vs[seeded].sum() - vp[r]) <= 1e-5 * vp[r]
    del gcol, gval
    print(f"{name}: interior-point iters {info['ip_iters']}, cg iters {info['cg_iters']}, constraint residual "
          f"{info['kkt_rel']:.1e}, entries at bounds {info['n_at_bounds']}, max row residual "
          f"{info['max_rel_row_res']:.2e}, minimisation {info['ms_stage']['minimise']:.0f} ms, "
          f"converged {info['qp_converged']}")
    if name != "deform3d_256":
        assert info["qp_converged"]
    assert info["n_at_bounds"] >= 0 and info["spill_rows"] >= 0
    assert abs(info["mass_after"] - info["mass_before"]) <= 1e-12 * info["mass_before"]
    assert info["max_rel_col_res"] <= 1e-13
    assert np.all(c_gpu >= 0)
    if c_gpu.dtype == np.float32:
        # one rounding per stored value: the stored mass is within 2^-24 of the FP64 one
        stored = float(np.dot(vp, c_gpu.astype(np.float64)))
        assert abs(info["mass_after_stored"] - stored) <= 1e-12 * stored
        assert abs(info["mass_after_stored"] - info["mass_after"]) <= (2.0 ** -24 + 1e-14) * info["mass_after"]
    mesh.close()


@pytest.mark.parametrize("name", ["stretched3d", "porous3d"])
def test_fp32_storage_rounds_the_fp64_update(bc, name):
    """c stored in FP32: the update reads the FP32 values, sums in FP64 and
    rounds once on store.  The result is bitwise the FP64-storage step of the
    same (promoted) input rounded to FP32; the mass certificate comes from the
    FP64 sums, and the stored mass differs from it by that rounding alone."""
    wl = _case(name)
    faces = wl.faces(2)
    c32 = wl.c0.astype(np.float32)
    m32, i32, out32 = _gpu_step(bc, wl, faces, c32)
    m64, i64, out64 = _gpu_step(bc, wl, faces, c32.astype(np.float64))
    assert out32.dtype == np.float32
    assert np.array_equal(out32, out64.astype(np.float32))
    assert i32["mass_before"] == i64["mass_before"] and i32["mass_after"] == i64["mass_after"]
    assert abs(i32["mass_after"] - i32["mass_before"]) <= 1e-12 * i32["mass_before"]
    vp = oracle.Mesh(wl.coords, wl.phi).volphi()
    stored = float(np.dot(vp, out32.astype(np.float64)))
    assert abs(i32["mass_after_stored"] - stored) <= 1e-12 * stored
    assert abs(i32["mass_after_stored"] - i32["mass_after"]) <= (2.0 ** -24 + 1e-14) * i32["mass_after"]
    assert i64["mass_after_stored"] == i64["mass_after"]
    ref = oracle.step(oracle.Mesh(wl.coords, wl.phi), faces, wl.dt, c32.astype(np.float64))
    assert np.abs(out32 - ref["c"]).sum() / np.abs(ref["c"]).sum() <= 1e-5
    m32.close()
    m64.close()


def test_step_is_bitwise_reproducible(bc):
    wl = _case("stretched2d")
    faces = wl.faces(1)
    c = wl.c0.astype(np.float64)
    m1, _, c1 = _gpu_step(bc, wl, faces, c, precision=bc.FP32_SPLIT)
    m2, _, c2 = _gpu_step(bc, wl, faces, c, precision=bc.FP32_SPLIT)
    assert np.array_equal(c1, c2)
    assert np.array_equal(m1.export_matrix(2)[2], m2.export_matrix(2)[2])
    m1.close()
    m2.close()


def test_zero_velocity_is_identity_on_gpu(bc):
    wl = _case("porous3d")
    faces = [np.zeros_like(f) for f in wl.faces(0)]
    c = np.random.Generator(np.random.PCG64(4)).uniform(size=wl.nc)
    mesh, info, c_gpu = _gpu_step(bc, wl, faces, c)
    assert info["nnz"] == wl.nc
    assert np.allclose(c_gpu, c, rtol=1e-13, atol=0)
    mesh.close()


def test_error_statuses(bc):
    import torch
    wl = _case("uniform2d")
    faces = wl.faces(0)
    mesh = bc.Mesh(wl.coords, wl.phi)
    c = torch.zeros(wl.nc, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(c)
    with pytest.raises(bc.BcharError) as e:
        mesh.step(wl.dt, c, out)
    assert e.value.name == "NO_VELOCITY"
    bad = [f.copy() for f in faces]
    bad[0][:, 0] = 0.3  # flux through the left wall
    with pytest.raises(bc.BcharError) as e:
        mesh.set_velocity(bad)
    assert e.value.name == "BOUNDARY_FLUX"
    bad = [f.copy() for f in faces]
    bad[0][5, 7] += 0.1  # a source in two cells
    with pytest.raises(bc.BcharError) as e:
        mesh.set_velocity(bad)
    assert e.value.name == "DIVERGENCE"
    bad = [f.copy() for f in faces]
    bad[1][3, 3] = np.nan
    with pytest.raises(bc.BcharError) as e:
        mesh.set_velocity(bad)
    assert e.value.name == "NONFINITE"
    mesh.set_velocity(faces)
    with pytest.raises(bc.BcharError) as e:
        mesh.step(-1.0, c, out)
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(bc.BcharError) as e:
        mesh.step(wl.dt, c, c)
    assert e.value.name == "INVALID_ARG"
    mesh.close()
    with pytest.raises(bc.BcharError) as e:
        bc.Mesh([wl.coords[0][::-1], wl.coords[1]], wl.phi)
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(bc.BcharError) as e:
        bc.Mesh(wl.coords, -wl.phi)
    assert e.value.name == "INVALID_ARG"
