"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: every expected value comes from
a different route (a quadrature, a Monte Carlo estimate, a closed special
value, the exact RK4 polynomial of a linear ODE, a brute-force search, the
paper's own A-hat example, a hand computation, an SVD least-squares solve, a
dense exact solve certified by the optimality conditions, a linear programme
(HiGHS) deciding feasibility, or an invariant the method must satisfy)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.integrate import quad
from scipy.optimize import linprog

import oracle
from paper_1908_05834_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- lens


def _lens2d_quad(d, r1, r2):
    # centres on the x axis: the intersection's vertical chord at x is the
    # shorter of the two discs' chords
    def chord(x):
        h1 = r1 * r1 - x * x
        h2 = r2 * r2 - (x - d) ** 2
        return 2.0 * math.sqrt(min(h1, h2)) if h1 > 0 and h2 > 0 else 0.0
    lo, hi = max(-r1, d - r2), min(r1, d + r2)
    return quad(chord, lo, hi, epsabs=1e-14, epsrel=1e-12, limit=200)[0] if hi > lo else 0.0


def _lens3d_quad(d, r1, r2):
    # sections perpendicular to the axis of the centres are concentric discs
    def area(x):
        h1 = r1 * r1 - x * x
        h2 = r2 * r2 - (x - d) ** 2
        return math.pi * min(h1, h2) if h1 > 0 and h2 > 0 else 0.0
    lo, hi = max(-r1, d - r2), min(r1, d + r2)
    return quad(area, lo, hi, epsabs=1e-14, epsrel=1e-12, limit=200)[0] if hi > lo else 0.0


CASES = [(0.3, 1.0, 1.0), (1.0, 1.0, 1.0), (1.5, 1.0, 0.7), (0.45, 0.5, 0.2), (1.69, 1.0, 0.7),
         (0.05, 1.0, 1.0), (0.9, 0.25, 0.75), (1.999, 1.0, 1.0)]


@pytest.mark.parametrize("d,r1,r2", CASES)
def test_lens_area_matches_chord_quadrature(d, r1, r2):
    assert oracle.lens_area(d, r1, r2) == pytest.approx(_lens2d_quad(d, r1, r2), rel=1e-9, abs=1e-13)


@pytest.mark.parametrize("d,r1,r2", CASES)
def test_lens_volume_matches_section_quadrature(d, r1, r2):
    assert oracle.lens_volume(d, r1, r2) == pytest.approx(_lens3d_quad(d, r1, r2), rel=1e-9, abs=1e-13)


def test_lens_special_values():
    r = 0.37
    # equal radii at distance r: 2D r^2 (2 pi/3 - sqrt(3)/2), 3D 5 pi r^3 / 12
    assert oracle.lens_area(r, r, r) == pytest.approx(r * r * (2 * math.pi / 3 - math.sqrt(3) / 2), rel=1e-14)
    assert oracle.lens_volume(r, r, r) == pytest.approx(5 * math.pi * r ** 3 / 12, rel=1e-14)
    # disjoint and tangent balls
    for f in (oracle.lens_area, oracle.lens_volume):
        assert f(2 * r, r, r) == 0.0
        assert f(3.0, 1.0, 1.5) == 0.0
    # one ball inside the other, and coincident balls
    assert oracle.lens_area(0.1, 1.0, 0.5) == pytest.approx(math.pi * 0.25, rel=1e-15)
    assert oracle.lens_volume(0.0, 1.0, 0.5) == pytest.approx(4 / 3 * math.pi * 0.125, rel=1e-15)
    assert oracle.lens_area(0.0, r, r) == pytest.approx(math.pi * r * r, rel=1e-15)


def test_lens_monte_carlo():
    rng = np.random.Generator(np.random.PCG64(7))
    n = 10_000_000
    for dim, f, (d, r1, r2) in [(2, oracle.lens_area, (0.8, 1.0, 0.6)), (3, oracle.lens_volume, (1.1, 1.0, 0.8))]:
        p = rng.uniform(-r1, r1, size=(n, dim))
        inside1 = np.sum(p * p, axis=1) < r1 * r1
        q = p.copy()
        q[:, 0] -= d
        inside2 = np.sum(q * q, axis=1) < r2 * r2
        frac = np.mean(inside1 & inside2)
        box = (2 * r1) ** dim
        est = frac * box
        sigma = box * math.sqrt(frac * (1 - frac) / n)
        assert abs(f(d, r1, r2) - est) < 4 * sigma


# ---------------------------------------------------------------- balls


def _stretched_mesh(n=(5, 4), seed=11, dim=2, phi_var=True):
    rng = np.random.Generator(np.random.PCG64(seed))
    coords = [inputs.stretched_coords(rng, k, 0.5, 1.5) for k in n[:dim]]
    nc = int(np.prod(n[:dim]))
    phi = inputs.log_uniform_phi(rng, nc, 0.1, 0.3) if phi_var else np.ones(nc)
    return oracle.Mesh(coords, phi)


def test_ball_packing_square_cells_has_4_and_8_balls():
    m2 = oracle.Mesh([inputs.uniform_coords(4)] * 2, np.ones(16))
    m3 = oracle.Mesh([inputs.uniform_coords(3)] * 3, np.ones(27))
    assert np.all(oracle.ball_counts(m2) == 4)
    assert np.all(oracle.ball_counts(m3) == 8)


@pytest.mark.parametrize("dim", [2, 3])
def test_balls_disjoint_inside_and_carry_the_porous_volume(dim):
    mesh = _stretched_mesh(n=(4, 3, 3), dim=dim)
    rad = mesh.radii()
    w = mesh.widths()
    rho = oracle.porous_density(mesh)
    cnt = oracle.ball_counts(mesh)
    # eq. def:porous.density: rho_K sum_s |B_{K,s}|_phi = |K|_phi
    bvol = np.pi * rad ** 2 if dim == 2 else 4 / 3 * np.pi * rad ** 3
    assert np.allclose(rho * cnt * mesh.phi * bvol, mesh.volphi(), rtol=1e-14)
    assert np.allclose(oracle.ball_masses(mesh) * cnt, mesh.volphi(), rtol=1e-14)
    n3 = mesh.n + [1] * (3 - dim)
    for k in range(mesh.nc):
        c = oracle.ball_centres(mesh, k)
        assert c.shape[0] == cnt[k]
        idx = [k % n3[0], (k // n3[0]) % n3[1], k // (n3[0] * n3[1])]
        for a in range(dim):
            lo, hi = mesh.coords[a][idx[a]], mesh.coords[a][idx[a] + 1]
            assert np.all(c[:, a] - rad[k] >= lo - 1e-15) and np.all(c[:, a] + rad[k] <= hi + 1e-15)
            # tight packing: neighbours along an axis are 2r .. 2r(nb+1)/nb apart
            steps = np.unique(np.round(np.diff(np.unique(c[:, a])), 14))
            if steps.size:
                assert steps.min() >= 2 * rad[k] * (1 - 1e-12) and steps.max() <= 3 * rad[k] * (1 + 1e-12)
        dd = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=2) + np.eye(c.shape[0]) * 1e9
        assert dd.min() >= 2 * rad[k] * (1 - 1e-12)
        assert w[k].min() / 4 == pytest.approx(rad[k], rel=1e-15)


# ---------------------------------------------------------------- tracking


def test_substep_rule():
    wl = inputs.workload("vortex2d_32")
    mesh = oracle.Mesh(wl.coords, wl.phi)
    f = wl.faces(0)
    vmax = oracle.max_speed(mesh, f)
    assert vmax == pytest.approx(max(np.abs(f[0]).max(), np.abs(f[1]).max()), rel=1e-15)
    assert oracle.substep_count(mesh, f, 0.01) == math.ceil(0.01 * vmax / (0.5 / 32))
    assert oracle.substep_count(mesh, f, 1e-9) == 1


@pytest.mark.parametrize("substeps", [1, 3, 7])
def test_rk4_on_linear_field_is_the_rk4_polynomial(substeps):
    # u = (alpha x, -alpha y) is divergence free and its RT0 interpolant is
    # exact on any tensor mesh; backward tracking solves x' = -(alpha/phi) x,
    # y' = (alpha/phi) y, for which one classical RK4 step of size h multiplies
    # by R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, z = -+ alpha h / phi.
    rng = np.random.Generator(np.random.PCG64(3))
    coords = [inputs.stretched_coords(rng, 9, 0.5, 1.5), inputs.stretched_coords(rng, 7, 0.5, 1.5)]
    phi0 = 0.7
    mesh = oracle.Mesh(coords, np.full(63, phi0))
    alpha, tau = 1.3, 0.21
    ux = np.tile(alpha * coords[0], (7, 1))
    uy = np.tile(-alpha * coords[1][:, None], (1, 9))
    p0 = np.array([[0.41, 0.52, 0.0], [0.6, 0.35, 0.0], [0.47, 0.61, 0.0]])
    cells = [oracle.locate(mesh, p) for p in p0]
    out = oracle.track_points(mesh, [ux, uy], tau, substeps, p0, cells)
    h = tau / substeps

    def R(z):
        return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    exp_x = p0[:, 0] * R(-alpha * h / phi0) ** substeps
    exp_y = p0[:, 1] * R(alpha * h / phi0) ** substeps
    assert np.allclose(out[:, 0], exp_x, rtol=1e-14, atol=0)
    assert np.allclose(out[:, 1], exp_y, rtol=1e-14, atol=0)


def test_zero_field_does_not_move_and_keeps_radii():
    mesh = _stretched_mesh(n=(4, 3, 3), dim=3)
    faces = [np.zeros(mesh.face_count(a)) for a in range(3)]
    rows = np.arange(mesh.nc)
    off, cen, rh = oracle.track_balls(mesh, faces, 0.1, 3, rows)
    for k in rows:
        assert np.array_equal(cen[off[k]:off[k + 1]], oracle.ball_centres(mesh, k))
        assert np.allclose(rh[off[k]:off[k + 1]], mesh.radii()[k], rtol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_tracked_radius_on_a_linear_field_is_the_rk4_closed_form(dim):
    """eq. rTrackedBall (and its 3D reading with six axis points): with phi not
    constant the 2 dim axis points C +- r e_a are tracked and r_hat is their
    mean distance to the tracked centre.  On the linear field u = (al x, be y,
    -(al + be) z) (exactly representable by face values, div u = 0) with
    phi = phi0 wherever the points travel and one distant cell set to 2 phi0
    (so the cardinal-point path runs), s RK4 substeps of dp/dt = -u/phi0 map
    each coordinate by the exact polynomial R(z)^s, R(z) = 1 + z + z^2/2 +
    z^3/6 + z^4/24: the tracked centre is C_a R_a^s and every axis point of
    axis a lands r |R_a^s| from it, so r_hat = r mean_a |R_a^s|.  Measuring
    from the untracked centre, or averaging another point set, gives other
    values."""
    n = (9, 8, 7)[:dim]
    coords = [np.linspace(0.0, 1.0, k + 1) for k in n]
    phi0 = 0.8
    phi = np.full(int(np.prod(n)), phi0)
    phi[-1] = 2.0 * phi0  # the far corner cell, which no tracked point reaches
    mesh = oracle.Mesh(coords, phi)
    rates = (1.1, 0.7, -1.8)[:dim] if dim == 3 else (1.3, -1.3)
    faces = []
    for a in range(dim):
        shape = [k for k in reversed(n)]
        shape[dim - 1 - a] += 1
        xa = coords[a].reshape([-1 if b == dim - 1 - a else 1 for b in range(dim)])
        faces.append(np.ascontiguousarray(np.broadcast_to(rates[a] * xa, shape)))
    dt, substeps = 0.07, 3
    h = dt / substeps

    def R(z):
        return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    amp = [R(-rates[a] * h / phi0) ** substeps for a in range(dim)]
    cell = 1 + n[0] * (1 if dim == 2 else 1 + n[1])   # an interior cell near the origin
    off, cen, rh = oracle.track_balls(mesh, faces, dt, substeps, [cell])
    c0 = oracle.ball_centres(mesh, cell)
    rad = mesh.radii()[cell]
    for s_ in range(c0.shape[0]):
        for a in range(dim):
            assert cen[s_, a] == pytest.approx(c0[s_, a] * amp[a], rel=1e-14)
        assert rh[s_] == pytest.approx(rad * np.mean(np.abs(amp)), rel=1e-14)
        assert abs(rh[s_] - rad) > 1e-3 * rad  # the field does change the radius


# ---------------------------------------------------------------- A^(0)


def _vortex(mesh, g=1.0):
    return inputs.vortex2d_faces(mesh.coords, g) if mesh.dim == 2 else inputs.deform3d_faces(mesh.coords, g)


@pytest.mark.parametrize("dim,phi_var", [(2, False), (2, True), (3, True)])
def test_row_sums_are_the_porous_volumes(dim, phi_var):
    # Sec 3.2: sum_M V_{K,M} = |F_{-dt}(K)|_phi = |K|_phi (eq. ball_int, eq. volTracked)
    mesh = _stretched_mesh(n=(7, 6, 5), dim=dim, phi_var=phi_var)
    f = _vortex(mesh)
    s = oracle.substep_count(mesh, f, 0.03)
    A0, info = oracle.initial_matrix(mesh, f, 0.03, s, drop_tol=0.0)
    rows = np.asarray(A0.sum(axis=1)).ravel()
    assert info["empty_cols"] == 0
    assert np.allclose(rows, mesh.volphi(), rtol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_zero_velocity_gives_the_diagonal(dim):
    mesh = _stretched_mesh(n=(5, 4, 3), dim=dim)
    faces = [np.zeros(mesh.face_count(a)) for a in range(dim)]
    A0, _ = oracle.initial_matrix(mesh, faces, 0.1, 1)
    assert A0.nnz == mesh.nc
    assert np.allclose(A0.diagonal(), mesh.volphi(), rtol=1e-15)


def test_whole_cell_translation_is_a_shift():
    # uniform grid, constant field carrying everything one cell in +x over dt:
    # each tracked ball lands exactly on the matching ball of the cell to the
    # left, whose neighbours it only touches (TC1 idea, Sec 4.1)
    n = 6
    mesh = oracle.Mesh([inputs.uniform_coords(n)] * 2, np.ones(n * n))
    h = 1.0 / n
    faces = [np.full((n, n + 1), h), np.zeros((n + 1, n))]
    A0, info = oracle.initial_matrix(mesh, faces, 1.0, 4)
    # nothing lands in the last column of cells (the field enters through the
    # left wall), so those n columns are seeded into their own rows
    assert info["empty_cols"] == n
    for k in range(mesh.nc):
        i = k % n
        if i == 0 or i == n - 1:
            continue
        row = A0.getrow(k)
        assert row.nnz == 1 and row.indices[0] == k - 1
        assert row.data[0] == pytest.approx(h * h, rel=1e-12)
    # the seeds (reading of the empty columns): the centre of an empty cell M_j
    # carried forward over dt leaves through the right wall and is clamped into
    # M_j itself, so row j gains a_jj = |M_j|_phi exactly, the only entry of
    # column j, on top of its own transfer to the cell on its left
    Ac = A0.tocsc()
    for j in range(n - 1, mesh.nc, n):
        col = Ac.getcol(j)
        assert col.nnz == 1 and col.indices[0] == j and col.data[0] == mesh.volphi()[j]
        row = A0.getrow(j)
        assert sorted(row.indices) == [j - 1, j]
        assert row.sum() == pytest.approx(2 * mesh.volphi()[j], rel=1e-12)


def test_initial_matrix_matches_brute_force():
    # every tracked ball against every residing ball of the mesh, eq. ball_int
    # written out directly (no candidate window)
    mesh = _stretched_mesh(n=(4, 3), dim=2, phi_var=True)
    f = _vortex(mesh)
    dt, s = 0.04, 5
    rows = np.arange(mesh.nc)
    off, cen, rh = oracle.track_balls(mesh, f, dt, s, rows)
    row_len, cols, vals, voids = oracle.assemble_rows(mesh, f, off, cen, rh, rows, drop_tol=0.0)
    got = sp.csr_matrix((vals, cols, np.concatenate([[0], np.cumsum(row_len)])), shape=(mesh.nc, mesh.nc)).toarray()
    rad = mesh.radii()
    cnt = oracle.ball_counts(mesh)
    rhophi = mesh.volphi() / (cnt * np.pi * rad ** 2)
    res = [(M, oracle.ball_centres(mesh, M)) for M in range(mesh.nc)]
    want = np.zeros((mesh.nc, mesh.nc))
    for K in range(mesh.nc):
        for b in range(off[K], off[K + 1]):
            w = np.zeros(mesh.nc)
            for M, cM in res:
                for q in cM:
                    w[M] += rhophi[M] * oracle.lens_area(float(np.linalg.norm(cen[b, :2] - q[:2])), rh[b], rad[M])
            assert w.sum() > 0
            want[K] += mesh.volphi()[K] / cnt[K] * w / w.sum()
    assert np.allclose(got, want, rtol=1e-12, atol=1e-18)


# ---------------------------------------------------------------- A-hat, scaling, minimisation


def test_hat_matrix_is_the_papers_example():
    g = json.load(open(os.path.join(GOLDEN, "hat_a_example.json")))
    A = sp.csr_matrix(np.array(g["A"], dtype=float))
    H = oracle.hat_matrix(A).toarray()
    assert np.array_equal(H, np.array(g["hat"], dtype=float))
    # A-hat 1 = (row sums; column sums)
    A = np.array(g["A"], dtype=float)
    assert np.array_equal(H.sum(axis=1), np.concatenate([A.sum(axis=1), A.sum(axis=0)]))


def test_one_scaling_iteration_by_hand():
    A0 = sp.csr_matrix(np.array([[2.0, 1.0], [1.0, 1.0]]))
    A1 = oracle.scale(A0, np.ones(2), np.ones(2), 1).toarray()
    # columns: (2,1)/3 and (1,1)/2 -> [[2/3, 1/2], [1/3, 1/2]]; rows: 7/6, 5/6
    assert np.allclose(A1, [[4 / 7, 3 / 7], [2 / 5, 3 / 5]], rtol=1e-15)


def test_scaling_leaves_rows_exact_after_every_iteration():
    mesh = _stretched_mesh(n=(6, 6), dim=2)
    f = _vortex(mesh)
    A0, _ = oracle.initial_matrix(mesh, f, 0.05, 4)
    vp = mesh.volphi()
    for n_iter in (1, 2, 5, 10):
        AN = oracle.scale(A0, vp, vp, n_iter)
        assert np.allclose(np.asarray(AN.sum(axis=1)).ravel(), vp, rtol=1e-14)


def test_minimise_is_the_min_norm_adjustment_when_feasible():
    # uniform mesh, phi = 1: the constraints are consistent and the paper's
    # minimiser lies inside the bounds; it is A-hat^+ r (SVD least squares)
    wl = inputs.workload("vortex2d_32", n=8)
    mesh = oracle.Mesh(wl.coords, wl.phi)
    f = wl.faces(0)
    A0, _ = oracle.initial_matrix(mesh, f, 0.02, oracle.substep_count(mesh, f, 0.02))
    vp = mesh.volphi()
    AN = oracle.scale(A0, vp, vp, 10)
    factor, x, info = oracle.minimise(AN, vp, vp)
    H = oracle.hat_matrix(AN).toarray()
    r = np.concatenate([vp, vp]) - H.sum(axis=1)
    ref = np.linalg.lstsq(H, r, rcond=None)[0]
    assert info["converged"] and info["n_at_bounds"] == 0
    assert np.max(np.abs(x - ref)) < 1e-8 * max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(H @ (1 + x) - np.concatenate([vp, vp]))) < 1e-10 * vp.max()


def _matrices(name, n):
    wl = inputs.workload(name, n=n)
    mesh = oracle.Mesh(wl.coords, wl.phi)
    faces = wl.faces(0)
    A0, _ = oracle.initial_matrix(mesh, faces, wl.dt, oracle.substep_count(mesh, faces, wl.dt))
    vp = mesh.volphi()
    R, _ = oracle.balanced_targets(A0, vp)
    return oracle.scale(A0, R, vp, 10), R, vp


def _lp_min_violation(AN, R, C):
    """min sum_l |s_l| / b_l over 0 <= f <= 2 with A-hat f + s = b (HiGHS): 0 iff
    the paper's problem (eq. opti_masscons with its bounds) has a solution."""
    H = oracle.hat_matrix(AN)
    nz, m = H.shape[1], H.shape[0]
    b = np.concatenate([R, C])
    A_eq = sp.hstack([H, sp.eye(m), -sp.eye(m)]).tocsr()
    cost = np.concatenate([np.zeros(nz), 1.0 / b, 1.0 / b])
    res = linprog(cost, A_eq=A_eq, b_eq=b, bounds=[(0.0, 2.0)] * nz + [(0.0, None)] * (2 * m), method="highs")
    assert res.status == 0
    return res.fun


def _certified_minimiser(AN, R, C, guess, active_tol=1e-8):
    """The paper's minimiser (hard constraints, 0 <= f <= 2), certified by the
    optimality conditions of this convex problem.  Starting from the active
    set read off the guess, the min-norm solution of the equality-constrained
    problem on the free entries is formed densely (least squares); free
    entries that leave [0, 2] join the active set and it is formed again.
    The result is the paper's minimiser iff it satisfies the constraints,
    lies inside the bounds, and some multipliers y satisfy x_F = G_F^T y on
    the free entries with (G^T y)_k <= -1 on entries at 0 and >= 1 on entries
    at 2 -- the existence of such y is decided by a linear programme
    (HiGHS).  Returns f or None."""
    b = np.concatenate([R, C])
    G = (sp.diags(1.0 / b) @ oracle.hat_matrix(AN)).toarray()
    lo, hi = guess < active_tol, guess > 2.0 - active_tol
    for _ in range(20):
        free = ~(lo | hi)
        f = np.where(hi, 2.0, 0.0)
        GF = G[:, free]
        r = 1.0 - G[:, ~free] @ f[~free] - GF.sum(axis=1)
        f[free] = 1.0 + GF.T @ np.linalg.lstsq(GF @ GF.T, r, rcond=1e-13)[0]
        out_lo, out_hi = free & (f < 0.0), free & (f > 2.0)
        if not (out_lo.any() or out_hi.any()):
            break
        lo, hi = lo | out_lo, hi | out_hi
    if np.max(np.abs(G @ f - 1.0)) > 1e-11 or f.min() < 0.0 or f.max() > 2.0:
        return None
    A_ub = np.vstack([G[:, lo].T, -G[:, hi].T])
    b_ub = -np.ones(A_ub.shape[0])
    res = linprog(np.zeros(G.shape[0]), A_ub=A_ub if A_ub.size else None, b_ub=b_ub if A_ub.size else None,
                  A_eq=GF.T, b_eq=f[free] - 1.0, bounds=[(None, None)] * G.shape[0], method="highs")
    return f if res.status == 0 else None


@pytest.mark.parametrize("name,n", [("vortex2d_1024", 7), ("vortex2d_1024", 10), ("deform3d_128", 3),
                                    ("deform3d_128", 5), ("deform3d_256", 4)])
def test_minimise_equals_the_certified_paper_minimiser_with_active_bounds(name, n):
    """Sec 3.2, eq. opti_masscons with 0 <= 1 + x <= 2 inside the problem: on
    small stretched and porous cases where bounds are active and the LP says
    the paper's problem is feasible, the oracle's penalised interior-point
    result agrees with the exactly certified minimiser up to the penalty:
    every adjusted volume a_k (1 + x_k) within 1e-7 of its row target, and
    1 + x within 2e-6 on every entry of at least 1e-2 of its row target."""
    AN, R, vp = _matrices(name, n)
    assert AN.shape[0] <= 125
    assert _lp_min_violation(AN, R, vp) < 1e-12
    f, x, info = oracle.minimise(AN, R, vp)
    assert info["converged"] and info["n_at_bounds"] > 0
    fstar = _certified_minimiser(AN, R, vp, f)
    assert fstar is not None
    rel = AN.data / np.repeat(R, np.diff(AN.indptr))
    assert np.max(np.abs(rel * (f - fstar))) < 1e-7
    assert np.max(np.abs((f - fstar)[rel >= 1e-2])) < 2e-6


@pytest.mark.parametrize("name,n,rows_tol,median_tol", [("vortex2d_1024", 45, 1e-7, 1e-11),
                                                        ("deform3d_128", 12, 1e-9, 1e-11),
                                                        ("deform3d_256", 8, 1e-7, 1e-9)])
def test_feasible_cases_meet_the_mass_constraints(name, n, rows_tol, median_tol):
    """Where the LP says the paper's problem is feasible, the oracle's
    adjustment meets every row and column constraint up to the penalty's
    residual eps^2 y_l (relative): <= 1e-9 on the porous case, and <= 1e-7
    where an entry of ~1e-7 of its row target must reach a bound (the 2D
    and 3D stretched cases); the median row far below either."""
    AN, R, vp = _matrices(name, n)
    assert _lp_min_violation(AN, R, vp) < 1e-12
    f, x, info = oracle.minimise(AN, R, vp)
    assert info["converged"]
    assert f.min() >= 0.0 and f.max() <= 2.0
    Aq = AN.copy()
    Aq.data = AN.data * f
    rows = np.abs(np.asarray(Aq.sum(axis=1)).ravel() - R) / R
    cols = np.abs(np.asarray(Aq.sum(axis=0)).ravel() - vp) / vp
    assert rows.max() < rows_tol and cols.max() < rows_tol
    assert np.median(rows) < median_tol


def test_penalty_residuals_follow_the_multipliers():
    """Optimality of the elastic penalty (quadratic up to a relative
    violation delta = 1e-6, linear beyond): every constraint's relative
    violation v_l = s_l / b_l is eps^2 y_l where |v_l| < delta, and its
    multiplier sits at the linear slope gamma = delta / eps^2 where
    |v_l| > delta; on a feasible and on an infeasible case."""
    eps, delta = 1e-7, 1e-6
    gamma = delta / eps ** 2
    for name, n in (("deform3d_128", 8), ("deform3d_256", 9)):
        AN, R, vp = _matrices(name, n)
        f, x, info = oracle.minimise(AN, R, vp)
        b = np.concatenate([R, vp])
        v = (b - oracle.hat_matrix(AN) @ f) / b
        assert np.max(np.abs(v - info["violation"])) < 1e-12
        ys = info["y"] * b
        inner = np.abs(v) < 0.999 * delta
        assert np.max(np.abs(v[inner] - eps ** 2 * ys[inner])) < 1e-12
        outer = np.abs(v) > 1.001 * delta
        assert np.all(np.abs(np.abs(ys[outer]) - gamma) <= 1e-6 * gamma)
        assert np.all(np.sign(ys[outer]) == np.sign(v[outer]))


def test_lp_shows_an_infeasible_case_and_the_reading_holds():
    """The stretched 3D recipe at 9^3 after N = 10 scalings: the LP proves
    that no adjustment within 0 <= 1 + x <= 2 meets all 2 n_c constraints
    (the doubling cap is what fails).  The reading then keeps the bounds
    exactly, its total relative violation equals the LP's minimum, and the
    step still conserves global mass to 1e-12 (final column scaling)."""
    AN, R, vp = _matrices("deform3d_256", 9)
    lp_min = _lp_min_violation(AN, R, vp)
    assert lp_min > 1e-3
    f, x, info = oracle.minimise(AN, R, vp)
    assert info["converged"]
    assert f.min() >= 0.0 and f.max() <= 2.0
    # the linear part of the penalty makes the total relative violation the
    # LP's minimum, up to the quadratic zone (delta = 1e-6 per constraint)
    total = float(np.sum(np.abs(info["violation"])))
    assert lp_min - 1e-9 <= total <= lp_min + 1e-6 * info["violation"].size
    wl = inputs.workload("deform3d_256", n=9)
    mesh = oracle.Mesh(wl.coords, wl.phi)
    r = oracle.step(mesh, wl.faces(0), wl.dt, np.asarray(wl.c0, dtype=np.float64))
    assert r["max_rel_col_res"] < 1e-13
    assert abs(r["mass_after"] - r["mass_before"]) <= 1e-12 * r["mass_before"]
    assert 1e-3 < r["max_rel_row_res"] < 0.2


# ---------------------------------------------------------------- whole step


def test_step_keeps_a_constant_and_conserves_mass():
    wl = inputs.workload("vortex2d_32", n=16)
    mesh = oracle.Mesh(wl.coords, wl.phi)
    r = oracle.step(mesh, wl.faces(0), wl.dt, np.ones(mesh.nc))
    assert np.max(np.abs(r["c"] - 1.0)) < 1e-8
    assert abs(r["mass_after"] - r["mass_before"]) <= 1e-12 * r["mass_before"]


@pytest.mark.parametrize("name,n", [("vortex2d_1024", 24), ("deform3d_128", 6), ("deform3d_256", 6)])
def test_step_conserves_mass_on_stretched_and_porous_meshes(name, n):
    wl = inputs.workload(name, n=n)
    mesh = oracle.Mesh(wl.coords, wl.phi)
    c = np.asarray(wl.c0, dtype=np.float64)
    for st in range(2):
        r = oracle.step(mesh, wl.faces(st), wl.dt, c)
        assert abs(r["mass_after"] - r["mass_before"]) <= 1e-12 * r["mass_before"]
        assert np.all(r["c"] >= 0.0)
        c = r["c"]


def test_zero_velocity_step_is_the_identity():
    mesh = _stretched_mesh(n=(5, 4, 3), dim=3)
    faces = [np.zeros(mesh.face_count(a)) for a in range(3)]
    c = np.random.Generator(np.random.PCG64(5)).uniform(size=mesh.nc)
    r = oracle.step(mesh, faces, 0.1, c)
    assert np.allclose(r["c"], c, rtol=1e-13, atol=0)


def test_balanced_targets_by_hand():
    # rows {0 -> col 1}, {1 -> col 0}, {2 -> col 2} with |K|_phi = (1, 2, 3): the first
    # two components have rows summing to 1 and 2 but columns to 2 and 1
    A0 = sp.csr_matrix(np.array([[0.0, 1.0, 0.0], [2.0, 0.0, 0.0], [0.0, 0.0, 3.0]]))
    b, n_unbal = oracle.balanced_targets(A0, np.array([1.0, 2.0, 3.0]))
    assert n_unbal == 2
    assert np.array_equal(b, [2.0, 1.0, 3.0])
    # one connected block: nothing changes, bit for bit
    A1 = sp.csr_matrix(np.array([[0.6, 0.4], [0.4, 0.6]]))
    b1, n1 = oracle.balanced_targets(A1, np.array([0.3, 0.7]))
    assert n1 == 0 and np.array_equal(b1, [0.3, 0.7])
    # a sliver entry of 1e-9 joins the first two blocks into one component whose
    # rows and columns both sum to 3: every non-zero links, so nothing is rescaled
    A2 = sp.csr_matrix(np.array([[1e-9, 1.0, 0.0], [2.0, 0.0, 0.0], [0.0, 0.0, 3.0]]))
    b2, n2 = oracle.balanced_targets(A2, np.array([1.0, 2.0, 3.0]))
    assert n2 == 0 and np.array_equal(b2, [1.0, 2.0, 3.0])


def test_column_fix_by_hand():
    """The column fix (reading of eq. volAdj's first half after the bounds):
    every column is scaled to its global target; a column whose entries were
    all clipped to zero takes its A^(N) entries before that scaling."""
    AN = sp.csr_matrix(np.array([[0.5, 0.2, 0.0],
                                 [0.1, 0.3, 0.4],
                                 [0.0, 0.1, 0.6]]))
    Aq = AN.copy()
    Aq.data = AN.data * np.array([1.2, 0.0, 0.9, 0.0, 0.8, 0.0, 1.1])  # column 1 fully clipped
    Aq.data[Aq.data == 0.0] = 0.0
    target = np.array([0.7, 0.9, 1.3])
    A = oracle.column_fix(Aq, AN, target).toarray()
    # column 0: (0.6, 0.09) scaled to 0.7; column 1: A^(N) (0.2, 0.3, 0.1) scaled to 0.9;
    # column 2: (0.32, 0.66) scaled to 1.3
    exp = np.zeros((3, 3))
    exp[:, 0] = np.array([0.6, 0.09, 0.0]) * (0.7 / 0.69)
    exp[:, 1] = np.array([0.2, 0.3, 0.1]) * (0.9 / 0.6)
    exp[:, 2] = np.array([0.0, 0.32, 0.66]) * (1.3 / 0.98)
    assert np.allclose(A, exp, rtol=1e-14, atol=0)
    assert np.allclose(A.sum(axis=0), target, rtol=1e-14)
