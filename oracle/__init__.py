"""FP64 CPU oracle of one B-char time step (Cheng & Droniou, arXiv 1908.05834).

TEST INFRASTRUCTURE ONLY.  This package is the independent reference the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the CUDA library and its
Python binding never do, and the two share no code.

Every function follows one passage of the paper, cited in its docstring, in
the paper's order and notation, in double precision:

* ball packing, porous density (Sec 3, eq. def:porous.density)
* tracking the ball centres along the flow (Sec 2 eq. charac; Sec 3)
* tracked radius (Sec 3, eq. ball_volChange / eq. rTrackedBall)
* initial weights V_{K,M}                   (Sec 3.1, eq. fracMaterial, eq. ball_int)
* consistent local targets per component    (Sec 3.2, eq. localmassconsMat / globalmassconsMat)
* alternating column/row scaling, N times   (Sec 3.2, eq. volAdj)
* the matrix A-hat and the bound-constrained
  minimisation, 0 <= 1 + x <= 2 inside it   (Sec 3.2, eq. opti_masscons)
* a final column scaling                    (Sec 3.2, first half of eq. volAdj)
* the update |K|_phi c_K^{n+1} = sum_M a_KM c_M^n (Sec 2, eq. phys-inter-ELLAM)

The per-ball loops (tracking, intersections) are plain C in
``bchar_oracle.c``; the matrix steps use numpy / scipy.sparse, with a sparse
direct solve (SuperLU) as the linear-algebra primitive of every interior-point
iteration of the minimisation.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph
import scipy.sparse.linalg as spla

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bchar_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile ``bchar_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc, no
    fast-math, no FMA contraction, so x86 and Arm round alike)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _OrcMesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nb", ctypes.c_int), ("n", ctypes.c_int64 * 3),
                ("x", ctypes.c_void_p * 3), ("phi", ctypes.c_void_p), ("u", ctypes.c_void_p * 3)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        M = ctypes.POINTER(_OrcMesh)
        lib.orc_lens_area.argtypes = [D, D, D]
        lib.orc_lens_area.restype = D
        lib.orc_lens_volume.argtypes = [D, D, D]
        lib.orc_lens_volume.restype = D
        lib.orc_rk4_many.argtypes = [M, D, D, ctypes.c_int, I64, P, P, P]
        lib.orc_rk4_many.restype = None
        lib.orc_track_balls.argtypes = [M, D, ctypes.c_int, ctypes.c_int, I64, P, P, P, P]
        lib.orc_track_balls.restype = None
        lib.orc_assemble_rows.argtypes = [M, I64, P, P, P, P, D, I64, P, P, P, P]
        lib.orc_assemble_rows.restype = I64
        lib.orc_ball_totals.argtypes = [M, I64, P, P]
        lib.orc_ball_totals.restype = None
        lib.orc_locate.argtypes = [M, P]
        lib.orc_locate.restype = I64
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def lens_area(d: float, r1: float, r2: float) -> float:
    """Area of the intersection of two discs (the 2D ball intersection of Sec 3)."""
    return _load().orc_lens_area(d, r1, r2)


def lens_volume(d: float, r1: float, r2: float) -> float:
    """Volume of the intersection of two balls (the 3D ball intersection of Sec 3)."""
    return _load().orc_lens_volume(d, r1, r2)


# ---------------------------------------------------------------- mesh


@dataclass
class Mesh:
    """Tensor-product mesh of a box (Sec 1.2): node coordinates per axis,
    piecewise-constant porosity per cell (x index fastest) and the ball packing
    parameter nb (Sec 3; nb = 2 gives the 4 balls per cell in 2D and 8 in 3D of
    Sec 4 on square cells; stretched cells hold more balls along their long
    axes, see ``ball_counts``)."""

    coords: list
    phi: np.ndarray
    nb: int = 2
    _keep: list = field(default_factory=list, repr=False)

    def __post_init__(self):
        self.coords = [np.ascontiguousarray(c, dtype=np.float64) for c in self.coords]
        self.dim = len(self.coords)
        assert self.dim in (2, 3)
        self.n = [len(c) - 1 for c in self.coords]
        self.nc = int(np.prod(self.n))
        self.phi = np.ascontiguousarray(self.phi, dtype=np.float64).reshape(-1)
        assert self.phi.size == self.nc
        assert all(np.all(np.diff(c) > 0) for c in self.coords)
        assert np.all(self.phi > 0)

    # cell-wise quantities, x fastest
    def widths(self):
        """Per-cell widths, shape (nc, dim)."""
        w = [np.diff(c) for c in self.coords]
        grids = np.meshgrid(*w, indexing="ij")  # axis order (x, y, z)
        return np.stack([g.transpose(*reversed(range(self.dim))).reshape(-1) for g in grids], axis=1)

    def volumes(self):
        """|K|."""
        return np.prod(self.widths(), axis=1)

    def volphi(self):
        """|K|_phi = phi_K |K| (Sec 2, porous volume)."""
        return self.phi * self.volumes()

    def radii(self):
        """Ball radius per cell: min width / (2 nb)."""
        return self.widths().min(axis=1) / (2.0 * self.nb)

    def phi_const(self) -> bool:
        """'phi constant in Omega' (Sec 3): exact equality of every phi_K."""
        return bool(np.all(self.phi == self.phi[0]))

    def c_struct(self, faces=None) -> _OrcMesh:
        s = _OrcMesh()
        s.dim = self.dim
        s.nb = self.nb
        n3 = list(self.n) + [1] * (3 - self.dim)
        for a in range(3):
            s.n[a] = n3[a]
        self._keep = [self.coords, self.phi]
        for a in range(self.dim):
            s.x[a] = _ptr(self.coords[a])
        s.phi = _ptr(self.phi)
        if faces is not None:
            f = [np.ascontiguousarray(v, dtype=np.float64).reshape(-1) for v in faces]
            for a in range(self.dim):
                assert f[a].size == self.face_count(a)
                s.u[a] = _ptr(f[a])
            self._keep.append(f)
        return s

    def face_count(self, a: int) -> int:
        n = list(self.n)
        n[a] += 1
        return int(np.prod(n))


def ball_counts(mesh: Mesh, cells=None) -> np.ndarray:
    """n_K, the number of balls of each listed cell (all cells by default):
    the product over the axes of max(nb, floor(nb w_a / w_min))."""
    cells = np.arange(mesh.nc, dtype=np.int64) if cells is None else np.asarray(cells, dtype=np.int64)
    cells = np.ascontiguousarray(cells.reshape(-1))
    out = np.zeros(cells.size, dtype=np.int64)
    ms = mesh.c_struct()
    _load().orc_ball_totals(ctypes.byref(ms), cells.size, _ptr(cells), _ptr(out))
    return out


def ball_masses(mesh: Mesh) -> np.ndarray:
    """Equivalent porous volume of one ball of each cell, rho_K |B_{K,s}|_phi =
    |K|_phi / n_K (eq. def:porous.density with equal balls)."""
    return mesh.volphi() / ball_counts(mesh)


def porous_density(mesh: Mesh) -> np.ndarray:
    """rho_K with rho_K sum_s |B_{K,s}|_phi = |K|_phi (eq. def:porous.density)."""
    r = mesh.radii()
    bvol = np.pi * r ** 2 if mesh.dim == 2 else 4.0 / 3.0 * np.pi * r ** 3
    return mesh.volphi() / (ball_counts(mesh) * mesh.phi * bvol)


def ball_centres(mesh: Mesh, cell: int) -> np.ndarray:
    """Centres of the balls of one cell, shape (n_K, 3): the centres of an equal
    split of the cell into n_x x n_y (x n_z) blocks, x fastest."""
    n = mesh.n + [1] * (3 - mesh.dim)
    cc = [cell % n[0], (cell // n[0]) % n[1], cell // (n[0] * n[1])]
    w = [mesh.coords[a][cc[a] + 1] - mesh.coords[a][cc[a]] for a in range(mesh.dim)]
    cnt = [max(mesh.nb, int(math.floor(mesh.nb * w[a] / min(w) + 1e-9))) for a in range(mesh.dim)] + [1] * (3 - mesh.dim)
    out = np.zeros((cnt[0] * cnt[1] * cnt[2], 3))
    for s in range(out.shape[0]):
        sub = [s % cnt[0], (s // cnt[0]) % cnt[1], s // (cnt[0] * cnt[1])]
        for a in range(mesh.dim):
            out[s, a] = mesh.coords[a][cc[a]] + (sub[a] + 0.5) * w[a] / cnt[a]
    return out


# ---------------------------------------------------------------- tracking


def max_speed(mesh: Mesh, faces) -> float:
    """max over cells of the largest |face velocity| of the cell divided by phi_K."""
    best = np.zeros(mesh.nc)
    shape = list(reversed(mesh.n))
    for a in range(mesh.dim):
        fshape = list(shape)
        fshape[mesh.dim - 1 - a] += 1
        f = np.abs(np.asarray(faces[a], dtype=np.float64).reshape(fshape))
        sl_lo = [slice(None)] * mesh.dim
        sl_hi = [slice(None)] * mesh.dim
        sl_lo[mesh.dim - 1 - a] = slice(0, -1)
        sl_hi[mesh.dim - 1 - a] = slice(1, None)
        best = np.maximum(best, np.maximum(f[tuple(sl_lo)], f[tuple(sl_hi)]).reshape(-1))
    return float(np.max(best / mesh.phi))


def substep_count(mesh: Mesh, faces, dt: float, cfl: float = 0.5) -> int:
    """Number of RK4 substeps: the smallest s with dt*vmax/s <= cfl*hmin (the
    paper does not fix the integrator; this is the stated reading)."""
    vmax = max_speed(mesh, faces)
    hmin = min(float(np.min(np.diff(c))) for c in mesh.coords)
    return max(1, int(math.ceil(dt * vmax / (cfl * hmin))))


def track_points(mesh: Mesh, faces, tau: float, substeps: int, points, start_cells, sign: float = -1.0):
    """RK4 solution of dp/dt = sign*u(p)/phi(p) over a span tau (eq. charac);
    sign=-1 gives F_{-tau}(p)."""
    lib = _load()
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
    cells = np.ascontiguousarray(np.asarray(start_cells, dtype=np.int64).reshape(-1))
    out = np.zeros_like(pts)
    ms = mesh.c_struct(faces)
    lib.orc_rk4_many(ctypes.byref(ms), sign, tau, substeps, pts.shape[0], _ptr(pts), _ptr(cells), _ptr(out))
    return out


def track_balls(mesh: Mesh, faces, dt: float, substeps: int, rows):
    """Tracked centres C_hat (eq. charac back over dt) and tracked radii r_hat
    (eq. ball_volChange if phi is constant, else eq. rTrackedBall) of every
    ball of the listed cells.  Returns (offset, centres, rhat): the balls of
    listed row r are offset[r] .. offset[r+1]-1, centres has shape (nballs, 3)."""
    lib = _load()
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64).reshape(-1))
    offset = np.concatenate([[0], np.cumsum(ball_counts(mesh, rows))]).astype(np.int64)
    centres = np.zeros((int(offset[-1]), 3))
    rhat = np.zeros(int(offset[-1]))
    ms = mesh.c_struct(faces)
    lib.orc_track_balls(ctypes.byref(ms), dt, substeps, int(mesh.phi_const()), rows.size, _ptr(rows),
                        _ptr(offset), _ptr(centres), _ptr(rhat))
    return offset, centres, rhat


def locate(mesh: Mesh, p) -> int:
    """Index of the cell containing p (last node <= p per axis, clamped)."""
    q = np.zeros(3)
    q[: mesh.dim] = np.asarray(p, dtype=np.float64)[: mesh.dim]
    ms = mesh.c_struct()
    return int(_load().orc_locate(ctypes.byref(ms), _ptr(q)))


# ---------------------------------------------------------------- A^(0)


def assemble_rows(mesh: Mesh, faces, offset, centres, rhat, rows, drop_tol: float = 1e-12):
    """Rows of A^(0), a_ij^(0) = V_{K_i, M_j} (eq. ball_int), for the listed
    cells from their tracked balls (as returned by ``track_balls``).
    Returns (row_len, cols, vals, voids)."""
    lib = _load()
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64).reshape(-1))
    offset = np.ascontiguousarray(offset, dtype=np.int64)
    centres = np.ascontiguousarray(centres, dtype=np.float64)
    rhat = np.ascontiguousarray(rhat, dtype=np.float64)
    cap = max(1024, rows.size * 64)
    while True:
        cols = np.zeros(cap, dtype=np.int64)
        vals = np.zeros(cap)
        row_len = np.zeros(rows.size, dtype=np.int64)
        voids = np.zeros(1, dtype=np.int64)
        ms = mesh.c_struct(faces)
        n = lib.orc_assemble_rows(ctypes.byref(ms), rows.size, _ptr(rows), _ptr(offset), _ptr(centres), _ptr(rhat),
                                  drop_tol, cap, _ptr(cols), _ptr(vals), _ptr(row_len), _ptr(voids))
        if n >= 0:
            return row_len, cols[:n], vals[:n], int(voids[0])
        cap *= 4


def cell_centres(mesh: Mesh, cells) -> np.ndarray:
    cells = np.asarray(cells, dtype=np.int64)
    n = mesh.n + [1] * (3 - mesh.dim)
    cc = [cells % n[0], (cells // n[0]) % n[1], cells // (n[0] * n[1])]
    out = np.zeros((cells.size, 3))
    for a in range(mesh.dim):
        x = mesh.coords[a]
        out[:, a] = 0.5 * (x[cc[a]] + x[cc[a] + 1])
    return out


def seed_empty_columns(mesh: Mesh, faces, dt: float, substeps: int, A0: sp.csr_matrix):
    """Reading for Sec 3.2's assumption sum_i a_ij^(0) > 0: a residing cell M_j
    that no tracked ball reaches sends its whole porous volume to the cell that
    contains its centre carried forward over dt (F_{+dt}).  Returns the new
    matrix and the number of seeded columns."""
    colsum = np.asarray(A0.sum(axis=0)).reshape(-1)
    empty = np.flatnonzero(colsum == 0.0)
    if empty.size == 0:
        return A0, 0
    fwd = track_points(mesh, faces, dt, substeps, cell_centres(mesh, empty), empty, sign=+1.0)
    dest = np.array([locate(mesh, p) for p in fwd], dtype=np.int64)
    seeds = sp.csr_matrix((mesh.volphi()[empty], (dest, empty)), shape=A0.shape)
    A = (A0 + seeds).tocsr()
    A.sort_indices()
    return A, int(empty.size)


def initial_matrix(mesh: Mesh, faces, dt: float, substeps: int, drop_tol: float = 1e-12):
    """A^(0) of Algorithm 1 for every cell (rows = tracked cells K_i, columns =
    residing cells M_j), with empty columns seeded.  Returns (A0, info)."""
    rows = np.arange(mesh.nc, dtype=np.int64)
    offset, centres, rhat = track_balls(mesh, faces, dt, substeps, rows)
    row_len, cols, vals, voids = assemble_rows(mesh, faces, offset, centres, rhat, rows, drop_tol)
    indptr = np.concatenate([[0], np.cumsum(row_len)])
    A0 = sp.csr_matrix((vals, cols, indptr), shape=(mesh.nc, mesh.nc))
    A0, n_empty = seed_empty_columns(mesh, faces, dt, substeps, A0)
    return A0, {"void_balls": voids, "empty_cols": n_empty, "ball_offset": offset, "centres": centres, "rhat": rhat}


def balanced_targets(A0: sp.csr_matrix, volphi: np.ndarray, tol: float = 1e-12):
    """Local targets made consistent with the global ones (reading).

    eq. localmassconsMat and eq. globalmassconsMat can hold together only if,
    on every connected component of the pattern of A (row i linked to column
    j whenever a_ij != 0), the sum of |K_i|_phi over its rows equals the sum of
    |M_j|_phi over its columns: both sums equal the sum of the component's
    entries once the constraints hold.  Where a component breaks this by more
    than tol (relative), its row targets are multiplied by sum_cols / sum_rows,
    so global mass conservation stays exact and local conservation is relaxed
    by that factor on that component only.  Returns (b_loc, number of rescaled
    components)."""
    n = A0.shape[0]
    rows = np.repeat(np.arange(n), np.diff(A0.indptr))
    nz = A0.data != 0.0
    G = sp.csr_matrix((np.ones(int(nz.sum())), (rows[nz], A0.indices[nz] + n)), shape=(2 * n, 2 * n))
    ncomp, labels = csgraph.connected_components(G, directed=False)
    sum_rows = np.zeros(ncomp)
    sum_cols = np.zeros(ncomp)
    for lab, grp in _groups(labels[:n]):
        sum_rows[lab] = math.fsum(volphi[grp].tolist())
    for lab, grp in _groups(labels[n:]):
        sum_cols[lab] = math.fsum(volphi[grp].tolist())
    bad = np.abs(sum_cols - sum_rows) > tol * sum_rows
    factor = np.where(bad, sum_cols / np.where(sum_rows > 0, sum_rows, 1.0), 1.0)
    return volphi * factor[labels[:n]], int(np.sum(bad))


def _groups(labels: np.ndarray):
    order = np.argsort(labels, kind="stable")
    cuts = np.flatnonzero(np.diff(labels[order])) + 1
    for grp in np.split(order, cuts):
        if grp.size:
            yield int(labels[grp[0]]), grp


# ---------------------------------------------------------------- scaling


def scale(A0: sp.csr_matrix, row_target, col_target, n_iter: int = 10):
    """N iterations of eq. volAdj: first every column is scaled to its global
    target |M_j|_phi, then every row to its local target
    |F_{-dt}(K_i)|_phi = |K_i|_phi (eq. exactVol_traceback).  Returns A^(N)."""
    A = A0.tocsr(copy=True)
    for _ in range(n_iter):
        colsum = np.asarray(A.sum(axis=0)).reshape(-1)
        A = (A @ sp.diags(col_target / colsum)).tocsr()  # a^{(n+1/2)}
        rowsum = np.asarray(A.sum(axis=1)).reshape(-1)
        A = (sp.diags(row_target / rowsum) @ A).tocsr()  # a^{(n+1)}
    A.sort_indices()
    return A


# ---------------------------------------------------------------- minimisation


def hat_matrix(AN: sp.csr_matrix) -> sp.csr_matrix:
    """The 2 n_c x n_z matrix A-hat of Sec 3.2: its first n_c rows hold the
    non-zero entries of each row of A^(N), staggered one row after another;
    row n_c + m holds, in the same columns, the entries of column m of A^(N).
    Unknown k is the k-th non-zero of A^(N) in row-major order."""
    AN = AN.tocsr()
    AN.sort_indices()
    n = AN.shape[0]
    nz = AN.nnz
    rows_of_k = np.repeat(np.arange(n), np.diff(AN.indptr))
    k = np.arange(nz)
    top = sp.csr_matrix((AN.data, (rows_of_k, k)), shape=(n, nz))
    bottom = sp.csr_matrix((AN.data, (AN.indices, k)), shape=(AN.shape[1], nz))
    return sp.vstack([top, bottom]).tocsr()


def minimise(AN: sp.csr_matrix, row_target, col_target, tol: float = 1e-12, penalty: float = 1e-7,
             linear_from: float = 1e-6, max_iter: int = 200):
    """The mass-conservation minimisation of Sec 3.2 (eq. opti_masscons), with
    the paper's bounds 0 <= 1 + x <= 2 enforced inside it.

    The paper minimises x.x over x in R^{n_z} subject to A-hat (1 + x) = b
    (row sums |K_i|_phi, eq. localmassconsMat; column sums |M_j|_phi,
    eq. globalmassconsMat) and the bounds.  On stretched and porous meshes the
    balls can make these constraints contradictory (a cell whose only tracked
    overlap is a smaller neighbour must send it more than it holds), so the
    reading used throughout keeps the bounds hard (closed: the open bound
    0 < 1 + x has no minimiser) and enforces the 2 n_c mass constraints by an
    elastic penalty on their relative violations v_l = s_l / b_l,
    s = b - A-hat (1 + x):

        minimise  1/2 x.x + sum_l h(v_l)   over 0 <= 1 + x <= 2,
        h(v) = v^2 / (2 eps^2)                      for |v| <= delta,
             = (delta |v| - delta^2 / 2) / eps^2    beyond,

    eps = penalty, delta = linear_from.  The minimiser is unique.  Where the
    paper's problem has a solution whose multipliers stay below delta / eps^2
    (1e8), this is that solution up to residuals v_l = eps^2 y_l <= delta; where
    the constraints cannot all hold, the penalty grows linearly, so the total
    relative violation is (up to O(delta)) the least the bounds allow -- the
    linear programme's minimum -- and the multipliers stay bounded.

    Solved by a primal-dual interior-point method (Mehrotra's predictor-
    corrector), written out for this problem with f = 1 + x, the constraints
    divided by their targets (G = diag(b)^-1 A-hat, every target 1), the
    violation split as v = eps^2 y + p - q (p, q >= 0 the parts beyond the
    quadratic zone, priced at gamma = delta / eps^2) and the upper bound
    carried by its own slack u = 2 - f (f near 2 would lose u to rounding):
        stationarity  f - 1 - G^T y - zeta_lo + zeta_hi = 0,
                      gamma - y - zeta_p = 0,  gamma + y - zeta_q = 0
        constraints   G f + eps^2 y + p - q = 1
        bounds        f, u, p, q and their multipliers >= 0, products -> mu.
    Every iteration solves the normal equations
    (G D G^T + diag(eps^2 + D_p + D_q)) dy = r, D = 1 / (1 + zeta_lo / f +
    zeta_hi / u), D_p = p / zeta_p, D_q = q / zeta_q, twice (predictor and
    corrector) with one sparse factorisation (SuperLU, the linear-algebra
    primitive), and steps 0.99 of the way to the boundary.  It stops when the
    constraint residual is <= tol, mu <= 1e-14, and the stationarity
    residuals are <= 1e-12 of the largest dual value (resp. of gamma), the
    rounding those carry.

    Returns (f = 1 + x in [0, 2], x, info); info has the iteration count, the
    final constraint residual, converged, the number of entries within 1e-9
    of a bound, the violations v and the dual y of the unscaled constraints."""
    H = hat_matrix(AN)
    b = np.concatenate([row_target, col_target])
    G = (sp.diags(1.0 / b) @ H).tocsr()
    GT = G.T.tocsr()
    m, nz = G.shape
    w = penalty * penalty
    gamma = linear_from / w
    f, u, zlo, zhi = np.ones(nz), np.ones(nz), np.ones(nz), np.ones(nz)
    p, q, zp, zq = np.ones(m), np.ones(m), np.ones(m), np.ones(m)
    y = np.zeros(m)
    one = np.ones(m)
    converged = False
    it = 0
    rp = one.copy()
    n_pairs = 2 * nz + 2 * m

    def to_boundary(pairs):
        a = 1.0
        for v, dv in pairs:
            neg = dv < 0.0
            if neg.any():
                a = min(a, float(np.min(-v[neg] / dv[neg])))
        return a

    for it in range(max_iter + 1):
        rd = (f - 1.0) - GT @ y - zlo + zhi
        rdp = gamma - y - zp
        rdq = gamma + y - zq
        rp = one - G @ f - w * y - p + q
        ru = 2.0 - f - u
        mu = float(f @ zlo + u @ zhi + p @ zp + q @ zq) / n_pairs
        dual_scale = 1.0 + max(float(np.max(np.abs(y))), float(zlo.max()), float(zhi.max()))
        if (np.max(np.abs(rp)) <= tol and mu <= 1e-14 and np.max(np.abs(rd)) <= 1e-12 * dual_scale
                and max(float(np.max(np.abs(rdp))), float(np.max(np.abs(rdq)))) <= 1e-12 * (1.0 + gamma)):
            converged = True
            break
        if it == max_iter:
            break
        D = 1.0 / (1.0 + zlo / f + zhi / u)
        Dp, Dq = p / zp, q / zq
        lu = spla.splu((G @ sp.diags(D) @ GT + sp.diags(w + Dp + Dq)).tocsc(), permc_spec="COLAMD")

        def direction(c_lo, c_hi, c_p, c_q):
            # linearised complementarity: zeta df + f dzeta = c per pair (du = ru - df for the upper one)
            qf = -rd + c_lo / f - c_hi / u + (zhi / u) * ru
            sp_ = -rdp + c_p / p       # dp = Dp (sp_ + dy)
            sq_ = -rdq + c_q / q       # dq = Dq (sq_ - dy)
            dy = lu.solve(rp - G @ (D * qf) - Dp * sp_ + Dq * sq_)
            df = D * (qf + GT @ dy)
            du = ru - df
            dp, dq = Dp * (sp_ + dy), Dq * (sq_ - dy)
            return (df, du, dp, dq, dy, (c_lo - zlo * df) / f, (c_hi - zhi * du) / u, (c_p - zp * dp) / p,
                    (c_q - zq * dq) / q)

        df, du, dp, dq, dy, dzlo, dzhi, dzp, dzq = direction(-f * zlo, -u * zhi, -p * zp, -q * zq)  # predictor
        ap = to_boundary([(f, df), (u, du), (p, dp), (q, dq)])
        ad = to_boundary([(zlo, dzlo), (zhi, dzhi), (zp, dzp), (zq, dzq)])
        mu_aff = float((f + ap * df) @ (zlo + ad * dzlo) + (u + ap * du) @ (zhi + ad * dzhi)
                       + (p + ap * dp) @ (zp + ad * dzp) + (q + ap * dq) @ (zq + ad * dzq)) / n_pairs
        sm = min(1.0, (mu_aff / mu) ** 3) * mu
        df, du, dp, dq, dy, dzlo, dzhi, dzp, dzq = direction(sm - f * zlo - df * dzlo, sm - u * zhi - du * dzhi,
                                                              sm - p * zp - dp * dzp, sm - q * zq - dq * dzq)
        ap = 0.99 * to_boundary([(f, df), (u, du), (p, dp), (q, dq)])
        ad = 0.99 * to_boundary([(zlo, dzlo), (zhi, dzhi), (zp, dzp), (zq, dzq)])
        f, u, p, q = f + ap * df, u + ap * du, p + ap * dp, q + ap * dq
        y, zlo, zhi, zp, zq = y + ad * dy, zlo + ad * dzlo, zhi + ad * dzhi, zp + ad * dzp, zq + ad * dzq
    f = np.clip(f, 0.0, 2.0)
    info = {"iterations": it, "kkt_l1": float(np.max(np.abs(rp))), "converged": converged,
            "n_at_bounds": int(np.sum((f < 1e-9) | (f > 2.0 - 1e-9))), "y": y / b,
            "violation": w * y + p - q}
    return f, f - 1.0, info


def column_fix(Aq: sp.csr_matrix, AN: sp.csr_matrix, col_target) -> sp.csr_matrix:
    """Scale every column to its global target |M_j|_phi (the first half of
    eq. volAdj), so that eq. globalmassconsMat holds to rounding after the
    minimisation.  A column whose entries were all clipped to zero keeps its
    A^(N) entries (no scaling could restore it otherwise)."""
    colsum = np.asarray(Aq.sum(axis=0)).reshape(-1)
    dead = colsum == 0.0
    A = Aq.copy()
    if dead.any():
        A = A.tocsc()
        ANc = AN.tocsc()
        for j in np.flatnonzero(dead):
            A.data[A.indptr[j]:A.indptr[j + 1]] = ANc.data[ANc.indptr[j]:ANc.indptr[j + 1]]
        A = A.tocsr()
        colsum = np.asarray(A.sum(axis=0)).reshape(-1)
    out = (A @ sp.diags(col_target / colsum)).tocsr()
    out.sort_indices()
    return out


# ---------------------------------------------------------------- the step


def total_mass(mesh: Mesh, c) -> float:
    """sum_K |K|_phi c_K (Sec 2.1, discrete form of eq. mass-bal), exactly
    rounded."""
    return math.fsum((mesh.volphi() * np.asarray(c, dtype=np.float64)).tolist())


@dataclass
class StepOptions:
    n_scale: int = 10          # N of Algorithm 1 (Sec 4: N = 10)
    qp_tol: float = 1e-12      # scaled constraint residual at which the minimisation stops
    penalty: float = 1e-7      # eps of the constraint penalty in ``minimise``
    linear_from: float = 1e-6  # delta: relative violation beyond which that penalty is linear
    drop_tol: float = 1e-12
    cfl: float = 0.5
    substeps: int = 0          # 0: from the CFL rule


def step(mesh: Mesh, faces, dt: float, c, opts: StepOptions | None = None):
    """One B-char time step (Algorithm 1 followed by eq. phys-inter-ELLAM).

    Returns a dict with the intermediate matrices (A0, AN, A final, W), the
    minimisation result, the new c and the masses before and after."""
    opts = opts or StepOptions()
    s = opts.substeps or substep_count(mesh, faces, dt, opts.cfl)
    volphi = mesh.volphi()
    A0, ainfo = initial_matrix(mesh, faces, dt, s, opts.drop_tol)
    b_loc, n_unbal = balanced_targets(A0, volphi)
    AN = scale(A0, b_loc, volphi, opts.n_scale)
    colsum = np.asarray(AN.sum(axis=0)).reshape(-1)
    scale_err = float(np.max(np.abs(colsum - volphi) / volphi))
    factor, x, qinfo = minimise(AN, b_loc, volphi, opts.qp_tol, opts.penalty, opts.linear_from)
    Aq = AN.copy()
    Aq.data = AN.data * factor
    Afin = column_fix(Aq, AN, volphi)
    rowsum = np.asarray(Afin.sum(axis=1)).reshape(-1)
    colsum = np.asarray(Afin.sum(axis=0)).reshape(-1)
    qinfo.update({"max_rel_row_res": float(np.max(np.abs(rowsum - volphi) / volphi)),
                  "max_rel_col_res": float(np.max(np.abs(colsum - volphi) / volphi))})
    W = (sp.diags(1.0 / volphi) @ Afin).tocsr()
    W.sort_indices()
    c = np.asarray(c, dtype=np.float64)
    c_new = W @ c
    return {
        "substeps": s, "A0": A0, "AN": AN, "Aq": Aq, "A": Afin, "W": W, "x": x, "factor": factor,
        "c": c_new, "mass_before": total_mass(mesh, c), "mass_after": total_mass(mesh, c_new),
        "scale_err": scale_err, "b_loc": b_loc, "unbalanced": n_unbal, **{k: v for k, v in ainfo.items()}, **qinfo,
    }
