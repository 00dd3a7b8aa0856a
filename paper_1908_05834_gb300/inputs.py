"""Seeded synthetic inputs for the B-char workloads.

This module holds problem data only -- meshes, porosity, the face velocities
of the analytic flow fields and the initial concentrations -- and none of the
method's arithmetic.  Both the CUDA path (through the tests and the benchmark)
and the CPU oracle are fed from here; neither depends on the other.

Workloads (mesh sizes, fields, time steps) follow the benchmark definitions:

* ``vortex2d_32``   uniform 32x32, phi = 1, steady field
  u = (-sin^2(pi x) sin(2 pi y), sin(2 pi x) sin^2(pi y)), disk c0, dt 0.01, 20 steps
* ``vortex2d_1024`` 1024x1024 tensor mesh, widths U[0.5h, 1.5h] (seed 1001),
  phi = 1, the same field times cos(pi t / T), T = 1, dt 0.005, 200 steps
* ``deform3d_128``  uniform 128^3, phi log-uniform in [0.1, 0.3] (seed 2002),
  u = (2 sin^2(pi x) sin(2pi y) sin(2pi z), -sin(2pi x) sin^2(pi y) sin(2pi z),
       -sin(2pi x) sin(2pi y) sin^2(pi z)) cos(pi t / T), T = 1.5, dt 0.01, 150 steps
* ``deform3d_256``  256^3 tensor mesh, widths U[0.7h, 1.3h] (seed 3001), phi
  log-uniform in [0.05, 0.3] (seed 3002), T = 1.5, dt 0.005, 300 steps,
  Gaussian c0 stored in FP32

Velocities are lowest-order Raviart-Thomas face values: the exact average of
u.n over each face at the mid-step time t^n + dt/2, with the boundary faces
set to exactly 0 (u.n = 0 on the boundary).  The fields are separable, so the
averages are closed forms and the discrete divergence of every cell vanishes
up to rounding.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import erf


def uniform_coords(n: int) -> np.ndarray:
    return np.linspace(0.0, 1.0, n + 1)


def stretched_coords(rng: np.random.Generator, n: int, lo: float, hi: float) -> np.ndarray:
    """n widths drawn uniformly in [lo*h, hi*h] (h = 1/n), renormalised to [0, 1]."""
    h = 1.0 / n
    w = rng.uniform(lo * h, hi * h, n)
    x = np.concatenate([[0.0], np.cumsum(w)]) / np.sum(w)
    x[0] = 0.0
    x[-1] = 1.0
    return x


def log_uniform_phi(rng: np.random.Generator, nc: int, lo: float, hi: float) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), nc))


def _avg_sin2pi(x: np.ndarray) -> np.ndarray:
    """Average of sin(2 pi s) over each interval [x_i, x_{i+1}]."""
    return (np.cos(2 * np.pi * x[:-1]) - np.cos(2 * np.pi * x[1:])) / (2 * np.pi * np.diff(x))


def _sin2(x: np.ndarray) -> np.ndarray:
    s = np.sin(np.pi * x) ** 2
    s[0] = 0.0
    s[-1] = 0.0
    return s


def vortex2d_faces(coords, g: float = 1.0):
    """Face averages of u = g * (-sin^2(pi x) sin(2 pi y), sin(2 pi x) sin^2(pi y)).
    Returns [U_x of shape (ny, nx+1), U_y of shape (ny+1, nx)], x index fastest."""
    x, y = coords
    ux = -g * np.outer(_avg_sin2pi(y), _sin2(x))
    uy = g * np.outer(_sin2(y), _avg_sin2pi(x))
    return [np.ascontiguousarray(ux), np.ascontiguousarray(uy)]


def deform3d_faces(coords, g: float = 1.0):
    """Face averages of u = g * (2 sin^2(pi x) sin(2pi y) sin(2pi z),
    -sin(2pi x) sin^2(pi y) sin(2pi z), -sin(2pi x) sin(2pi y) sin^2(pi z)).
    Shapes (nz, ny, nx+1), (nz, ny+1, nx), (nz+1, ny, nx)."""
    x, y, z = coords
    ax, ay, az = _avg_sin2pi(x), _avg_sin2pi(y), _avg_sin2pi(z)
    sx, sy, sz = _sin2(x), _sin2(y), _sin2(z)
    ux = 2.0 * g * az[:, None, None] * ay[None, :, None] * sx[None, None, :]
    uy = -g * az[:, None, None] * sy[None, :, None] * ax[None, None, :]
    uz = -g * sz[:, None, None] * ay[None, :, None] * ax[None, None, :]
    return [np.ascontiguousarray(u) for u in (ux, uy, uz)]


def indicator_ball_average(coords, centre, radius: float, q: int = 16) -> np.ndarray:
    """Cell averages of the indicator of |x - centre| < radius: 1 or 0 for cells
    wholly inside or outside, q^d-point midpoint rule for cut cells.  x fastest."""
    d = len(coords)
    lo1 = [np.asarray(c[:-1], dtype=np.float64) for c in coords]
    hi1 = [np.asarray(c[1:], dtype=np.float64) for c in coords]

    def along(v, a):  # a 1D per-axis array placed on axis a of the (n_0, ..., n_{d-1}) grid
        shape = [1] * d
        shape[a] = v.shape[0]
        return v.reshape(shape)

    near = np.zeros([len(v) for v in lo1])
    far = np.zeros([len(v) for v in lo1])
    for a in range(d):
        dlo = lo1[a] - centre[a]
        dhi = hi1[a] - centre[a]
        near = near + along(np.where((dlo <= 0) & (dhi >= 0), 0.0, np.minimum(dlo ** 2, dhi ** 2)), a)
        far = far + along(np.maximum(dlo ** 2, dhi ** 2), a)
    out = np.where(far <= radius ** 2, 1.0, 0.0)
    cut = (near < radius ** 2) & (far > radius ** 2)
    idx = np.nonzero(cut)
    t = (np.arange(q) + 0.5) / q
    # the q^d points of every cut cell at once: axis a varies along dimension 1 + a
    sq = []
    for a in range(d):
        l, h = lo1[a][idx[a]], hi1[a][idx[a]]
        p = l[:, None] + t[None, :] * (h - l)[:, None]
        shape = [p.shape[0]] + [1] * d
        shape[1 + a] = q
        sq.append(((p - centre[a]) ** 2).reshape(shape))
    r2 = sq[0]
    for a in range(1, d):
        r2 = r2 + sq[a]
    inside = (r2 < radius ** 2).reshape(r2.shape[0], -1)
    out[idx] = np.count_nonzero(inside, axis=1) / q ** d
    return np.ascontiguousarray(out.transpose(*reversed(range(d))).reshape(-1))


def gaussian_average(coords, centre, sigma2: float) -> np.ndarray:
    """Cell averages of exp(-|x - centre|^2 / sigma2) (separable, exact via erf)."""
    d = len(coords)
    s = math.sqrt(sigma2)
    f = []
    for a in range(d):
        x = coords[a]
        f.append(0.5 * math.sqrt(math.pi) * s * (erf((x[1:] - centre[a]) / s) - erf((x[:-1] - centre[a]) / s))
                 / np.diff(x))
    out = f[0]
    for a in range(1, d):
        out = np.multiply.outer(f[a], out) if a == 1 else np.multiply.outer(f[a], out)
    # out has axes (z, y, x) or (y, x): x fastest after reshape
    return np.ascontiguousarray(out.reshape(-1))


@dataclass
class Workload:
    name: str
    dim: int
    coords: list
    phi: np.ndarray
    dt: float
    steps: int
    T: float | None          # None: steady field
    field: str               # "vortex2d" | "deform3d"
    c0: np.ndarray
    c_dtype: str = "f64"
    precision: str = "fp64"  # "fp64" | "fp32split"

    @property
    def nc(self) -> int:
        return int(np.prod([len(c) - 1 for c in self.coords]))

    def time_factor(self, step: int) -> float:
        """cos(pi t / T) at the mid-step time t = (step + 1/2) dt; 1 for a steady field."""
        if self.T is None:
            return 1.0
        return math.cos(math.pi * (step + 0.5) * self.dt / self.T)

    def faces(self, step: int = 0, amplitude: float = 1.0):
        g = amplitude * self.time_factor(step)
        if self.field == "vortex2d":
            return vortex2d_faces(self.coords, g)
        return deform3d_faces(self.coords, g)


def workload(name: str, n: int | None = None, steps: int | None = None) -> Workload:
    """One of the named workloads; ``n`` overrides the cells per axis with the
    same recipe (same seeds, distributions and fields) for smaller test cases."""
    if name == "vortex2d_32":
        nn = n or 32
        coords = [uniform_coords(nn), uniform_coords(nn)]
        c0 = indicator_ball_average(coords, (0.5, 0.75), 0.15)
        return Workload(name, 2, coords, np.ones(nn * nn), 0.01, steps or 20, None, "vortex2d", c0)
    if name == "vortex2d_1024":
        nn = n or 1024
        rng = np.random.Generator(np.random.PCG64(1001))
        coords = [stretched_coords(rng, nn, 0.5, 1.5), stretched_coords(rng, nn, 0.5, 1.5)]
        c0 = indicator_ball_average(coords, (0.5, 0.75), 0.15)
        return Workload(name, 2, coords, np.ones(nn * nn), 0.005, steps or 200, 1.0, "vortex2d", c0,
                        precision="fp32split")
    if name == "deform3d_128":
        nn = n or 128
        coords = [uniform_coords(nn)] * 3
        rng = np.random.Generator(np.random.PCG64(2002))
        phi = log_uniform_phi(rng, nn ** 3, 0.1, 0.3)
        c0 = indicator_ball_average(coords, (0.35, 0.35, 0.35), 0.15)
        return Workload(name, 3, coords, phi, 0.01, steps or 150, 1.5, "deform3d", c0, precision="fp32split")
    if name == "deform3d_256":
        nn = n or 256
        rng = np.random.Generator(np.random.PCG64(3001))
        coords = [stretched_coords(rng, nn, 0.7, 1.3) for _ in range(3)]
        rng2 = np.random.Generator(np.random.PCG64(3002))
        phi = log_uniform_phi(rng2, nn ** 3, 0.05, 0.3)
        c0 = gaussian_average(coords, (0.35, 0.35, 0.35), 0.01).astype(np.float32)
        return Workload(name, 3, coords, phi, 0.005, steps or 300, 1.5, "deform3d", c0, c_dtype="f32",
                        precision="fp32split")
    raise KeyError(name)


WORKLOADS = ("vortex2d_32", "vortex2d_1024", "deform3d_128", "deform3d_256")

_SPLIT = "FP32 tracking and intersections, FP64 sums/scalings/minimisation/update"
_RECIPES = {
    "vortex2d_32": (32, "uniform {n}x{n} mesh, phi=1, steady single vortex, dt=0.01, disk c0; FP64 throughout"),
    "vortex2d_1024": (1024, "{n}x{n} stretched tensor mesh (widths U[0.5h,1.5h], seed 1001), phi=1, single vortex "
                            "x cos(pi t/T), T=1, dt=0.005, disk c0; " + _SPLIT),
    "deform3d_128": (128, "uniform {n}^3 mesh, phi log-U[0.1,0.3] (seed 2002), deformation field x cos(pi t/T), "
                          "T=1.5, dt=0.01, ball c0; " + _SPLIT),
    "deform3d_256": (256, "{n}^3 stretched tensor mesh (widths U[0.7h,1.3h], seed 3001), phi log-U[0.05,0.3] "
                          "(seed 3002), deformation field x cos(pi t/T), T=1.5, dt=0.005, Gaussian c0 stored in "
                          "FP32; " + _SPLIT),
}


def describe(name: str, n: int | None = None) -> str:
    """One line naming a workload's recipe and size (for measurement records)."""
    default, text = _RECIPES[name]
    return text.format(n=n or default)


# ---------------------------------------------------------------- serving stream

@dataclass
class ServeRequest:
    """One request of the serving stream: a small transport problem, run for
    ``steps`` steps.  Arrays are built by ``materialize`` (problem data only)."""
    rid: int
    arrival_s: float         # offset from the start of the stream
    dim: int
    n: int                   # cells per axis (uniform mesh)
    amplitude: float         # A: the field is A u(x) cos(pi t / T)
    cfl: float
    steps: int
    phi_seed: int

    @property
    def nc(self) -> int:
        return self.n ** self.dim

    @property
    def T(self) -> float:
        return 1.0 if self.dim == 2 else 1.5

    @property
    def dt(self) -> float:
        """dt = CFL h phi_min / (A U_max), U_max = 1 (2D) or 2 (3D), phi_min = 1 (2D) or 0.1 (3D)."""
        h = 1.0 / self.n
        phi_min, umax = (1.0, 1.0) if self.dim == 2 else (0.1, 2.0)
        return self.cfl * h * phi_min / (self.amplitude * umax)

    def time_factor(self, step: int) -> float:
        """A cos(pi t / T) at the mid-step time of ``step``."""
        return self.amplitude * math.cos(math.pi * (step + 0.5) * self.dt / self.T)

    def materialize(self, q: int = 4):
        """(coords, phi, base face velocities u(x), c0): the face arrays are the
        unscaled field; step k uses them times ``time_factor(k)``."""
        coords = [uniform_coords(self.n)] * self.dim
        if self.dim == 2:
            phi = np.ones(self.nc)
            faces = vortex2d_faces(coords, 1.0)
            c0 = indicator_ball_average(coords, (0.5, 0.75), 0.15, q)
        else:
            rng = np.random.Generator(np.random.PCG64(self.phi_seed))
            phi = log_uniform_phi(rng, self.nc, 0.1, 0.3)
            faces = deform3d_faces(coords, 1.0)
            c0 = indicator_ball_average(coords, (0.35, 0.35, 0.35), 0.15, q)
        return coords, phi, faces, c0


def serving_requests(count: int = 512, seed: int = 4004, mean_gap_s: float = 0.002) -> list[ServeRequest]:
    """The serving stream: Poisson arrivals (mean gap 2 ms); 60 % 2D requests,
    N log-uniform in [64, 1024], phi = 1, the vortex field; 40 % 3D requests, N
    log-uniform in [32, 160], phi log-uniform in [0.1, 0.3], the deformation
    field; amplitude U[0.5, 2], CFL U[0.5, 4], 10-100 steps (uniform)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out, t = [], 0.0
    for rid in range(count):
        t += rng.exponential(mean_gap_s)
        two_d = rng.uniform() < 0.6
        lo, hi = (64, 1024) if two_d else (32, 160)
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        out.append(ServeRequest(rid=rid, arrival_s=t, dim=2 if two_d else 3, n=n,
                                amplitude=float(rng.uniform(0.5, 2.0)), cfl=float(rng.uniform(0.5, 4.0)),
                                steps=int(rng.integers(10, 101)), phi_seed=int(rng.integers(1, 2 ** 31))))
    return out
