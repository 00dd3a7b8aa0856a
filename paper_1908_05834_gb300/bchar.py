"""ctypes binding of libbchar.so (include/bchar.h).

Argument marshalling only: every stage of a step runs in the library's CUDA
kernels.  The functions keep the C names (``bchar_create_mesh``,
``bchar_set_velocity``, ``bchar_step``, ``bchar_destroy`` ...); ``Mesh`` wraps
a handle.  Device arrays are torch CUDA tensors (PyTorch is used for device
memory and streams only).  There is no CPU fallback: if the compiled library
is missing this module raises on import.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbchar.so")

BCHAR_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA", 4: "BOUNDARY_FLUX", 5: "DIVERGENCE",
          6: "NONFINITE", 7: "NO_VELOCITY", 8: "CAPACITY"}
FP64, FP32_SPLIT = 0, 1
C_F64, C_F32 = 0, 1


class Options(ctypes.Structure):
    _fields_ = [("balls_per_axis", ctypes.c_int), ("n_scale", ctypes.c_int), ("precision", ctypes.c_int),
                ("substeps", ctypes.c_int), ("cfl", ctypes.c_double), ("drop_tol", ctypes.c_double),
                ("penalty", ctypes.c_double), ("qp_tol", ctypes.c_double), ("qp_max_iter", ctypes.c_int),
                ("qp_max_refine", ctypes.c_int), ("div_tol", ctypes.c_double), ("qp_precond", ctypes.c_int),
                ("qp_warm_start", ctypes.c_int), ("slab_width", ctypes.c_int)]


class StepInfo(ctypes.Structure):
    _fields_ = [("mass_before", ctypes.c_double), ("mass_after", ctypes.c_double),
                ("mass_after_stored", ctypes.c_double), ("max_rel_row_res", ctypes.c_double),
                ("max_rel_col_res", ctypes.c_double), ("scale_err", ctypes.c_double), ("kkt_rel", ctypes.c_double),
                ("nnz", ctypes.c_int64), ("substeps", ctypes.c_int32), ("cg_iters", ctypes.c_int32),
                ("ip_iters", ctypes.c_int32), ("qp_converged", ctypes.c_int32), ("void_balls", ctypes.c_int32),
                ("empty_cols", ctypes.c_int32), ("n_at_bounds", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("amg_levels", ctypes.c_int32), ("amg_coarsest", ctypes.c_int32), ("unbalanced", ctypes.c_int32),
                ("row_cap", ctypes.c_int32), ("spill_rows", ctypes.c_int32), ("max_row_len", ctypes.c_int32),
                ("ms_stage", ctypes.c_float * 8)]

    STAGES = ("track", "assemble", "columns_balance", "scaling", "minimise", "finalise", "update", "total")

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "ms_stage"}
        d["ms_stage"] = dict(zip(self.STAGES, (float(x) for x in self.ms_stage)))
        return d


class BcharError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{self.name}: {detail}" if detail else self.name)


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libbchar.so is not built ({LIB_PATH}); run __graft_entry__.build() first")

lib = ctypes.CDLL(LIB_PATH)
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_H = ctypes.c_void_p  # bchar_mesh_t

lib.bchar_default_options.argtypes = [ctypes.POINTER(Options)]
lib.bchar_default_options.restype = None
lib.bchar_create_mesh.argtypes = [ctypes.c_int, _P, _P, _P, ctypes.POINTER(Options), _P, ctypes.POINTER(_H)]
lib.bchar_create_mesh.restype = ctypes.c_int
lib.bchar_set_velocity.argtypes = [_H, _P, ctypes.c_int]
lib.bchar_set_velocity.restype = ctypes.c_int
lib.bchar_step.argtypes = [_H, ctypes.c_double, _P, _P, ctypes.c_int, ctypes.POINTER(StepInfo)]
lib.bchar_step.restype = ctypes.c_int
lib.bchar_destroy.argtypes = [_H]
lib.bchar_destroy.restype = None
lib.bchar_status_string.argtypes = [ctypes.c_int]
lib.bchar_status_string.restype = ctypes.c_char_p
lib.bchar_last_error.argtypes = [_H]
lib.bchar_last_error.restype = ctypes.c_char_p
lib.bchar_cell_count.argtypes = [_H]
lib.bchar_cell_count.restype = _I64
lib.bchar_ball_count.argtypes = [_H]
lib.bchar_ball_count.restype = _I64
lib.bchar_export_matrix.argtypes = [_H, ctypes.c_int, _P, _P, _P, _I64, ctypes.POINTER(_I64)]
lib.bchar_export_matrix.restype = ctypes.c_int
lib.bchar_export_tracked.argtypes = [_H, _P, _P, _P, _I64]
lib.bchar_export_tracked.restype = ctypes.c_int

lib.bchar_time_stage.argtypes = [_H, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]
lib.bchar_time_stage.restype = ctypes.c_int

STAGE_CG_MATVEC, STAGE_UPDATE, STAGE_ASSEMBLE, STAGE_TRACK, STAGE_SMOOTH, STAGE_SCALING, STAGE_VCYCLE = range(7)

lib.bchar_mass_noalloc.argtypes = [_P, _P, ctypes.c_int, _I64, _P, _P]
lib.bchar_mass_noalloc.restype = ctypes.c_int
lib.bchar_set_velocity_scaled.argtypes = [_H, _P, ctypes.c_int, ctypes.c_double]
lib.bchar_set_velocity_scaled.restype = ctypes.c_int
lib.bchar_device_bytes.argtypes = [_H, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]
lib.bchar_device_bytes.restype = ctypes.c_int
lib.bchar_estimate_device_bytes.argtypes = [ctypes.c_int, _P, _P, ctypes.POINTER(Options), ctypes.POINTER(_I64)]
lib.bchar_estimate_device_bytes.restype = ctypes.c_int
lib.bchar_step_batch.argtypes = [ctypes.c_int, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int]
lib.bchar_step_batch.restype = ctypes.c_int

bchar_default_options = lib.bchar_default_options
bchar_create_mesh = lib.bchar_create_mesh
bchar_set_velocity = lib.bchar_set_velocity
bchar_step = lib.bchar_step
bchar_destroy = lib.bchar_destroy
bchar_status_string = lib.bchar_status_string
bchar_last_error = lib.bchar_last_error
bchar_export_matrix = lib.bchar_export_matrix
bchar_export_tracked = lib.bchar_export_tracked
bchar_time_stage = lib.bchar_time_stage
bchar_mass_noalloc = lib.bchar_mass_noalloc
bchar_set_velocity_scaled = lib.bchar_set_velocity_scaled
bchar_device_bytes = lib.bchar_device_bytes
bchar_estimate_device_bytes = lib.bchar_estimate_device_bytes
bchar_step_batch = lib.bchar_step_batch


def default_options(**kw) -> Options:
    o = Options()
    lib.bchar_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr_array(arrs):
    return (ctypes.c_void_p * 3)(*([int(a) for a in arrs] + [0] * (3 - len(arrs))))


def _current_stream() -> int:
    import torch
    return torch.cuda.current_stream().cuda_stream


class Mesh:
    """A bchar_mesh_t: a tensor-product mesh with porosity, on the current
    CUDA stream (or ``stream``, a raw cudaStream_t)."""

    def __init__(self, coords, phi, options: Options | None = None, stream: int | None = None):
        self.coords = [np.ascontiguousarray(c, dtype=np.float64) for c in coords]
        self.dim = len(self.coords)
        self.n = [len(c) - 1 for c in self.coords]
        self.phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        self.options = options or default_options()
        self.stream = _current_stream() if stream is None else stream
        n_cells = (ctypes.c_int64 * 3)(*(self.n + [1] * (3 - self.dim)))
        cptrs = _ptr_array([c.ctypes.data for c in self.coords])
        h = _H()
        st = lib.bchar_create_mesh(self.dim, ctypes.addressof(n_cells), ctypes.addressof(cptrs),
                                   self.phi.ctypes.data, ctypes.byref(self.options), self.stream, ctypes.byref(h))
        if st != BCHAR_OK:
            raise BcharError(st, "bchar_create_mesh")
        self.handle = h
        self.nc = int(lib.bchar_cell_count(h))
        self.nballs = int(lib.bchar_ball_count(h))

    def _check(self, st: int, what: str):
        if st != BCHAR_OK:
            detail = lib.bchar_last_error(self.handle)
            raise BcharError(st, f"{what}: {detail.decode() if detail else ''}")

    def set_velocity(self, faces, scale: float = 1.0):
        """faces: dim face-velocity arrays, numpy (host) or torch CUDA tensors (device);
        the library multiplies them by ``scale`` on the device."""
        try:
            import torch
            on_device = isinstance(faces[0], torch.Tensor) and faces[0].is_cuda
        except ImportError:
            on_device = False
        if on_device:
            self._faces_keep = [f.contiguous().to(dtype=torch.float64) for f in faces]
            ptrs = _ptr_array([f.data_ptr() for f in self._faces_keep])
        else:
            self._faces_keep = [np.ascontiguousarray(f, dtype=np.float64).reshape(-1) for f in faces]
            ptrs = _ptr_array([f.ctypes.data for f in self._faces_keep])
        if scale == 1.0:
            st = lib.bchar_set_velocity(self.handle, ctypes.addressof(ptrs), int(on_device))
        else:
            st = lib.bchar_set_velocity_scaled(self.handle, ctypes.addressof(ptrs), int(on_device), float(scale))
        self._check(st, "set_velocity")

    def device_bytes(self) -> tuple[int, int]:
        """(bytes held now, peak) of the handle's device memory."""
        now, peak = _I64(0), _I64(0)
        self._check(lib.bchar_device_bytes(self.handle, ctypes.byref(now), ctypes.byref(peak)), "device_bytes")
        return int(now.value), int(peak.value)

    def step(self, dt: float, c_in, c_out) -> dict:
        """One time step; c_in / c_out are torch CUDA tensors of n_c float64 or float32."""
        import torch
        assert c_in.is_cuda and c_out.is_cuda and c_in.dtype == c_out.dtype
        assert c_in.is_contiguous() and c_out.is_contiguous() and c_in.numel() == self.nc == c_out.numel()
        dtype = C_F64 if c_in.dtype == torch.float64 else C_F32
        info = StepInfo()
        self._check(lib.bchar_step(self.handle, float(dt), c_in.data_ptr(), c_out.data_ptr(), dtype,
                                   ctypes.byref(info)), "step")
        return info.as_dict()

    def export_matrix(self, which: int):
        """(row_ptr, cols, vals) of the last step: 0 = A^(0), 1 = A^(N), 2 = final a_KM."""
        cap = _I64(0)
        row_ptr = np.zeros(self.nc + 1, dtype=np.int64)
        one = np.zeros(1, dtype=np.int32)
        oned = np.zeros(1)
        lib.bchar_export_matrix(self.handle, which, row_ptr.ctypes.data, one.ctypes.data, oned.ctypes.data, 0,
                                ctypes.byref(cap))
        nnz = cap.value
        cols = np.zeros(max(nnz, 1), dtype=np.int32)
        vals = np.zeros(max(nnz, 1))
        self._check(lib.bchar_export_matrix(self.handle, which, row_ptr.ctypes.data, cols.ctypes.data,
                                            vals.ctypes.data, nnz, ctypes.byref(cap)), "export_matrix")
        return row_ptr, cols[:nnz], vals[:nnz]

    def export_tracked(self):
        """(positions (nballs, 3), rhat (nballs,), ball_offset (n_c + 1,)) of the last step."""
        pos = np.zeros((self.nballs, 3))
        rh = np.zeros(self.nballs)
        off = np.zeros(self.nc + 1, dtype=np.int64)
        self._check(lib.bchar_export_tracked(self.handle, pos.ctypes.data, rh.ctypes.data, off.ctypes.data,
                                             self.nballs), "export_tracked")
        return pos, rh, off

    def time_stage(self, stage: int, reps: int = 20) -> float:
        """Mean milliseconds of one launch of a stage's kernel, replayed on the last step's data."""
        ms = ctypes.c_float(0.0)
        self._check(lib.bchar_time_stage(self.handle, stage, reps, ctypes.byref(ms)), "time_stage")
        return float(ms.value)

    def close(self):
        if getattr(self, "handle", None):
            lib.bchar_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def estimate_device_bytes(coords, options: Options | None = None) -> int:
    """A-priori device-memory estimate of a handle on this mesh (bchar_estimate_device_bytes)."""
    coords = [np.ascontiguousarray(c, dtype=np.float64) for c in coords]
    dim = len(coords)
    n_cells = (ctypes.c_int64 * 3)(*([len(c) - 1 for c in coords] + [1] * (3 - dim)))
    cptrs = _ptr_array([c.ctypes.data for c in coords])
    out = _I64(0)
    opt = options or default_options()
    st = lib.bchar_estimate_device_bytes(dim, ctypes.addressof(n_cells), ctypes.addressof(cptrs), ctypes.byref(opt),
                                         ctypes.byref(out))
    if st != BCHAR_OK:
        raise BcharError(st, "bchar_estimate_device_bytes")
    return int(out.value)


def step_batch(meshes, dts, c_ins, c_outs, max_workers: int = 0):
    """One step of several handles at once (bchar_step_batch).  Returns
    (infos, statuses); raises BcharError with the first failing status."""
    import torch
    k = len(meshes)
    hs = (ctypes.c_void_p * k)(*[m.handle.value for m in meshes])
    dt = (ctypes.c_double * k)(*[float(d) for d in dts])
    ci = (ctypes.c_void_p * k)(*[c.data_ptr() for c in c_ins])
    co = (ctypes.c_void_p * k)(*[c.data_ptr() for c in c_outs])
    for m, a, b in zip(meshes, c_ins, c_outs):
        assert a.is_cuda and b.is_cuda and a.dtype == b.dtype and a.numel() == b.numel() == m.nc
    dty = (ctypes.c_int * k)(*[C_F64 if c.dtype == torch.float64 else C_F32 for c in c_ins])
    infos = (StepInfo * k)()
    sts = (ctypes.c_int * k)()
    st = lib.bchar_step_batch(k, hs, dt, ci, co, dty, infos, sts, int(max_workers))
    if st != BCHAR_OK:
        bad = next(i for i in range(k) if sts[i] != BCHAR_OK) if any(sts[i] != BCHAR_OK for i in range(k)) else -1
        detail = lib.bchar_last_error(meshes[bad].handle) if bad >= 0 else b""
        raise BcharError(st, f"step_batch instance {bad}: {detail.decode() if detail else ''}")
    return [infos[i].as_dict() for i in range(k)], [int(sts[i]) for i in range(k)]
