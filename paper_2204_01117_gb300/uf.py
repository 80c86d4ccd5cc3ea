"""ctypes binding of the C ABI in ``include/uf.h`` (argument marshalling only).

Every step of the solver runs in the CUDA library ``_build/libuf.so``; this
module builds nothing at import time and has no fallback: if the library is
missing, ``load()`` raises.  PyTorch supplies device memory (the workspace) and
the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import re
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(_HERE)
CSRC = os.path.join(_HERE, "csrc")
LIB_PATH = os.path.join(_HERE, "_build", "libuf.so")
# debug build with device-side bounds checks of every global index (-DUF_BOUNDS_CHECK)
CHECKED_LIB_PATH = os.path.join(_HERE, "_build_checked", "libuf.so")
HEADER = os.path.join(ROOT, "include", "uf.h")
SOURCES = ["capi.cu", "noalloc.cu", "batch.cu"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-lineinfo",
              "--expt-extended-lambda", "-Xcompiler", "-fPIC", "-shared"]

UF_OK, UF_ERR_ARG, UF_ERR_CUDA, UF_ERR_NOMEM, UF_ERR_NOT_CONVERGED, UF_ERR_NAN, UF_ERR_TIMEOUT, UF_ERR_STATE, UF_ERR_BOUNDS = range(9)
STATUS_NAMES = ["UF_OK", "UF_ERR_ARG", "UF_ERR_CUDA", "UF_ERR_NOMEM", "UF_ERR_NOT_CONVERGED", "UF_ERR_NAN",
                "UF_ERR_TIMEOUT", "UF_ERR_STATE", "UF_ERR_BOUNDS"]
F32, F64 = 0, 1
PRECOND = {"mg": 0, "ai1": 1, "jacobi": 2, "none": 3, "ai2": 4}
STOP_RULE = {"residual": 0, "paper": 1}
SMOOTHER = {"jacobi": 0, "rbgs": 1, "cheby": 2}
TRANSFER = {"constant": 0, "linear": 1}
FIELDS = {"u": 0, "v": 1, "w": 2, "p": 3, "k": 4, "omega": 5, "phi": 6, "nut": 7}


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("h", ctypes.c_double), ("precision", ctypes.c_int),
        ("wind_dir_deg", ctypes.c_double), ("u_ref", ctypes.c_double),
        ("z_ref", ctypes.c_double), ("z0", ctypes.c_double),
        ("inflow_loglaw", ctypes.c_int), ("ground_noslip", ctypes.c_int),
        ("rho", ctypes.c_double), ("nu", ctypes.c_double), ("Cd", ctypes.c_double),
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("e", ctypes.c_double),
        ("I", ctypes.c_double), ("L", ctypes.c_double),
        ("C_mu", ctypes.c_double), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
        ("sigma", ctypes.c_double), ("sigma_star", ctypes.c_double), ("C_lim", ctypes.c_double),
        ("cfl", ctypes.c_double), ("fixed_dt", ctypes.c_double),
        ("k_min", ctypes.c_double), ("omega_min", ctypes.c_double),
        ("precond", ctypes.c_int), ("cg_tol", ctypes.c_double), ("cg_max_iter", ctypes.c_int),
        ("ai_omega", ctypes.c_double), ("mg_jacobi_omega", ctypes.c_double),
        ("mg_coarse_max", ctypes.c_int), ("mg_smoother", ctypes.c_int),
        ("cg_stop_rule", ctypes.c_int), ("mg_transfer", ctypes.c_int),
    ]


class StepStats(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("cg_iters", ctypes.c_int),
                ("cg_rel_residual", ctypes.c_double), ("status", ctypes.c_int),
                ("cg_iters_total", ctypes.c_longlong)]


MAX_LEVELS = 16
# uf_substep: id, input fields, output fields (include/uf.h, "Sub-steps")
SUBSTEPS = {
    "eddy": (0, ("u", "v", "w", "k", "omega"), ("nut",)),
    "advect": (1, ("u", "v", "w"), ("u", "v", "w")),
    "diffuse": (2, ("u", "v", "w", "nut"), ("u", "v", "w")),
    "drag_bc": (3, ("u", "v", "w", "phi"), ("u", "v", "w")),
    "project": (4, ("u", "v", "w"), ("u", "v", "w")),
    "turb": (5, ("u", "v", "w", "k", "omega"), ("k", "omega")),
}
MAX_REGIONS = 8


class ObjectiveDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("z_lo", ctypes.c_double), ("z_hi", ctypes.c_double),
                ("u_hi", ctypes.c_double), ("u_lo", ctypes.c_double), ("nreg", ctypes.c_int),
                ("regions", ctypes.POINTER(ctypes.c_double)), ("u_t", ctypes.c_double)]


def objective_desc(objective=None, band=(1.0, 3.0, 4.0, 1.0)):
    """(uf_objective_desc, keep-alive).  objective: None or {"kind":
    "comfort", "band": (z_lo, z_hi, u_hi, u_lo)} for the comfort band, or
    {"kind": "regions", "regions": [(x0, x1, y0, y1, z0, z1), ...], "u_t":
    0.55} for the region-average objective of Sec. 6."""
    d = ObjectiveDesc()
    keep = None
    if objective is None or objective.get("kind", "comfort") == "comfort":
        b = band if objective is None else objective.get("band", band)
        d.kind = 0
        d.z_lo, d.z_hi, d.u_hi, d.u_lo = b
    else:
        r = np.ascontiguousarray(np.asarray(objective["regions"], dtype=np.float64).reshape(-1, 6))
        d.kind = 1
        d.nreg = r.shape[0]
        d.regions = r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.u_t = float(objective.get("u_t", 0.55))
        keep = r
    return d, keep


class Tuning(ctypes.Structure):
    _fields_ = [("tail_level", ctypes.c_int), ("march_zc", ctypes.c_int * MAX_LEVELS),
                ("advect_zc", ctypes.c_int), ("unfused", ctypes.c_int), ("coarse_start", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {"tail_level": self.tail_level, "march_zc": list(self.march_zc), "advect_zc": self.advect_zc,
                "unfused": self.unfused, "coarse_start": self.coarse_start}


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int), ("total_ms", ctypes.c_double),
                ("bytes_per_launch", ctypes.c_double)]


class UFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile the CUDA sources into _build/libuf.so for sm_103a (nvcc).
    checked=True: the debug build with bounds checks of every global index
    (-DUF_BOUNDS_CHECK; an index outside its array makes the call return
    UF_ERR_BOUNDS) into _build_checked/libuf.so; load it by setting
    UF_LIBRARY to that path before the first load()."""
    lib_path = CHECKED_LIB_PATH if checked else LIB_PATH
    with _lock:
        srcs = [os.path.join(CSRC, s) for s in SOURCES]
        deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")] + [HEADER]
        if (not force and os.path.exists(lib_path)
                and os.path.getmtime(lib_path) >= max(os.path.getmtime(p) for p in deps)):
            return lib_path
        os.makedirs(os.path.dirname(lib_path), exist_ok=True)
        tag = f".tmp{os.getpid()}"
        objs, procs = [], []
        compile_flags = [f for f in NVCC_FLAGS if f != "-shared"] + (["-DUF_BOUNDS_CHECK"] if checked else [])
        for src in srcs:   # translation units compile in parallel
            obj = os.path.join(os.path.dirname(lib_path), os.path.basename(src) + tag + ".o")
            cmd = ["nvcc", *compile_flags, "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd))
            procs.append(subprocess.Popen(cmd))
            objs.append(obj)
        codes = [pr.wait() for pr in procs]
        if any(codes):
            raise subprocess.CalledProcessError(max(codes), "nvcc")
        tmp = lib_path + tag
        subprocess.check_call(["nvcc", "-shared", "-gencode", "arch=compute_103a,code=sm_103a", *objs, "-o", tmp])
        for obj in objs:
            os.remove(obj)
        os.replace(tmp, lib_path)
        return lib_path


def declared_functions() -> list[str]:
    """Names of the functions include/uf.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(uf_[a-z_0-9]+)\s*\(", text)))


def load():
    """Load _build/libuf.so (or the library the environment variable
    UF_LIBRARY names, e.g. the bounds-checked build); raises OSError when it
    has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("UF_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: run paper_2204_01117_gb300.uf.build() first")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    lib.uf_default_desc.argtypes = [P(GridDesc)]
    lib.uf_default_desc.restype = None
    lib.uf_workspace_bytes.argtypes = [P(GridDesc)]
    lib.uf_workspace_bytes.restype = ctypes.c_size_t
    lib.uf_create_grid.argtypes = [P(GridDesc), vp, ctypes.c_size_t, vp, P(vp)]
    lib.uf_destroy.argtypes = [vp]
    lib.uf_set_porosity.argtypes = [vp, vp]
    lib.uf_set_state.argtypes = [vp, ip, vp]
    lib.uf_get_state.argtypes = [vp, ip, vp]
    lib.uf_init_state.argtypes = [vp]
    lib.uf_step.argtypes = [vp, P(StepStats)]
    lib.uf_run.argtypes = [vp, ip, P(StepStats)]
    lib.uf_objective.argtypes = [vp, dp, dp, dp, dp, P(dp)]
    lib.uf_divergence.argtypes = [vp, P(dp)]
    lib.uf_apply_poisson.argtypes = [vp, vp, vp]
    lib.uf_poisson_solve.argtypes = [vp, vp, P(ip), P(dp)]
    lib.uf_last_step_launches.argtypes = [vp]
    lib.uf_last_step_launches.restype = ip
    lib.uf_last_error.restype = ctypes.c_char_p
    lib.uf_profile_step.argtypes = [vp, P(KernelTime), ip, P(ip), P(StepStats)]
    lib.uf_profile_step.restype = ip
    lib.uf_launch_counts.argtypes = [vp, P(ip), P(ip)]
    lib.uf_launch_counts.restype = ip
    lib.uf_adjoint_workspace_bytes.argtypes = [vp, ip, ip]
    lib.uf_adjoint_workspace_bytes.restype = ctypes.c_size_t
    lib.uf_adjoint_run.argtypes = [vp, vp, ctypes.c_size_t, ip, ip, dp, dp, dp, dp, vp, P(dp)]
    lib.uf_adjoint_run.restype = ip
    lib.uf_set_fields.argtypes = [vp, ip, P(ip), P(vp)]
    lib.uf_set_fields.restype = ip
    lib.uf_get_fields.argtypes = [vp, ip, P(ip), P(vp)]
    lib.uf_get_fields.restype = ip
    lib.uf_state_bytes.argtypes = [vp]
    lib.uf_state_bytes.restype = ctypes.c_size_t
    lib.uf_save_state.argtypes = [vp, vp, ctypes.c_size_t]
    lib.uf_save_state.restype = ip
    lib.uf_load_state.argtypes = [vp, vp, ctypes.c_size_t]
    lib.uf_load_state.restype = ip
    lib.uf_objective_ex.argtypes = [vp, P(ObjectiveDesc), P(dp)]
    lib.uf_objective_ex.restype = ip
    lib.uf_adjoint_run_ex.argtypes = [vp, vp, ctypes.c_size_t, ip, ip, P(ObjectiveDesc), vp, P(dp)]
    lib.uf_adjoint_run_ex.restype = ip
    lib.uf_step_vjp.argtypes = [vp, vp, ctypes.c_size_t, P(vp), P(vp), vp]
    lib.uf_substep.argtypes = [vp, ip, ip, P(vp), P(vp), P(vp)]
    lib.uf_mesh_to_phi.argtypes = [vp, ip, P(dp), ip, P(ip), P(ip), P(dp), ip, vp]
    lib.uf_mesh_to_phi.restype = ip
    lib.uf_substep.restype = ip
    lib.uf_step_vjp.restype = ip
    lib.uf_design_to_phi.argtypes = [vp, ip, P(dp), P(dp), dp, vp]
    lib.uf_design_to_phi.restype = ip
    lib.uf_design_vjp.argtypes = [vp, ip, P(dp), P(dp), dp, vp, P(dp)]
    lib.uf_design_vjp.restype = ip
    lib.uf_poisson_solve_static.argtypes = [ip, ip, ip, dp, vp, vp, dp, ip, vp, P(ip), P(dp)]
    lib.uf_poisson_solve_static.restype = ip
    lib.uf_get_tuning.argtypes = [vp, P(Tuning), P(ip)]
    lib.uf_get_tuning.restype = ip
    lib.uf_set_tuning.argtypes = [vp, P(Tuning)]
    lib.uf_set_tuning.restype = ip
    lib.uf_autotune.argtypes = [vp, ip, P(Tuning), P(dp)]
    lib.uf_autotune.restype = ip
    lib.uf_batch_workspace_bytes.argtypes = [ip, P(GridDesc)]
    lib.uf_batch_workspace_bytes.restype = ctypes.c_size_t
    lib.uf_batch_create.argtypes = [ip, P(GridDesc), vp, ctypes.c_size_t, vp, P(vp)]
    lib.uf_batch_create.restype = ip
    lib.uf_batch_grid.argtypes = [vp, ip, P(vp)]
    lib.uf_batch_grid.restype = ip
    lib.uf_batch_run.argtypes = [vp, ip, P(StepStats)]
    lib.uf_batch_run.restype = ip
    lib.uf_batch_launch_counts.argtypes = [vp, P(ip), P(ip)]
    lib.uf_batch_launch_counts.restype = ip
    lib.uf_batch_autotune.argtypes = [vp, ip, P(ip)]
    lib.uf_batch_autotune.restype = ip
    lib.uf_batch_profile_step.argtypes = [vp, P(KernelTime), ip, P(ip)]
    lib.uf_batch_profile_step.restype = ip
    lib.uf_batch_destroy.argtypes = [vp]
    lib.uf_batch_destroy.restype = ip
    for name in ("uf_create_grid", "uf_destroy", "uf_set_porosity", "uf_set_state", "uf_get_state",
                 "uf_init_state", "uf_step", "uf_run", "uf_objective", "uf_divergence",
                 "uf_apply_poisson", "uf_poisson_solve"):
        getattr(lib, name).restype = ip
    _lib = lib
    return lib


def last_error() -> str:
    return load().uf_last_error().decode()


def check(status: int) -> None:
    if status != UF_OK:
        raise UFError(status, last_error())


def default_desc(**overrides) -> GridDesc:
    d = GridDesc()
    load().uf_default_desc(ctypes.byref(d))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = {"f32": F32, "f64": F64}[v]
        if k == "precond" and isinstance(v, str):
            v = PRECOND[v]
        if k == "mg_smoother" and isinstance(v, str):
            v = SMOOTHER[v]
        if k == "cg_stop_rule" and isinstance(v, str):
            v = STOP_RULE[v]
        if k == "mg_transfer" and isinstance(v, str):
            v = TRANSFER[v]
        if not hasattr(d, k):
            raise TypeError(f"unknown grid parameter {k!r}")
        setattr(d, k, v)
    return d


def workspace_bytes(desc: GridDesc) -> int:
    return int(load().uf_workspace_bytes(ctypes.byref(desc)))


def _torch():
    import torch
    return torch


def _is_tensor(buf) -> bool:
    try:
        return isinstance(buf, _torch().Tensor)
    except ImportError:
        return False


def _ptr(buf, dtype):
    """(pointer, keep-alive) of a torch tensor (device or host) or numpy array."""
    try:
        import torch
        if isinstance(buf, torch.Tensor):
            if buf.dtype != dtype[0] or not buf.is_contiguous():
                raise TypeError(f"expected a contiguous {dtype[0]} tensor")
            return ctypes.c_void_p(buf.data_ptr()), buf
    except ImportError:
        pass
    arr = np.ascontiguousarray(buf, dtype=dtype[1])
    return ctypes.c_void_p(arr.ctypes.data), arr


STATIC_MAX_CELLS = 800000
UNFUSED_ADVECT, UNFUSED_MOMENTUM = 1, 2
UNFUSED_ALL = UNFUSED_ADVECT | UNFUSED_MOMENTUM


_static_streams = {}


def poisson_solve_static(b, p, wind_dir_deg: float = 0.0, tol: float = 1e-7, max_iter: int = 5000, stream=None):
    """uf_poisson_solve_static on dense float32 CUDA tensors b (in) and p (in/out).

    The solve allocates no device memory: its scratch is a fixed array inside
    the library (see include/uf.h).  b and p must live on the current CUDA
    device, whose copy of the scratch the call uses.  The C entry point needs
    a created (non-default) stream; with stream=None the call runs on one
    such stream kept per device, after the work already queued on the
    current stream.  The call returns when the solve is done.  Returns
    (iterations, relative residual)."""
    import torch
    lib = load()
    if b.dtype != torch.float32 or p.dtype != torch.float32 or not b.is_cuda or not p.is_cuda:
        raise TypeError("b and p must be float32 CUDA tensors")
    if not (b.is_contiguous() and p.is_contiguous()) or b.shape != p.shape or b.dim() != 3:
        raise TypeError("b and p must be contiguous (nz, ny, nx) tensors of the same shape")
    dev = torch.cuda.current_device()
    if b.device.index != dev or p.device.index != dev:
        raise TypeError(f"b and p must be on the current CUDA device (cuda:{dev}); "
                        f"got {b.device} and {p.device}")
    nz, ny, nx = b.shape
    if stream is None:
        s = _static_streams.get(dev)
        if s is None:
            s = _static_streams[dev] = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream(dev))
    else:
        s = stream
    if s.cuda_stream == 0:
        raise TypeError("poisson_solve_static needs a created CUDA stream, not the legacy default stream")
    it, rel = ctypes.c_int(), ctypes.c_double()
    check(lib.uf_poisson_solve_static(nx, ny, nz, wind_dir_deg, ctypes.c_void_p(b.data_ptr()),
                                      ctypes.c_void_p(p.data_ptr()), tol, max_iter,
                                      ctypes.c_void_p(s.cuda_stream), ctypes.byref(it), ctypes.byref(rel)))
    return it.value, rel.value


class Grid:
    """One simulation grid on the current CUDA device (see include/uf.h)."""

    def __init__(self, nx: int, ny: int, nz: int, precision: str = "f32", stream=None, **params):
        import torch
        self.lib = load()
        self.desc = default_desc(nx=nx, ny=ny, nz=nz, precision=precision, **params)
        if precision == "f64":
            self.torch_dtype, self.np_dtype = torch.float64, np.float64
        else:
            self.torch_dtype, self.np_dtype = torch.float32, np.float32
        nbytes = workspace_bytes(self.desc)
        if nbytes == 0:
            raise UFError(UF_ERR_ARG, last_error())
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = ctypes.c_void_p()
        check(self.lib.uf_create_grid(ctypes.byref(self.desc), ctypes.c_void_p(self.workspace.data_ptr()),
                                      nbytes, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h
        self._owned = True
        self._init_shapes(nx, ny, nz)

    def _init_shapes(self, nx, ny, nz):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.shapes = {"u": (nz, ny, nx + 1), "v": (nz, ny + 1, nx), "w": (nz + 1, ny, nx),
                       "p": (nz, ny, nx), "k": (nz, ny, nx), "omega": (nz, ny, nx),
                       "phi": (nz, ny, nx), "nut": (nz, ny, nx)}

    @classmethod
    def _borrowed(cls, owner, handle, desc: GridDesc, stream):
        """A grid whose handle belongs to `owner` (a Batch): never destroyed here."""
        import torch
        g = cls.__new__(cls)
        g.lib = load()
        g.desc = desc
        if desc.precision == F64:
            g.torch_dtype, g.np_dtype = torch.float64, np.float64
        else:
            g.torch_dtype, g.np_dtype = torch.float32, np.float32
        g.workspace = None
        g.stream = stream
        g._h = handle
        g._owned = False
        g._owner = owner
        g._init_shapes(desc.nx, desc.ny, desc.nz)
        return g

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                self.lib.uf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dtypes(self):
        return (self.torch_dtype, self.np_dtype)

    def _arg(self, buf):
        """Pointer to a numpy array or tensor; a CUDA tensor made on torch's
        current stream is ordered before the grid's stream uses it."""
        ptr, keep = _ptr(buf, self.dtypes)
        if _is_tensor(buf) and buf.is_cuda:
            self.stream.wait_stream(_torch().cuda.current_stream())
        return ptr, keep

    def set_porosity(self, phi) -> None:
        ptr, keep = self._arg(phi)
        check(self.lib.uf_set_porosity(self._h, ptr))

    def set_state(self, name: str, value) -> None:
        if np.isscalar(value):
            value = np.full(self.shapes[name], value, dtype=self.np_dtype)
        ptr, keep = self._arg(value)
        check(self.lib.uf_set_state(self._h, FIELDS[name], ptr))

    def get_state(self, name: str, out=None):
        """Returns the field as a numpy array (host), or fills ``out``."""
        if out is None:
            out = np.empty(self.shapes[name], dtype=self.np_dtype)
        ptr, keep = self._arg(out)
        check(self.lib.uf_get_state(self._h, FIELDS[name], ptr))
        return out

    def init_state(self) -> None:
        check(self.lib.uf_init_state(self._h))

    def step(self, stats: bool = True):
        if not stats:
            check(self.lib.uf_step(self._h, None))
            return None
        s = StepStats()
        check(self.lib.uf_step(self._h, ctypes.byref(s)))
        return s

    def run(self, nsteps: int, stats: bool = True):
        s = StepStats()
        check(self.lib.uf_run(self._h, nsteps, ctypes.byref(s) if stats else None))
        return s if stats else None

    def objective(self, z_lo=1.0, z_hi=3.0, u_hi=4.0, u_lo=1.0) -> float:
        J = ctypes.c_double()
        check(self.lib.uf_objective(self._h, z_lo, z_hi, u_hi, u_lo, ctypes.byref(J)))
        return J.value

    def substep(self, name: str, inputs, cot=None):
        """One sub-step (uf_substep) on the given inputs (list of arrays in the
        order of SUBSTEPS[name]); with `cot` (cotangents of the outputs) its
        transpose instead.  Returns the outputs (or the input adjoints) as
        numpy arrays.  Test support: the grid's state is not kept."""
        which, ins, outs = SUBSTEPS[name]
        keep = [np.ascontiguousarray(a, dtype=self.np_dtype) for a in inputs]
        assert len(keep) == len(ins) and all(a.shape == self.shapes[n] for a, n in zip(keep, ins))
        vp = ctypes.c_void_p
        inp = (vp * len(keep))(*[a.ctypes.data for a in keep])
        if cot is None:
            res = [np.empty(self.shapes[n], dtype=self.np_dtype) for n in outs]
            cp = None
        else:
            ck = [np.ascontiguousarray(a, dtype=self.np_dtype) for a in cot]
            assert len(ck) == len(outs) and all(a.shape == self.shapes[n] for a, n in zip(ck, outs))
            keep += ck
            cp = (vp * len(ck))(*[a.ctypes.data for a in ck])
            res = [np.empty(self.shapes[n], dtype=self.np_dtype) for n in ins]
        outp = (vp * len(res))(*[a.ctypes.data for a in res])
        check(self.lib.uf_substep(self._h, which, 0 if cot is None else 1, inp, cp, outp))
        return res

    def objective_ex(self, objective) -> float:
        """Any objective of uf_objective_ex (see objective_desc)."""
        d, keep = objective_desc(objective)
        J = ctypes.c_double()
        check(self.lib.uf_objective_ex(self._h, ctypes.byref(d), ctypes.byref(J)))
        return J.value

    def divergence(self) -> float:
        out = ctypes.c_double()
        check(self.lib.uf_divergence(self._h, ctypes.byref(out)))
        return out.value

    def apply_poisson(self, x):
        xin, keep = _ptr(x, self.dtypes)
        y = np.empty(self.shapes["p"], dtype=self.np_dtype)
        yp, keep2 = _ptr(y, self.dtypes)
        check(self.lib.uf_apply_poisson(self._h, xin, yp))
        return y

    def poisson_solve(self, b):
        bp, keep = _ptr(b, self.dtypes)
        it, rel = ctypes.c_int(), ctypes.c_double()
        check(self.lib.uf_poisson_solve(self._h, bp, ctypes.byref(it), ctypes.byref(rel)))
        return it.value, rel.value

    def profile_step(self):
        """One eagerly launched, event-timed step; returns (stats, {label: dict})."""
        cap = 128
        arr = (KernelTime * cap)()
        n = ctypes.c_int()
        s = StepStats()
        check(self.lib.uf_profile_step(self._h, arr, cap, ctypes.byref(n), ctypes.byref(s)))
        out = {}
        for i in range(min(n.value, cap)):
            k = arr[i]
            out[k.name.decode()] = dict(launches=k.launches, total_ms=k.total_ms,
                                        bytes_per_launch=k.bytes_per_launch)
        return s, out

    # -- design gradients ------------------------------------------------
    def adjoint_run(self, nsteps: int, ckpt_every: int = 20, z_lo=1.0, z_hi=3.0, u_hi=4.0, u_lo=1.0, out=None,
                    objective=None):
        """Forward nsteps from the current state, objective, reverse sweep.
        Returns (J, dJ/dphi) -- dJ/dphi in ``out`` (a CUDA tensor or numpy
        array of the grid's precision) or a new numpy array; the grid ends at
        the final state.  The workspace is kept for the next call of the same
        size (release it with ``free_adjoint_workspace``)."""
        import torch
        nbytes = int(self.lib.uf_adjoint_workspace_bytes(self._h, nsteps, ckpt_every))
        if nbytes == 0:
            raise UFError(UF_ERR_ARG, "bad nsteps / ckpt_every")
        ws = getattr(self, "_adj_ws", None)
        if ws is None or ws.numel() < nbytes:
            self._adj_ws = None
            ws = self._adj_ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        if out is None:
            out = np.empty(self.shapes["phi"], dtype=self.np_dtype)
        optr, keep = self._arg(out)
        J = ctypes.c_double()
        if objective is None:
            check(self.lib.uf_adjoint_run(self._h, ctypes.c_void_p(ws.data_ptr()), nbytes, nsteps, ckpt_every, z_lo,
                                          z_hi, u_hi, u_lo, optr, ctypes.byref(J)))
        else:
            d, dkeep = objective_desc(objective)
            check(self.lib.uf_adjoint_run_ex(self._h, ctypes.c_void_p(ws.data_ptr()), nbytes, nsteps, ckpt_every,
                                             ctypes.byref(d), optr, ctypes.byref(J)))
        return J.value, out

    STATE5 = ("u", "v", "w", "k", "omega")

    def step_vjp(self, lam_out: dict, with_phi: bool = False):
        """Cotangents of one step's input state (and of phi) from the
        cotangent of its output state; dicts keyed u, v, w, k, omega."""
        import torch
        nbytes = int(self.lib.uf_adjoint_workspace_bytes(self._h, 1, 1))
        ws = getattr(self, "_adj_ws", None)
        if ws is None or ws.numel() < nbytes:
            self._adj_ws = None
            ws = self._adj_ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        keep = []
        outs = (ctypes.c_void_p * 5)()
        ins = (ctypes.c_void_p * 5)()
        lam_in = {}
        for q, n in enumerate(self.STATE5):
            ptr, k = self._arg(np.asarray(lam_out[n], dtype=self.np_dtype).reshape(self.shapes[n]))
            keep.append(k)
            outs[q] = ptr
            lam_in[n] = np.empty(self.shapes[n], dtype=self.np_dtype)
            ins[q] = lam_in[n].ctypes.data
        lphi = np.empty(self.shapes["phi"], dtype=self.np_dtype) if with_phi else None
        check(self.lib.uf_step_vjp(self._h, ctypes.c_void_p(ws.data_ptr()), nbytes, outs, ins,
                                   ctypes.c_void_p(lphi.ctypes.data) if with_phi else None))
        return (lam_in, lphi) if with_phi else lam_in

    def free_adjoint_workspace(self) -> None:
        self._adj_ws = None

    @staticmethod
    def _design_arrays(boxes, theta):
        b = np.ascontiguousarray(np.asarray(boxes, dtype=np.float64).reshape(-1, 4))
        t = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1, 3))
        if b.shape[0] != t.shape[0]:
            raise ValueError("boxes and theta describe different numbers of buildings")
        return b, t

    def design_to_phi(self, boxes, theta, width: float, set_porosity: bool = True, out=None):
        """Sigmoid box design -> porosity; sets the grid's porosity (default)
        or returns the field (in ``out`` when given: CUDA tensor or numpy)."""
        b, t = self._design_arrays(boxes, theta)
        dptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if set_porosity and out is None:
            check(self.lib.uf_design_to_phi(self._h, b.shape[0], dptr(b), dptr(t), width, None))
            return None
        if out is None:
            out = np.empty(self.shapes["phi"], dtype=self.np_dtype)
        optr, keep = self._arg(out)
        check(self.lib.uf_design_to_phi(self._h, b.shape[0], dptr(b), dptr(t), width, optr))
        return out

    def mesh_to_phi(self, tris, objects, sub: int = 4, set_porosity: bool = True, out=None):
        """Porosity of closed triangle meshes (uf_mesh_to_phi): tris (n, 3, 3)
        [m]; objects [(first triangle, count, inside porosity)].  Sets the
        grid's porosity (default) or returns the field (in ``out`` when
        given: CUDA tensor or numpy)."""
        t = np.ascontiguousarray(np.asarray(tris, dtype=np.float64).reshape(-1, 9))
        ob = list(objects)
        first = np.ascontiguousarray([int(o[0]) for o in ob], dtype=np.int32)
        count = np.ascontiguousarray([int(o[1]) for o in ob], dtype=np.int32)
        pin = np.ascontiguousarray([float(o[2]) for o in ob], dtype=np.float64)
        dptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        iptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        if set_porosity and out is None:
            check(self.lib.uf_mesh_to_phi(self._h, t.shape[0], dptr(t), len(ob), iptr(first), iptr(count), dptr(pin),
                                          sub, None))
            return None
        if out is None:
            out = np.empty(self.shapes["phi"], dtype=self.np_dtype)
        optr, keep = self._arg(out)
        check(self.lib.uf_mesh_to_phi(self._h, t.shape[0], dptr(t), len(ob), iptr(first), iptr(count), dptr(pin), sub,
                                      optr))
        return out

    def design_vjp(self, boxes, theta, width: float, dJ_dphi):
        b, t = self._design_arrays(boxes, theta)
        dptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        lp, keep = self._arg(dJ_dphi if _is_tensor(dJ_dphi) else np.asarray(dJ_dphi, dtype=self.np_dtype))
        g = np.zeros(3 * b.shape[0], dtype=np.float64)
        check(self.lib.uf_design_vjp(self._h, b.shape[0], dptr(b), dptr(t), width, lp, dptr(g)))
        return g

    # -- launch tuning ----------------------------------------------------
    def get_tuning(self):
        """(tuning dict with resolved values, number of MG levels)."""
        t = Tuning()
        n = ctypes.c_int()
        check(self.lib.uf_get_tuning(self._h, ctypes.byref(t), ctypes.byref(n)))
        return t.as_dict(), n.value

    def set_tuning(self, tail_level: int = 0, march_zc=None, advect_zc: int = 0, unfused: int = 0,
                   coarse_start: int = 0) -> None:
        """0 / None: automatic.  march_zc: per-level z planes per block;
        advect_zc: z planes per block of the fused advection; unfused: bit
        mask of fused kernels to run as their separate sub-step kernels
        (1: advection, 2: diffusion + drag + BCs + pressure right-hand side;
        True: all); coarse_start: first MG level of the one-launch cluster
        V-cycle (0 automatic = per-level launches, -1 per-level launches).
        Every choice gives the same values."""
        t = Tuning()
        t.tail_level = tail_level
        for l, z in enumerate(march_zc or []):
            t.march_zc[l] = z
        t.advect_zc = advect_zc
        t.unfused = UNFUSED_ALL if unfused is True else int(unfused)
        t.coarse_start = int(coarse_start)
        check(self.lib.uf_set_tuning(self._h, ctypes.byref(t)))

    def autotune(self, reps: int = 5):
        """Times the candidate tunings, keeps the fastest: (tuning, ms per solve)."""
        t = Tuning()
        ms = ctypes.c_double()
        check(self.lib.uf_autotune(self._h, reps, ctypes.byref(t), ctypes.byref(ms)))
        return t.as_dict(), ms.value

    def launch_counts(self):
        """(kernels per step outside the CG loop, kernels per CG iteration)."""
        fixed = ctypes.c_int()
        per = ctypes.c_int()
        check(self.lib.uf_launch_counts(self._h, ctypes.byref(fixed), ctypes.byref(per)))
        return fixed.value, per.value

    def launches_last_step(self) -> int:
        return int(self.lib.uf_last_step_launches(self._h))

    def put_fields(self, bufs: dict) -> None:
        """uf_set_fields: {name: array or tensor} in one call (dense layout)."""
        names = list(bufs)
        fl = (ctypes.c_int * len(names))(*[FIELDS[n] for n in names])
        ptrs = (ctypes.c_void_p * len(names))()
        keep = []
        for q, n in enumerate(names):
            p, k = self._arg(bufs[n])
            ptrs[q] = p
            keep.append(k)
        check(self.lib.uf_set_fields(self._h, len(names), fl, ptrs))
        self._keep_put = keep   # pinned buffers must outlive the enqueued copies

    def take_fields(self, outs: dict) -> dict:
        """uf_get_fields into {name: preallocated array or tensor}; one sync."""
        names = list(outs)
        fl = (ctypes.c_int * len(names))(*[FIELDS[n] for n in names])
        ptrs = (ctypes.c_void_p * len(names))()
        keep = []
        for q, n in enumerate(names):
            p, k = self._arg(outs[n])
            ptrs[q] = p
            keep.append(k)
        check(self.lib.uf_get_fields(self._h, len(names), fl, ptrs))
        return outs

    def state(self) -> dict:
        return {n: self.get_state(n) for n in ("u", "v", "w", "p", "k", "omega")}

    def set_fields(self, st: dict) -> None:
        for n, val in st.items():
            self.set_state(n, val if _is_tensor(val) else np.asarray(val, dtype=self.np_dtype))

    # -- checkpoint / resume ------------------------------------------------
    def save_checkpoint(self, out=None):
        """uf_save_state into a CUDA uint8 tensor (new, or `out`): the whole
        time-stepping state, pressure history included."""
        import torch
        n = int(self.lib.uf_state_bytes(self._h))
        buf = out if out is not None else torch.empty(n, dtype=torch.uint8, device="cuda")
        if not (buf.is_cuda and buf.dtype == torch.uint8 and buf.numel() >= n):
            raise TypeError(f"checkpoint buffer must be a CUDA uint8 tensor of >= {n} bytes")
        check(self.lib.uf_save_state(self._h, ctypes.c_void_p(buf.data_ptr()), buf.numel()))
        return buf

    def load_checkpoint(self, buf) -> None:
        """uf_load_state from a tensor written by save_checkpoint."""
        check(self.lib.uf_load_state(self._h, ctypes.c_void_p(buf.data_ptr()), buf.numel()))


class Batch:
    """Many grids advanced together by batched persistent launches under one
    CUDA graph (include/uf.h, "Batched execution").  `instances` is a list of
    dicts of grid parameters (nx, ny, nz and any uf_grid_desc field); all
    share `precision`.  batch.grids[i] is a Grid handle of instance i owned
    by the batch."""

    def __init__(self, instances, precision: str = "f32", stream=None):
        import torch
        self.lib = load()
        n = len(instances)
        descs = (GridDesc * n)()
        for i, p in enumerate(instances):
            descs[i] = default_desc(precision=precision, **p)
        self.descs = descs
        nbytes = int(self.lib.uf_batch_workspace_bytes(n, descs))
        if nbytes == 0:
            raise UFError(UF_ERR_ARG, last_error())
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = ctypes.c_void_p()
        check(self.lib.uf_batch_create(n, descs, ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                       ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h
        self.n = n
        self.grids = []
        for i in range(n):
            gh = ctypes.c_void_p()
            check(self.lib.uf_batch_grid(h, i, ctypes.byref(gh)))
            self.grids.append(Grid._borrowed(self, gh, descs[i], self.stream))

    def run(self, nsteps: int, stats: bool = True):
        """nsteps batched steps; per-instance StepStats after the last one."""
        if not stats:
            check(self.lib.uf_batch_run(self._h, nsteps, None))
            return None
        arr = (StepStats * self.n)()
        check(self.lib.uf_batch_run(self._h, nsteps, arr))
        return list(arr)

    def launch_counts(self):
        fixed = ctypes.c_int()
        per = ctypes.c_int()
        check(self.lib.uf_batch_launch_counts(self._h, ctypes.byref(fixed), ctypes.byref(per)))
        return fixed.value, per.value

    def profile_step(self, capacity: int = 96):
        """One eager batched step with per-launch CUDA events:
        {kernel name: dict(launches, total_ms, bytes_per_launch)}."""
        arr = (KernelTime * capacity)()
        n = ctypes.c_int()
        check(self.lib.uf_batch_profile_step(self._h, arr, capacity, ctypes.byref(n)))
        out = {}
        for i in range(min(n.value, capacity)):
            k = arr[i]
            out[k.name.decode()] = dict(launches=k.launches, total_ms=k.total_ms, bytes_per_launch=k.bytes_per_launch)
        return out

    def autotune(self, reps: int = 5) -> int:
        """Per size class autotuning; returns the number of classes."""
        c = ctypes.c_int()
        check(self.lib.uf_batch_autotune(self._h, reps, ctypes.byref(c)))
        return c.value

    @property
    def cells(self) -> int:
        return sum(d.nx * d.ny * d.nz for d in self.descs)

    def close(self):
        if getattr(self, "_h", None):
            for g in self.grids:
                g._h = None
            self.lib.uf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_functions():
    import torch

    class ComfortObjective(torch.autograd.Function):
        """J(phi): the pedestrian comfort objective after `nsteps` steps from a
        fixed initial state x0, as a function of the porosity field phi.
        forward runs the steps (uf_run) and the objective (uf_objective);
        backward re-runs the checkpointed forward and the discrete adjoint
        (uf_adjoint_run) and returns dJ/dphi on the device."""

        @staticmethod
        def forward(ctx, phi, grid, x0, nsteps, ckpt_every, objective):
            phi = phi.detach().contiguous()
            grid.set_porosity(phi)
            grid.set_fields(x0)
            grid.run(nsteps, stats=False)
            J = grid.objective_ex(objective)
            ctx.save_for_backward(phi)
            ctx.grid, ctx.x0, ctx.nsteps, ctx.ckpt_every, ctx.objective = grid, x0, nsteps, ckpt_every, objective
            return torch.tensor(J, dtype=torch.float64, device=phi.device)

        @staticmethod
        def backward(ctx, gJ):
            (phi,) = ctx.saved_tensors
            g = ctx.grid
            g.set_porosity(phi)
            g.set_fields(ctx.x0)
            dphi = torch.empty_like(phi)
            g.adjoint_run(ctx.nsteps, ctx.ckpt_every, out=dphi, objective=ctx.objective)
            return gJ.to(dphi.dtype) * dphi, None, None, None, None, None

    class DesignPorosity(torch.autograd.Function):
        """phi(theta): porosity of the logistic-box design (uf_design_to_phi);
        backward is uf_design_vjp."""

        @staticmethod
        def forward(ctx, theta, grid, boxes, width):
            th = theta.detach().cpu().numpy().astype(np.float64)
            phi = torch.empty(grid.shapes["phi"], dtype=grid.torch_dtype, device="cuda")
            grid.design_to_phi(boxes, th, width, out=phi)
            ctx.grid, ctx.boxes, ctx.width, ctx.th = grid, boxes, width, th
            ctx.like = (theta.dtype, theta.device)
            return phi

        @staticmethod
        def backward(ctx, gphi):
            g = ctx.grid.design_vjp(ctx.boxes, ctx.th, ctx.width, gphi.contiguous().to(ctx.grid.torch_dtype))
            dtype, device = ctx.like
            return torch.as_tensor(g).reshape(ctx.th.shape).to(dtype=dtype, device=device), None, None, None

    return ComfortObjective, DesignPorosity


_functions = None


def _fns():
    global _functions
    if _functions is None:
        _functions = _make_functions()
    return _functions


def comfort_objective(phi, grid: "Grid", x0: dict, nsteps: int, ckpt_every: int = 20, band=(1.0, 3.0, 4.0, 1.0),
                      objective=None):
    """Differentiable J(phi) (torch.autograd): see ComfortObjective.  phi is a
    CUDA tensor of the grid's precision and shape (nz, ny, nx); the objective
    is the comfort band `band` unless `objective` names another one (see
    objective_desc)."""
    if objective is None:
        objective = {"kind": "comfort", "band": tuple(band)}
    return _fns()[0].apply(phi, grid, x0, nsteps, ckpt_every, objective)


def optimize_design(grid: "Grid", boxes, theta0, x0: dict, nsteps: int, iterations: int, step_size: float,
                    width: float, objective=None, ckpt_every: int = 20, lower=None, upper=None):
    """Gradient descent on the design parameters (Sec. 4, "Automatic Design
    Optimization"): theta <- clip(theta - step_size dL/dtheta, lower, upper),
    the gradient from the discrete adjoint through design_porosity and
    comfort_objective instead of the N + 1 forward simulations of the paper's
    forward differences.  The descent sign is the reading of the paper's
    update rule.  Returns (theta, history of (L, theta, gradient)) with the
    objective of every evaluated design."""
    import torch
    theta = torch.tensor(np.asarray(theta0, dtype=np.float64).reshape(-1, 3), requires_grad=True)
    lo = None if lower is None else torch.as_tensor(np.asarray(lower, dtype=np.float64).reshape(-1, 3))
    hi = None if upper is None else torch.as_tensor(np.asarray(upper, dtype=np.float64).reshape(-1, 3))
    history = []
    for _ in range(iterations):
        phi = design_porosity(theta, grid, boxes, width)
        L = comfort_objective(phi, grid, x0, nsteps, ckpt_every, objective=objective)
        (g,) = torch.autograd.grad(L, theta)
        history.append((L.item(), theta.detach().clone().numpy(), g.numpy().copy()))
        with torch.no_grad():
            theta -= step_size * g
            if lo is not None:
                theta.copy_(torch.maximum(theta, lo))
            if hi is not None:
                theta.copy_(torch.minimum(theta, hi))
    return theta.detach().numpy(), history


def wind_robustness(params: dict, phi, winds, nsteps: int, objective=None, precision: str = "f32"):
    """The objective of one design under several wind directions (the +-10
    degree re-runs of Sec. 6), all directions advanced together as one batch
    (uf_batch_*): params are the grid parameters (nx, ny, nz, ...) without
    wind_dir_deg, phi the design's porosity.  Returns [L per direction]."""
    insts = [dict(params, wind_dir_deg=float(d)) for d in winds]
    b = Batch(insts, precision=precision)
    ph = np.asarray(phi, dtype=b.grids[0].np_dtype)
    for g in b.grids:
        g.set_porosity(ph)
        g.init_state()
    b.run(nsteps, stats=False)
    out = [g.objective_ex(objective) for g in b.grids]
    b.close()
    return out


def design_porosity(theta, grid: "Grid", boxes, width: float):
    """Differentiable phi(theta) (torch.autograd): theta holds (H, dx, dy) per
    box, as a float64 tensor of shape (nbox, 3) or (3 * nbox,)."""
    return _fns()[1].apply(theta, grid, boxes, width)
