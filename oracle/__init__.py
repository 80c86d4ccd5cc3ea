"""FP64 CPU oracle of the UrbanFlow RANS step (arXiv 2204.01117, Sec. 3).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_2204_01117_gb300``) never imports it, and it imports nothing from the
product.

The arithmetic lives in ``oracle.cpp`` (plain loops, FP64).  This module only
compiles it with gcc and marshals arguments through ctypes.

Parameter defaults follow the paper: Table 1 for the k-omega coefficients;
the Sec. 3 footnote for the porosity drag (a = 0.62, b = 2.5, e = 1e-10);
Appendix A.2 for C_d = 1.0.  The values the paper leaves open use the
readings the test-suite documents: rho = 1.225, nu = 1.5e-5, I = 0.1,
L = 10 m, CFL 0.5, k >= 1e-10 and omega >= 1e-6.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

FIELDS = {"u": 0, "v": 1, "w": 2, "p": 3, "k": 4, "omega": 5, "phi": 6, "nut": 7, "c": 8}
SIDE_NAMES = ["inflow", "outflow", "slip", "noslip"]


class OrcDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("h", ctypes.c_double),
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
        ("cg_tol", ctypes.c_double), ("cg_max_iter", ctypes.c_int),
    ]


class OrcStats(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double), ("cg_iters", ctypes.c_int),
        ("cg_rel_residual", ctypes.c_double),
        ("div_before", ctypes.c_double), ("div_after", ctypes.c_double),
    ]


# Paper constants (Table 1; Sec. 3 footnote; App. A.2) and the stated readings.
DEFAULTS = dict(
    h=2.0, wind_dir_deg=0.0, u_ref=5.0, z_ref=10.0, z0=0.5, inflow_loglaw=0,
    ground_noslip=1, rho=1.225, nu=1.5e-5, Cd=1.0, a=0.62, b=2.5, e=1e-10,
    I=0.1, L=10.0, C_mu=0.09, alpha=0.52, beta=0.0708, sigma=0.5,
    sigma_star=0.6, C_lim=7.0 / 8.0, cfl=0.5, fixed_dt=0.0, k_min=1e-10,
    omega_min=1e-6, cg_tol=1e-13, cg_max_iter=100000,
)


def build(force: bool = False) -> str:
    """Compile oracle.cpp into _build/liboracle.so (gcc, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    lib.orc_create.restype = vp
    lib.orc_create.argtypes = [ctypes.POINTER(OrcDesc)]
    lib.orc_destroy.argtypes = [vp]
    for name in ("orc_inlet_k", "orc_inlet_omega", "orc_compute_dt", "orc_get_dt",
                 "orc_divergence"):
        getattr(lib, name).restype = ctypes.c_double
        getattr(lib, name).argtypes = [vp]
    lib.orc_profile.restype = ctypes.c_double
    lib.orc_profile.argtypes = [vp, ip]
    lib.orc_drag_coeff.restype = ctypes.c_double
    lib.orc_drag_coeff.argtypes = [vp, ctypes.c_double]
    lib.orc_side.restype = ip
    lib.orc_side.argtypes = [vp, ip]
    lib.orc_field_size.restype = ctypes.c_long
    lib.orc_field_size.argtypes = [vp, ip]
    lib.orc_get.argtypes = [vp, ip, dp]
    lib.orc_set.argtypes = [vp, ip, dp]
    lib.orc_set_dt.argtypes = [vp, ctypes.c_double]
    for name in ("orc_eddy_viscosity", "orc_advect", "orc_apply_bc", "orc_diffuse", "orc_drag",
                 "orc_project", "orc_turbulence", "orc_init"):
        getattr(lib, name).argtypes = [vp]
    lib.orc_pressure_rhs.argtypes = [vp, dp]
    lib.orc_apply_A.argtypes = [vp, dp, dp]
    lib.orc_cg.restype = ip
    lib.orc_cg.argtypes = [vp, dp, dp, ctypes.c_double, ip, dp]
    lib.orc_pressure_project.restype = ip
    lib.orc_pressure_project.argtypes = [vp]
    lib.orc_objective.restype = ctypes.c_double
    lib.orc_objective.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double]
    lib.orc_step.restype = ip
    lib.orc_step.argtypes = [vp, ctypes.POINTER(OrcStats)]
    lib.orc_run.restype = ip
    lib.orc_run.argtypes = [vp, ip, ctypes.POINTER(OrcStats)]
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """One FP64 grid instance of the oracle solver."""

    def __init__(self, nx: int, ny: int, nz: int, **params):
        self.lib = _load()
        p = dict(DEFAULTS)
        unknown = set(params) - set(p)
        if unknown:
            raise TypeError(f"unknown oracle parameters: {sorted(unknown)}")
        p.update(params)
        self.params = p
        self.nx, self.ny, self.nz = nx, ny, nz
        d = OrcDesc(nx=nx, ny=ny, nz=nz, **p)
        self._h = self.lib.orc_create(ctypes.byref(d))
        if not self._h:
            raise ValueError("oracle rejected the grid description")
        self.shapes = {
            "u": (nz, ny, nx + 1), "v": (nz, ny + 1, nx), "w": (nz + 1, ny, nx),
            "p": (nz, ny, nx), "k": (nz, ny, nx), "omega": (nz, ny, nx),
            "phi": (nz, ny, nx), "nut": (nz, ny, nx), "c": (nz, ny, nx),
        }

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self.lib.orc_destroy(h)
            self._h = None

    # -- state ------------------------------------------------------------
    def get(self, name: str) -> np.ndarray:
        out = np.empty(self.shapes[name], dtype=np.float64)
        if self.lib.orc_get(self._h, FIELDS[name], _dptr(out)) != 0:
            raise KeyError(name)
        return out

    def set(self, name: str, value) -> None:
        arr = np.ascontiguousarray(np.broadcast_to(np.asarray(value, dtype=np.float64),
                                                   self.shapes[name]))
        if self.lib.orc_set(self._h, FIELDS[name], _dptr(arr)) != 0:
            raise KeyError(name)

    def state(self) -> dict:
        return {n: self.get(n) for n in ("u", "v", "w", "p", "k", "omega")}

    def set_state(self, st: dict) -> None:
        for n, val in st.items():
            self.set(n, val)

    @property
    def dt(self) -> float:
        return self.lib.orc_get_dt(self._h)

    @dt.setter
    def dt(self, value: float) -> None:
        self.lib.orc_set_dt(self._h, float(value))

    def side(self, q: int) -> str:
        return SIDE_NAMES[self.lib.orc_side(self._h, q)]

    def profile(self, k: int) -> float:
        return self.lib.orc_profile(self._h, k)

    @property
    def inlet_k(self) -> float:
        return self.lib.orc_inlet_k(self._h)

    @property
    def inlet_omega(self) -> float:
        return self.lib.orc_inlet_omega(self._h)

    def drag_coeff(self, phi: float) -> float:
        return self.lib.orc_drag_coeff(self._h, float(phi))

    # -- sub-steps ----------------------------------------------------------
    def compute_dt(self) -> float:
        return self.lib.orc_compute_dt(self._h)

    def eddy_viscosity(self) -> np.ndarray:
        self.lib.orc_eddy_viscosity(self._h)
        return self.get("nut")

    def advect(self):
        self.lib.orc_advect(self._h)

    def apply_bc(self):
        self.lib.orc_apply_bc(self._h)

    def diffuse(self):
        self.lib.orc_diffuse(self._h)

    def drag(self):
        self.lib.orc_drag(self._h)

    def pressure_rhs(self) -> np.ndarray:
        b = np.empty(self.shapes["p"])
        self.lib.orc_pressure_rhs(self._h, _dptr(b))
        return b

    def apply_A(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.shapes["p"])
        y = np.empty_like(x)
        self.lib.orc_apply_A(self._h, _dptr(x), _dptr(y))
        return y

    def cg(self, b: np.ndarray, x0=None, tol: float = 1e-13, max_iter: int = 100000):
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(self.shapes["p"])
        x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64).reshape(b.shape)
        rel = ctypes.c_double(0.0)
        it = self.lib.orc_cg(self._h, _dptr(b), _dptr(x), tol, max_iter, ctypes.byref(rel))
        return x, it, rel.value

    def pressure_project(self) -> int:
        return self.lib.orc_pressure_project(self._h)

    def project(self):
        self.lib.orc_project(self._h)

    def turbulence(self):
        self.lib.orc_turbulence(self._h)

    def divergence(self) -> float:
        return self.lib.orc_divergence(self._h)

    def objective(self, z_lo=1.0, z_hi=3.0, u_hi=4.0, u_lo=1.0) -> float:
        return self.lib.orc_objective(self._h, z_lo, z_hi, u_hi, u_lo)

    # -- whole steps ----------------------------------------------------------
    def init(self):
        self.lib.orc_init(self._h)

    def step(self) -> OrcStats:
        st = OrcStats()
        self.lib.orc_step(self._h, ctypes.byref(st))
        return st

    def run(self, nsteps: int) -> OrcStats:
        st = OrcStats()
        self.lib.orc_run(self._h, nsteps, ctypes.byref(st))
        return st


def cell_speed(u, v, w) -> np.ndarray:
    """|u_c| at every cell centre from the face averages of the three
    staggered components (arrays shaped (nz, ny, nx+1), (nz, ny+1, nx),
    (nz+1, ny, nx))."""
    uc = 0.5 * (u[:, :, :-1] + u[:, :, 1:])
    vc = 0.5 * (v[:, :-1, :] + v[:, 1:, :])
    wc = 0.5 * (w[:-1, :, :] + w[1:, :, :])
    return np.sqrt(uc * uc + vc * vc + wc * wc)


def region_objective(u, v, w, h: float, regions, u_t: float):
    """Region-average objective of Sec. 6 ("Avoiding Heat Pockets in Early
    Design Stages"): L = sum_i (ubar_i - u_t)^2 with ubar_i the mean cell
    speed over the cells whose centres lie in box i = (x0, x1, y0, y1, z0,
    z1) [m].  Returns (L, [ubar_i])."""
    speed = cell_speed(u, v, w)
    nz, ny, nx = speed.shape
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * h, (np.arange(ny) + 0.5) * h, (np.arange(nx) + 0.5) * h,
                          indexing="ij")
    means = []
    for x0, x1, y0, y1, z0, z1 in np.asarray(regions, dtype=np.float64).reshape(-1, 6):
        sel = (x >= x0) & (x <= x1) & (y >= y0) & (y <= y1) & (z >= z0) & (z <= z1)
        if not sel.any():
            raise ValueError("region holds no cell centre")
        means.append(float(speed[sel].mean()))
    return float(sum((m - u_t) ** 2 for m in means)), means


def design_to_phi(nx: int, ny: int, nz: int, h: float, boxes, theta, width: float) -> np.ndarray:
    """Porosity of the parametric design, in FP64 numpy: the product over
    boxes of (1 - chi), chi the product of five logistic ramps at the cell
    centre -- across the two x faces and the two y faces of the shifted box
    footprint and below its height (the smoothed cut-cell idea of Sec. 3,
    "Urban model resolving")."""
    boxes = np.asarray(boxes, dtype=np.float64).reshape(-1, 4)
    theta = np.asarray(theta, dtype=np.float64).reshape(-1, 3)
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * h, (np.arange(ny) + 0.5) * h, (np.arange(nx) + 0.5) * h,
                          indexing="ij")
    s = lambda t: 1.0 / (1.0 + np.exp(-t))
    phi = np.ones((nz, ny, nx))
    for (xa, xb, ya, yb), (H, dx, dy) in zip(boxes, theta):
        chi = (s((x - (xa + dx)) / width) * s(((xb + dx) - x) / width) * s((y - (ya + dy)) / width)
               * s(((yb + dy) - y) / width) * s((H - z) / width))
        phi *= 1.0 - chi
    return phi
