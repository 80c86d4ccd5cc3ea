"""Seeded synthetic urban layouts (porosity fields) for the RANS step.

This module only generates inputs.  It holds none of the solver's arithmetic
and imports nothing from the rest of the package, so the CUDA path and the
test oracle can both be fed from it.

Porosity follows the paper's unified model: phi = 1 in air, phi = 0 inside a
solid building, phi in (0, 1) inside a porous tree canopy (Sec. 3 footnote;
App. A.2), and cut cells get the fraction of a uniform 4x4x4 sub-sample that
lies outside the objects (Sec. 3, "Urban model resolving").  Where objects
overlap, a sub-sample takes the smallest porosity of the objects that hold it.

Random draws come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the state advances by
0x9E3779B97F4A7C15 and each output is the state passed through the two
xor-shift-multiply rounds of that paper.  A uniform double in [0, 1) takes the
top 53 bits of one output.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream; ``next_u64`` returns successive 64-bit outputs."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on [lo, hi] inclusive (multiply-shift on 32 high bits)."""
        span = hi - lo + 1
        return lo + (((self.next_u64() >> 32) * span) >> 32)


@dataclass
class Box:
    x0: float
    x1: float
    y0: float
    y1: float
    z0: float
    z1: float
    phi: float = 0.0


@dataclass
class Ellipsoid:
    cx: float
    cy: float
    cz: float
    rx: float
    ry: float
    rz: float
    phi: float = 0.5


@dataclass
class Scenario:
    """Grid, inflow and porosity of one synthetic run."""
    nx: int
    ny: int
    nz: int
    h: float
    phi: np.ndarray                     # (nz, ny, nx) float64
    wind_dir_deg: float = 0.0
    u_ref: float = 5.0
    z_ref: float = 10.0
    z0: float = 0.5
    inflow_loglaw: bool = False
    ground_noslip: bool = True
    steps: int = 100
    name: str = ""
    objects: list = field(default_factory=list)

    def params(self) -> dict:
        """Physical parameters shared by every solver that runs this input."""
        return dict(h=self.h, wind_dir_deg=self.wind_dir_deg, u_ref=self.u_ref,
                    z_ref=self.z_ref, z0=self.z0, inflow_loglaw=int(self.inflow_loglaw),
                    ground_noslip=int(self.ground_noslip))

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


def rasterize(nx: int, ny: int, nz: int, h: float, objects, sub: int = 4) -> np.ndarray:
    """Cell porosity from objects by sub-sampling each cell sub^3 times."""
    phi = np.ones((nz, ny, nx), dtype=np.float64)
    off = (np.arange(sub) + 0.5) / sub
    xs = ((np.arange(nx)[:, None] + off[None, :]) * h).reshape(-1)   # nx*sub
    ys = ((np.arange(ny)[:, None] + off[None, :]) * h).reshape(-1)
    for k in range(nz):
        zs = (k + off) * h                                            # sub
        touching = []
        for ob in objects:
            if isinstance(ob, Box):
                lo, hi = ob.z0, ob.z1
            else:
                lo, hi = ob.cz - ob.rz, ob.cz + ob.rz
            if hi > k * h and lo < (k + 1) * h:
                touching.append(ob)
        if not touching:
            continue
        pts = np.ones((sub, ny * sub, nx * sub), dtype=np.float64)
        for ob in touching:
            if isinstance(ob, Box):
                ix = np.nonzero((xs >= ob.x0) & (xs < ob.x1))[0]
                iy = np.nonzero((ys >= ob.y0) & (ys < ob.y1))[0]
                iz = np.nonzero((zs >= ob.z0) & (zs < ob.z1))[0]
                if len(ix) == 0 or len(iy) == 0 or len(iz) == 0:
                    continue
                sl = pts[iz[0]:iz[-1] + 1, iy[0]:iy[-1] + 1, ix[0]:ix[-1] + 1]
                np.minimum(sl, ob.phi, out=sl)
            else:
                ix = np.nonzero(np.abs(xs - ob.cx) < ob.rx)[0]
                iy = np.nonzero(np.abs(ys - ob.cy) < ob.ry)[0]
                if len(ix) == 0 or len(iy) == 0:
                    continue
                X = xs[ix[0]:ix[-1] + 1][None, None, :]
                Y = ys[iy[0]:iy[-1] + 1][None, :, None]
                Z = zs[:, None, None]
                inside = (((X - ob.cx) / ob.rx) ** 2 + ((Y - ob.cy) / ob.ry) ** 2
                          + ((Z - ob.cz) / ob.rz) ** 2) < 1.0
                sl = pts[:, iy[0]:iy[-1] + 1, ix[0]:ix[-1] + 1]
                sl[inside] = np.minimum(sl[inside], ob.phi)
        phi[k] = pts.reshape(sub, ny, sub, nx, sub).mean(axis=(0, 2, 4))
    return phi


def single_box(nx=64, ny=32, nz=16, h=2.0, size=(20.0, 10.0, 12.0), u_ref=5.0,
               steps=100) -> Scenario:
    """One solid box (porosity 0) centred in x and y, standing on the ground;
    uniform inflow on x-, zero-gradient outflow on x+, slip top and sides,
    no-slip ground."""
    lx, ly = nx * h, ny * h
    b = Box(lx / 2 - size[0] / 2, lx / 2 + size[0] / 2, ly / 2 - size[1] / 2,
            ly / 2 + size[1] / 2, 0.0, size[2], 0.0)
    phi = rasterize(nx, ny, nz, h, [b])
    return Scenario(nx, ny, nz, h, phi, wind_dir_deg=0.0, u_ref=u_ref, inflow_loglaw=False,
                    ground_noslip=True, steps=steps, name=f"single_box_{nx}x{ny}x{nz}",
                    objects=[b])


def urban_block(nx=256, ny=256, nz=64, h=2.0, n_boxes=40, n_trees=60, seed=0,
                footprint=(10.0, 40.0), height=(10.0, 60.0), radius=(3.0, 8.0),
                tree_phi=(0.3, 0.8), trunk=(2.0, 5.0), u_ref=3.0, wind_dir_deg=0.0,
                margin=0.10, steps=500) -> Scenario:
    """Seeded urban block: axis-aligned solid boxes plus porous ellipsoidal
    canopies, log-law inflow.

    Draw order per box: x-extent, y-extent, height, centre x, centre y.
    Per canopy: radius, porosity, trunk height, centre x, centre y.
    Objects keep a margin (fraction of the domain length) from the four
    lateral sides, so inflow and outflow faces stay clear.
    """
    rng = SplitMix64(seed)
    lx, ly, lz = nx * h, ny * h, nz * h
    mx, my = margin * lx, margin * ly
    objects = []
    for _ in range(n_boxes):
        sx = rng.uniform(*footprint)
        sy = rng.uniform(*footprint)
        hz = min(rng.uniform(*height), lz - h)
        cx = rng.uniform(mx + sx / 2, lx - mx - sx / 2)
        cy = rng.uniform(my + sy / 2, ly - my - sy / 2)
        objects.append(Box(cx - sx / 2, cx + sx / 2, cy - sy / 2, cy + sy / 2, 0.0, hz, 0.0))
    for _ in range(n_trees):
        r = rng.uniform(*radius)
        ph = rng.uniform(*tree_phi)
        tz = rng.uniform(*trunk)
        cx = rng.uniform(mx + r, lx - mx - r)
        cy = rng.uniform(my + r, ly - my - r)
        objects.append(Ellipsoid(cx, cy, 0.75 * r + tz, r, r, 0.75 * r, ph))
    phi = rasterize(nx, ny, nz, h, objects)
    return Scenario(nx, ny, nz, h, phi, wind_dir_deg=wind_dir_deg, u_ref=u_ref,
                    z_ref=10.0, z0=0.5, inflow_loglaw=True, ground_noslip=True, steps=steps,
                    name=f"urban_{nx}x{ny}x{nz}_s{seed}", objects=objects)


def scaled_urban_block(nx, ny, nz, h=2.0, seed=0, wind_dir_deg=0.0, u_ref=3.0, steps=300,
                       ref_cells_xy=256 * 256, ref_boxes=40, ref_trees=60) -> Scenario:
    """Urban block whose object counts scale with the footprint area."""
    area = nx * ny / ref_cells_xy
    nb = max(1, int(round(ref_boxes * area)))
    nt = max(1, int(round(ref_trees * area)))
    return urban_block(nx, ny, nz, h, n_boxes=nb, n_trees=nt, seed=seed, u_ref=u_ref,
                       wind_dir_deg=wind_dir_deg, steps=steps)


@dataclass
class DesignScenario(Scenario):
    """A parametric design: base footprints and the design parameters of
    each building.  The porosity comes from the method's design map, not
    from this module (``phi`` holds open air)."""
    boxes: np.ndarray = None            # (nbox, 4): x_a, x_b, y_a, y_b of each base footprint [m]
    theta: np.ndarray = None            # (nbox, 3): height H, x shift, y shift [m]
    width: float = 2.0                  # logistic ramp width [m]
    fixed_dt: float = 0.2               # [s]
    ckpt_every: int = 20
    regions: np.ndarray = None          # (nreg, 6): x0, x1, y0, y1, z0, z1 of each target region [m]
    u_t: float = 0.55                   # target mean wind speed of a region [m/s]

    def params(self) -> dict:
        d = super().params()
        d["fixed_dt"] = self.fixed_dt
        return d


def design_lattice(nx=128, ny=128, nz=48, h=2.0, cols=4, rows=3, footprint=20.0, height=(20.0, 40.0),
                   seed=0, u_ref=3.0, fixed_dt=0.2, steps=200, ckpt_every=20) -> DesignScenario:
    """cols x rows parametric buildings of square footprint on an even
    lattice (centre of column c at (c + 1)/(cols + 1) of the domain length,
    likewise for rows), heights drawn uniformly, shifts zero; log-law
    inflow along +x; one-cell logistic ramps; the fixed time step of 0.2 s
    used for the design runs of Sec. 6 ("Avoiding Heat Pockets in Early
    Design Stages").  Draw order: one height per building, row by row.
    Target regions of the region-average objective (six in Sec. 6): square
    frames of one footprint side at pedestrian level, z in [0, 3] m, centred
    between four neighbouring buildings, for the first two row gaps."""
    rng = SplitMix64(seed)
    lx, ly = nx * h, ny * h
    boxes, theta = [], []
    for r in range(rows):
        for c in range(cols):
            cx, cy = lx * (c + 1) / (cols + 1), ly * (r + 1) / (rows + 1)
            boxes.append((cx - footprint / 2, cx + footprint / 2, cy - footprint / 2, cy + footprint / 2))
            theta.append((rng.uniform(*height), 0.0, 0.0))
    regions = []
    for r in range(min(rows - 1, 2)):
        for c in range(cols - 1):
            gx, gy = lx * (c + 1.5) / (cols + 1), ly * (r + 1.5) / (rows + 1)
            regions.append((gx - footprint / 2, gx + footprint / 2, gy - footprint / 2, gy + footprint / 2, 0.0, 3.0))
    return DesignScenario(nx, ny, nz, h, np.ones((nz, ny, nx)), wind_dir_deg=0.0, u_ref=u_ref, z_ref=10.0,
                          z0=0.5, inflow_loglaw=True, ground_noslip=True, steps=steps,
                          name=f"design_{nx}x{ny}x{nz}_{cols * rows}b_s{seed}",
                          boxes=np.array(boxes), theta=np.array(theta), width=h, fixed_dt=fixed_dt,
                          ckpt_every=ckpt_every, regions=np.array(regions).reshape(-1, 6))


@dataclass
class CylinderScenario(Scenario):
    """Flow past a circular cylinder in a quasi-2D channel (one cell in z,
    slip in z), for the vortex-shedding validation."""
    D: float = 0.046                    # cylinder diameter [m]
    centre: tuple = (0.512, 0.3)        # cylinder axis (x, y) [m]
    fixed_dt: float = 1e-4              # [s]
    I: float = 1e-3                     # inlet turbulence intensity
    L: float = 0.046                    # inlet turbulence length scale [m]

    def params(self) -> dict:
        d = super().params()
        d.update(fixed_dt=self.fixed_dt, I=self.I, L=self.L)
        return d


def karman_cylinder(U: float, nx=512, ny=768, h=2e-3, D=0.046, centre_y=0.3, dt=1e-4, I=1e-3,
                    L=None) -> CylinderScenario:
    """The vortex-street benchmark of the supplement's solver validation:
    512 x 768 cells of 2 mm, a cylinder of 0.046 m diameter, inflow U through
    the y- side (wind direction +y), outflow through y+, slip walls on the x
    sides, dt = 1e-4 s (or the dt given).  The cylinder is solid (phi = 0) in
    every cell whose centre lies inside it, open elsewhere; it sits on the
    channel axis, centre_y from the inlet.  The inlet turbulence is nearly
    laminar (I = 1e-3, length scale D): the supplement states none."""
    xc, yc = nx * h / 2, centre_y
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    X, Y = np.meshgrid(x, y)
    phi = ((X - xc) ** 2 + (Y - yc) ** 2 > (D / 2) ** 2).astype(np.float64)[None]
    return CylinderScenario(nx, ny, 1, h, phi, wind_dir_deg=90.0, u_ref=U, inflow_loglaw=False,
                            ground_noslip=False, name=f"karman_{nx}x{ny}_U{U:g}", D=D, centre=(xc, yc),
                            fixed_dt=dt, I=I, L=D if L is None else L)


# ------------------------------------------------------------ meshes ----
# Closed triangle meshes (n, 3, 3) [m] for the mesh resolver; every
# triangle wound counter-clockwise seen from outside.

def box_mesh(x0, x1, y0, y1, z0, z1) -> np.ndarray:
    """The 12 triangles of an axis-aligned box."""
    c = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]], dtype=np.float64)
    quads = [(0, 3, 2, 1), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7)]
    return np.array([[c[a], c[b], c[d]] for a, b, cc, d in quads for (b, d) in ((b, cc), (cc, d))])


def prism_mesh(cx, cy, radius, sides, angle, z0, z1) -> np.ndarray:
    """A building: the convex regular polygon of `sides` corners (first at
    `angle`) around (cx, cy) extruded from z0 to z1."""
    t = angle + 2 * np.pi * np.arange(sides) / sides
    ring = np.stack([cx + radius * np.cos(t), cy + radius * np.sin(t)], axis=1)
    tris = []
    for a in range(sides):
        b = (a + 1) % sides
        p0, p1 = ring[a], ring[b]
        tris.append([[cx, cy, z0], [p1[0], p1[1], z0], [p0[0], p0[1], z0]])     # floor
        tris.append([[cx, cy, z1], [p0[0], p0[1], z1], [p1[0], p1[1], z1]])     # roof
        tris.append([[p0[0], p0[1], z0], [p1[0], p1[1], z0], [p1[0], p1[1], z1]])
        tris.append([[p0[0], p0[1], z0], [p1[0], p1[1], z1], [p0[0], p0[1], z1]])
    return np.array(tris, dtype=np.float64)


def icosphere_mesh(cx, cy, cz, r, levels=1, scale=(1.0, 1.0, 1.0)) -> np.ndarray:
    """A canopy: the icosahedron subdivided `levels` times, projected onto
    the sphere of radius r and stretched by `scale` per axis."""
    g = (1 + 5 ** 0.5) / 2
    v = [(-1, g, 0), (1, g, 0), (-1, -g, 0), (1, -g, 0), (0, -1, g), (0, 1, g), (0, -1, -g), (0, 1, -g),
         (g, 0, -1), (g, 0, 1), (-g, 0, -1), (-g, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    tris = np.array([[v[a], v[b], v[c]] for a, b, c in f], dtype=np.float64)
    for _ in range(levels):
        out = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            out += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        tris = np.array(out)
    tris = tris / np.linalg.norm(tris, axis=2, keepdims=True)
    return tris * r * np.asarray(scale) + np.array([cx, cy, cz])


def mesh_city(nx=48, ny=40, nz=16, h=2.0, n_buildings=6, n_trees=4, seed=0):
    """Seeded closed meshes for the mesh resolver: prism buildings (4-8
    sides, radius U[4, 10] m, height U[8, 0.8 lz] m, porosity 0) and
    ellipsoidal canopies (radius U[3, 6] m, axes (r, r, 0.75 r), centre
    height U[4, 10] m, porosity U[0.3, 0.8]), placed uniformly inside a 10 %
    lateral margin; overlaps allowed.  Returns (triangles (n, 3, 3),
    objects [(first, count, inside porosity)]).  Draw order per building:
    x, y, radius, sides, angle, height; per canopy: x, y, radius, centre
    height, porosity."""
    rng = SplitMix64(seed)
    lx, ly, lz = nx * h, ny * h, nz * h
    meshes, objects, first = [], [], 0
    for _ in range(n_buildings):
        cx, cy = rng.uniform(0.1 * lx, 0.9 * lx), rng.uniform(0.1 * ly, 0.9 * ly)
        r = rng.uniform(4.0, 10.0)
        sides = rng.randint(4, 8)
        ang = rng.uniform(0.0, 2 * np.pi)
        H = rng.uniform(8.0, 0.8 * lz)
        m = prism_mesh(cx, cy, r, sides, ang, 0.0, H)
        meshes.append(m)
        objects.append((first, len(m), 0.0))
        first += len(m)
    for _ in range(n_trees):
        cx, cy = rng.uniform(0.1 * lx, 0.9 * lx), rng.uniform(0.1 * ly, 0.9 * ly)
        r = rng.uniform(3.0, 6.0)
        zc = rng.uniform(4.0, 10.0)
        phi_in = rng.uniform(0.3, 0.8)
        m = icosphere_mesh(cx, cy, zc, r, levels=1, scale=(1.0, 1.0, 0.75))
        meshes.append(m)
        objects.append((first, len(m), phi_in))
        first += len(m)
    return np.concatenate(meshes), objects


def empty_domain(nx, ny, nz, h=1.0, u_ref=2.0, wind_dir_deg=0.0, ground_noslip=False,
                 loglaw=False) -> Scenario:
    phi = np.ones((nz, ny, nx))
    return Scenario(nx, ny, nz, h, phi, wind_dir_deg=wind_dir_deg, u_ref=u_ref,
                    inflow_loglaw=loglaw, ground_noslip=ground_noslip, name="empty")


def random_fields(nx, ny, nz, seed=0, scale=1.0) -> dict:
    """Seeded random velocity / turbulence fields for operator-level tests."""
    g = np.random.default_rng(seed)
    return {
        "u": scale * g.standard_normal((nz, ny, nx + 1)),
        "v": scale * g.standard_normal((nz, ny + 1, nx)),
        "w": scale * g.standard_normal((nz + 1, ny, nx)),
        "p": g.standard_normal((nz, ny, nx)),
        "k": 0.1 + 0.5 * g.random((nz, ny, nx)),
        "omega": 0.05 + 0.5 * g.random((nz, ny, nx)),
    }


def batch_instances(n=32, seed=0, sizes_xy=(96, 256), sizes_z=(32, 64), speed=(2.0, 8.0),
                    steps=300):
    """Instances of uneven size, wind direction and speed for the batched run.

    Per instance, in order: nx, ny (multiples of 16), nz (multiple of 8),
    wind direction in [0, 360), speed, layout seed.
    """
    rng = SplitMix64(seed)
    out = []
    for _ in range(n):
        nx = 16 * rng.randint(sizes_xy[0] // 16, sizes_xy[1] // 16)
        ny = 16 * rng.randint(sizes_xy[0] // 16, sizes_xy[1] // 16)
        nz = 8 * rng.randint(sizes_z[0] // 8, sizes_z[1] // 8)
        wd = rng.uniform(0.0, 360.0)
        sp = rng.uniform(*speed)
        s = rng.next_u64() & 0xFFFFFFFF
        sc = scaled_urban_block(nx, ny, nz, seed=s, wind_dir_deg=wd, u_ref=sp, steps=steps)
        out.append(sc)
    return out


def config(name: str) -> Scenario:
    """Named workloads: the five configurations of the benchmark plan."""
    if name == "single_box":      # 64x32x16, FP64, 100 steps
        return single_box()
    if name == "urban256":        # 256x256x64, FP32 + FP64 reductions, 500 steps
        return urban_block()
    if name == "design128":       # 128x128x48, 12 parametric buildings, 200 steps
        return design_lattice()
    if name == "urban512":        # 512x512x128, 1 m cells
        return urban_block(512, 512, 128, h=1.0, n_boxes=400, n_trees=800,
                           height=(5.0, 120.0), u_ref=5.0, steps=1000)
    raise KeyError(name)


def angle_is_axis(deg: float) -> bool:
    return abs(math.sin(math.radians(deg))) < 1e-9 or abs(math.cos(math.radians(deg))) < 1e-9
