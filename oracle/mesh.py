"""Oracle of the mesh resolver of Sec. 3 ("Urban model resolving"), in FP64
numpy.  TEST INFRASTRUCTURE ONLY: only tests/ may import it; the product
never does, and it imports nothing from the product.

Each object is a closed triangle mesh with a porosity inside (0 for a
building, the canopy's value for a tree).  A point is inside an object when
it lies in the object's axis-aligned bounding box and a ray from it crosses
the object's triangles an odd number of times (even-odd rule); the crossings
follow Moller and Trumbore (1997), written without the division by the
determinant (the barycentric and distance tests compare against it, after
flipping its sign to positive).  A cell's porosity is the mean over a
uniform sub-grid of sub^3 points of the point porosity: the minimum inside
porosity over the objects containing the point, 1 in the open.

Every product and sum is a separate FP64 operation in a fixed order
(numpy does not fuse multiply-adds), so the classification of a point is a
deterministic function of its coordinates."""
from __future__ import annotations

import numpy as np

# ray direction: no component zero (no triangle of an axis-aligned face is
# parallel to it) and no simple ratio between components
RAY = (0.5741, 0.6219, 0.5327)


def sample_points(i, j, k, h, sub):
    """Sub-grid points of cells (i, j, k): ((i + (a + 1/2)/sub) h, ...)."""
    off = (np.arange(sub) + 0.5) / sub
    return ((i[:, None] + off[None, :]) * h, (j[:, None] + off[None, :]) * h, (k[:, None] + off[None, :]) * h)


def crossings(px, py, pz, tris):
    """Number of triangles the ray p + t RAY (t > 0) crosses, per point.
    px, py, pz: 1-D arrays of point coordinates; tris: (n, 3, 3)."""
    dx, dy, dz = RAY
    count = np.zeros(px.shape, dtype=np.int64)
    for tri in tris:
        v0, v1, v2 = tri
        e1x, e1y, e1z = v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]
        e2x, e2y, e2z = v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]
        # pvec = d x e2, det = e1 . pvec
        qx, qy, qz = dy * e2z - dz * e2y, dz * e2x - dx * e2z, dx * e2y - dy * e2x
        det = e1x * qx + e1y * qy + e1z * qz
        if det == 0.0:
            continue
        s = 1.0 if det > 0.0 else -1.0
        adet = det * s
        tx, ty, tz = px - v0[0], py - v0[1], pz - v0[2]
        u = (tx * qx + ty * qy + tz * qz) * s
        # qvec = tvec x e1
        rx, ry, rz = ty * e1z - tz * e1y, tz * e1x - tx * e1z, tx * e1y - ty * e1x
        v = (dx * rx + dy * ry + dz * rz) * s
        t = (e2x * rx + e2y * ry + e2z * rz) * s
        hit = (u >= 0.0) & (u <= adet) & (v >= 0.0) & (u + v <= adet) & (t > 0.0)
        count += hit
    return count


def mesh_porosity(nx: int, ny: int, nz: int, h: float, tris, objects, sub: int = 4) -> np.ndarray:
    """Cell porosity (nz, ny, nx) of the objects: tris (ntri, 3, 3) [m];
    objects: (first triangle, triangle count, inside porosity) per object."""
    tris = np.asarray(tris, dtype=np.float64).reshape(-1, 3, 3)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    xs, ys, zs = sample_points(ii, jj, kk, h, sub)
    acc = np.zeros(ii.size)
    for c in range(sub):
        for b in range(sub):
            for a in range(sub):
                px, py, pz = xs[:, a], ys[:, b], zs[:, c]
                val = np.ones(ii.size)
                for first, count, phi_in in objects:
                    t = tris[first:first + count]
                    lo, hi = t.reshape(-1, 3).min(axis=0), t.reshape(-1, 3).max(axis=0)
                    inb = ((px >= lo[0]) & (px <= hi[0]) & (py >= lo[1]) & (py <= hi[1]) & (pz >= lo[2])
                           & (pz <= hi[2]))
                    if not inb.any():
                        continue
                    sel = np.nonzero(inb)[0]
                    odd = (crossings(px[sel], py[sel], pz[sel], t) & 1) == 1
                    hit = sel[odd]
                    val[hit] = np.minimum(val[hit], phi_in)
                acc += val
    return (acc / (sub * sub * sub)).reshape(nz, ny, nx)


def mesh_volume(tris) -> float:
    """Enclosed volume of a closed, consistently oriented triangle mesh
    (divergence theorem: sum of signed tetrahedra with the origin)."""
    t = np.asarray(tris, dtype=np.float64).reshape(-1, 3, 3)
    return float(np.abs(np.einsum("ij,ij->i", t[:, 0], np.cross(t[:, 1], t[:, 2])).sum()) / 6.0)
