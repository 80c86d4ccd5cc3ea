"""Oracle of the mesh resolver (Sec. 3, "Urban model resolving") against
what fixes it independently: the analytic box rasterizer of the input
generator (same sample points, inside test by coordinates), enclosed
volumes by the divergence theorem, an exact half-cell cut, the even-odd
count of single points, and the minimum rule for overlaps."""
import numpy as np
import pytest

from oracle import mesh
from paper_2204_01117_gb300 import layouts


def test_box_meshes_match_the_box_rasterizer():
    boxes = [layouts.Box(3.3, 17.9, 5.1, 12.7, 0.0, 9.3), layouts.Box(20.2, 31.7, 2.9, 21.3, 0.0, 14.9)]
    nx, ny, nz, h = 18, 14, 9, 2.0
    tris, objects, first = [], [], 0
    for b in boxes:
        m = layouts.box_mesh(b.x0, b.x1, b.y0, b.y1, b.z0, b.z1)
        tris.append(m)
        objects.append((first, len(m), 0.0))
        first += len(m)
    got = mesh.mesh_porosity(nx, ny, nz, h, np.concatenate(tris), objects, sub=4)
    ref = layouts.rasterize(nx, ny, nz, h, boxes, sub=4)
    np.testing.assert_array_equal(got, ref)
    assert (got < 1).any() and (got > 0).any() and ((got > 0) & (got < 1)).any()


@pytest.mark.parametrize("shape", ["sphere", "prism"])
def test_solid_volume_matches_the_enclosed_volume(shape):
    nx, ny, nz, h = 20, 20, 12, 1.0
    if shape == "sphere":
        tris = layouts.icosphere_mesh(10.1, 9.7, 6.2, 4.3, levels=2)
    else:
        tris = layouts.prism_mesh(9.6, 10.3, 6.1, 7, 0.4, 0.0, 8.7)
    phi = mesh.mesh_porosity(nx, ny, nz, h, tris, [(0, len(tris), 0.0)], sub=4)
    vol = float(np.sum(1.0 - phi)) * h ** 3
    # sub-sampling error: the surface area times about a quarter of the sample spacing, random sign
    assert vol == pytest.approx(mesh.mesh_volume(tris), rel=0.01)


def test_half_cell_cut_is_exact():
    # face at x = 4.5 cells: sample planes at i + 0.125, 0.375 | 0.625, 0.875
    tris = layouts.box_mesh(0.0, 4.5, 0.0, 10.0, 0.0, 10.0)
    phi = mesh.mesh_porosity(8, 4, 3, 1.0, tris, [(0, 12, 0.0)], sub=4)
    assert np.all(phi[:, :, :4] == 0.0) and np.all(phi[:, :, 4] == 0.5) and np.all(phi[:, :, 5:] == 1.0)


def test_even_odd_count_of_points():
    tris = layouts.box_mesh(0.0, 2.0, 0.0, 2.0, 0.0, 2.0)
    px, py, pz = np.array([1.0, 3.0, -0.5, 1.3]), np.array([1.0, 1.0, 0.3, 0.2]), np.array([1.0, 1.0, 0.3, 1.9])
    n = mesh.crossings(px, py, pz, tris)
    # inside: one face crossed; outside beyond it: none; outside, the ray through it: two
    assert list(n) == [1, 0, 2, 1]


def test_overlap_takes_the_smaller_porosity():
    b = layouts.box_mesh(0.0, 6.0, 0.0, 6.0, 0.0, 6.0)
    t = layouts.icosphere_mesh(6.0, 3.0, 3.0, 2.9, levels=2)
    tris = np.concatenate([b, t])
    objs = [(0, len(b), 0.0), (len(b), len(t), 0.5)]
    phi = mesh.mesh_porosity(10, 6, 6, 1.0, tris, objs, sub=2)
    assert phi[3, 3, 2] == 0.0              # inside the box only
    assert phi[3, 3, 7] == 0.5              # inside the canopy only
    assert phi[3, 3, 5] == 0.0              # inside both
    assert phi[0, 0, 9] == 1.0              # open
