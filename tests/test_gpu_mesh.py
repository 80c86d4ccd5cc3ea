"""Mesh resolver (Sec. 3, "Urban model resolving") through the C ABI
against its oracle: the cell porosity counts sub-grid points classified by
an even-odd ray test, so it must match bit for bit (FP64 grid) or after
rounding to FP32 (FP32 grid)."""
import numpy as np
import pytest

from oracle import mesh
from paper_2204_01117_gb300 import layouts, uf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    uf.build()
    uf.load()


@pytest.mark.parametrize("seed, sub", [(0, 4), (1, 3), (2, 2)])
def test_mesh_porosity_matches_oracle_bit_for_bit(seed, sub):
    nx, ny, nz, h = 37, 29, 13, 2.0          # ragged against the 32 x 8 thread tiles
    tris, objs = layouts.mesh_city(nx, ny, nz, h, n_buildings=5, n_trees=3, seed=seed)
    ref = mesh.mesh_porosity(nx, ny, nz, h, tris, objs, sub=sub)
    assert (ref == 0).any() and ((ref > 0) & (ref < 1)).any() and (ref == 1).any()
    g64 = uf.Grid(nx, ny, nz, h=h, precision="f64")
    np.testing.assert_array_equal(g64.mesh_to_phi(tris, objs, sub=sub, set_porosity=False), ref)
    g32 = uf.Grid(nx, ny, nz, h=h, precision="f32")
    np.testing.assert_array_equal(g32.mesh_to_phi(tris, objs, sub=sub, set_porosity=False), ref.astype(np.float32))
    # the default sets the grid's porosity
    g64.mesh_to_phi(tris, objs, sub=sub)
    np.testing.assert_array_equal(g64.get_state("phi"), ref)
    # and to a device tensor
    out = torch.empty(g64.shapes["phi"], dtype=torch.float64, device="cuda")
    g64.mesh_to_phi(tris, objs, sub=sub, out=out)
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


def test_mesh_box_equals_box_rasterizer_on_device():
    b = layouts.Box(3.3, 17.9, 5.1, 12.7, 0.0, 9.3)
    g = uf.Grid(18, 14, 9, h=2.0, precision="f64")
    got = g.mesh_to_phi(layouts.box_mesh(b.x0, b.x1, b.y0, b.y1, b.z0, b.z1), [(0, 12, 0.0)], set_porosity=False)
    np.testing.assert_array_equal(got, layouts.rasterize(18, 14, 9, 2.0, [b], sub=4))


@pytest.mark.parametrize("objs, sub", [([(0, 13, 0.0)], 4), ([(-1, 3, 0.0)], 4), ([(0, 12, 1.5)], 4),
                                       ([(0, 12, 0.0)], 0), ([(0, 12, 0.0)], 17)])
def test_mesh_arguments_rejected(objs, sub):
    g = uf.Grid(8, 8, 4, h=1.0, precision="f32")
    with pytest.raises(uf.UFError) as ei:
        g.mesh_to_phi(layouts.box_mesh(1, 3, 1, 3, 0, 2), objs, sub=sub, set_porosity=False)
    assert ei.value.status == uf.UF_ERR_ARG
