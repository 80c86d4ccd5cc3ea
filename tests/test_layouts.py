"""Seeded input generator: SplitMix64 stream and cut-cell porosity."""
import numpy as np

from paper_2204_01117_gb300 import layouts


def test_splitmix64_reference_outputs():
    # Published first outputs of SplitMix64 seeded with 0 (Steele et al. 2014;
    # the same values seed xoshiro generators in their reference code).
    g = layouts.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                0x06C45D188009454F]


def test_uniform_range_and_determinism():
    a = layouts.SplitMix64(42)
    b = layouts.SplitMix64(42)
    xs = [a.uniform(2.0, 5.0) for _ in range(1000)]
    assert xs == [b.uniform(2.0, 5.0) for _ in range(1000)]
    assert min(xs) >= 2.0 and max(xs) < 5.0
    ks = [layouts.SplitMix64(s).randint(3, 7) for s in range(200)]
    assert set(ks) == {3, 4, 5, 6, 7}


def test_rasterize_aligned_and_cut_cells():
    nx, ny, nz, h = 8, 6, 4, 1.0
    box = layouts.Box(2.0, 5.0, 1.0, 3.0, 0.0, 2.0, 0.0)      # cell aligned
    phi = layouts.rasterize(nx, ny, nz, h, [box])
    assert np.all(phi[0:2, 1:3, 2:5] == 0.0)
    assert phi.sum() == nx * ny * nz - 3 * 2 * 2
    half = layouts.Box(2.5, 5.0, 1.0, 3.0, 0.0, 2.0, 0.0)      # half a cell in x
    phi = layouts.rasterize(nx, ny, nz, h, [half])
    assert np.all(phi[0:2, 1:3, 2] == 0.5)
    tree = layouts.Ellipsoid(4.0, 3.0, 2.0, 1.5, 1.5, 1.0, 0.4)
    both = layouts.rasterize(nx, ny, nz, h, [box, tree])
    assert both.min() == 0.0 and 0.4 <= both[both > 0].min() < 1.0


def test_single_box_layout():
    sc = layouts.single_box()
    assert (sc.nx, sc.ny, sc.nz, sc.h) == (64, 32, 16, 2.0)
    # 20 x 10 x 12 m box = 10 x 5 x 6 cells of solid volume
    assert np.isclose((1.0 - sc.phi).sum(), 10 * 5 * 6)


def test_urban_block_statistics():
    sc = layouts.urban_block(128, 128, 32, n_boxes=10, n_trees=15, seed=3)
    assert sc.phi.shape == (32, 128, 128)
    assert 0.0 <= sc.phi.min() and sc.phi.max() == 1.0
    assert (sc.phi == 0.0).any() and ((sc.phi > 0) & (sc.phi < 1)).any()
    # margin: the first and last 10% of x stay clear
    assert np.all(sc.phi[:, :, :12] == 1.0) and np.all(sc.phi[:, :, -12:] == 1.0)
    again = layouts.urban_block(128, 128, 32, n_boxes=10, n_trees=15, seed=3)
    assert np.array_equal(sc.phi, again.phi)


def test_design_lattice_workload():
    d = layouts.design_lattice()
    assert (d.nx, d.ny, d.nz, d.h) == (128, 128, 48, 2.0)
    assert d.boxes.shape == (12, 4) and d.theta.shape == (12, 3)
    # square 20 m footprints centred on the 4 x 3 lattice
    np.testing.assert_allclose(d.boxes[:, 1] - d.boxes[:, 0], 20.0)
    np.testing.assert_allclose(d.boxes[:, 3] - d.boxes[:, 2], 20.0)
    cx = 0.5 * (d.boxes[:, 0] + d.boxes[:, 1])
    cy = 0.5 * (d.boxes[:, 2] + d.boxes[:, 3])
    np.testing.assert_allclose(sorted(set(np.round(cx, 6))), [256 * c / 5 for c in (1, 2, 3, 4)])
    np.testing.assert_allclose(sorted(set(np.round(cy, 6))), [256 * r / 4 for r in (1, 2, 3)])
    assert np.all((d.theta[:, 0] >= 20.0) & (d.theta[:, 0] < 40.0))
    assert np.all(d.theta[:, 1:] == 0.0)
    assert d.params()["fixed_dt"] == 0.2 and d.width == d.h
    # seeded: same seed, same heights; another seed, other heights
    assert np.array_equal(layouts.design_lattice().theta, d.theta)
    assert not np.array_equal(layouts.design_lattice(seed=1).theta, d.theta)
    # six pedestrian-level target regions, each centred between four buildings
    assert d.regions.shape == (6, 6) and d.u_t == 0.55
    rx, ry = 0.5 * (d.regions[:, 0] + d.regions[:, 1]), 0.5 * (d.regions[:, 2] + d.regions[:, 3])
    for x, y in zip(rx, ry):
        near = np.sort(np.hypot(cx - x, cy - y))[:4]
        np.testing.assert_allclose(near, near[0])
    assert np.all(d.regions[:, 4:] == (0.0, 3.0))
