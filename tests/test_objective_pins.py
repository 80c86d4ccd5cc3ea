"""Oracle of the region-average objective (Sec. 6, "Avoiding Heat Pockets"):
closed forms and cell selection."""
import numpy as np

import oracle


def uniform(nx, ny, nz, U, V=0.0):
    return (np.full((nz, ny, nx + 1), U), np.full((nz, ny + 1, nx), V), np.zeros((nz + 1, ny, nx)))


def test_uniform_flow_closed_form():
    u, v, w = uniform(10, 8, 4, 3.0, 4.0)           # |u| = 5 everywhere
    regions = [(0, 20, 0, 16, 0, 4), (4, 8, 4, 8, 1, 3)]
    L, means = oracle.region_objective(u, v, w, 2.0, regions, 0.55)
    assert np.allclose(means, [5.0, 5.0])
    assert L == np.float64(2 * (5.0 - 0.55) ** 2)


def test_cell_selection_by_centre():
    # a field whose cell speed is the cell index i (u_c = i along x): u faces at i - 0.5 ... i + 0.5
    nx, ny, nz, h = 12, 3, 2, 1.0
    u = np.broadcast_to(np.arange(nx + 1) - 0.5, (nz, ny, nx + 1)).copy()
    v, w = np.zeros((nz, ny + 1, nx)), np.zeros((nz + 1, ny, nx))
    # centres at 0.5, 1.5, ...: x in [2.0, 5.0] selects i = 2, 3, 4 -> speeds 2, 3, 4 (mean 3)
    L, means = oracle.region_objective(u, v, w, h, [(2.0, 5.0, 0.0, 3.0, 0.0, 2.0)], 1.0)
    assert means == [3.0] and L == 4.0
    # a box edge exactly on a centre includes it
    _, m2 = oracle.region_objective(u, v, w, h, [(2.5, 2.5, 0.0, 3.0, 0.0, 2.0)], 0.0)
    assert m2 == [2.0]


def test_target_between_speeds():
    u, v, w = uniform(6, 6, 2, 1.0)
    u[:, :, 3:] = 3.0                                 # faces i >= 3: cell 2 averages 2, cells 3.. are 3
    L, means = oracle.region_objective(u, v, w, 1.0, [(0, 1.9, 0, 6, 0, 2), (3.6, 6, 0, 6, 0, 2)], 2.0)
    assert means == [1.0, 3.0] and L == 2.0
