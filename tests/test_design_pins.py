"""Oracle design -> porosity map: closed-form values of the logistic box."""
import numpy as np

import oracle


def test_design_map_inside_outside_and_edge():
    # one tall, wide box; h = 1 m so that the cell centre x = 4.5 sits on x_a
    boxes = [(4.5, 20.5, -100.0, 100.0)]
    theta = [(100.0, 0.0, 0.0)]
    phi = oracle.design_to_phi(32, 8, 4, 1.0, boxes, theta, width=1.0)
    # x = 10.5 m lies 6 m inside x_a and 10 m inside x_b: phi = 1 - s(6) s(10)
    s = lambda t: 1.0 / (1.0 + np.exp(-t))
    np.testing.assert_allclose(phi[:, :, 10], 1.0 - s(6.0) * s(10.0), rtol=1e-9)
    assert phi[:, :, 12].max() < 1e-3                  # deeper inside: nearly solid
    assert phi[:, :, 30].min() > 0.999                 # 9.5 m outside: open
    # on the x_a face the x ramp is s(0) = 1/2; the other ramps are ~1
    np.testing.assert_allclose(phi[:, :, 4], 0.5, atol=1e-3)


def test_design_map_shift_and_height():
    boxes = [(10.0, 20.0, 10.0, 20.0)]
    base = oracle.design_to_phi(32, 32, 16, 1.0, boxes, [(8.0, 0.0, 0.0)], width=0.5)
    shifted = oracle.design_to_phi(32, 32, 16, 1.0, boxes, [(8.0, 3.0, -2.0)], width=0.5)
    # a shift by whole cells moves the field
    np.testing.assert_allclose(shifted[:, 8:30, 3:29], base[:, 10:32, 0:26], atol=1e-12)
    # height: z = 7.5 lies below H = 8, z = 8.5 above
    assert base[7, 15, 15] < 0.3 and base[8, 15, 15] > 0.7


def test_design_map_overlap_is_product():
    boxes = [(2.0, 10.0, 2.0, 10.0), (6.0, 14.0, 2.0, 10.0)]
    theta = [(5.0, 0.0, 0.0), (5.0, 0.0, 0.0)]
    both = oracle.design_to_phi(16, 12, 6, 1.0, boxes, theta, width=1.0)
    a = oracle.design_to_phi(16, 12, 6, 1.0, boxes[:1], theta[:1], width=1.0)
    b = oracle.design_to_phi(16, 12, 6, 1.0, boxes[1:], theta[1:], width=1.0)
    np.testing.assert_allclose(both, a * b, rtol=1e-14)
