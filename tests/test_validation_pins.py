"""Host side of the vortex-shedding validation (the supplement's "Validation
of the Fluid Simulator"): the Strouhal relation it quotes, the frequency
estimator on signals of known frequency, and the cylinder workload."""
import numpy as np
import pytest

from paper_2204_01117_gb300 import layouts, validation


def test_strouhal_relation_values():
    # St = 0.198 (1 - 19.7/Re): the limit 0.198, zero at Re = 19.7, and the
    # supplement's range Re = 5.86e3 .. 5.86e4 (U = 2 .. 20 m/s, D = 0.046 m)
    assert validation.strouhal_formula(1e12, 1.0) == pytest.approx(0.198, rel=1e-12)
    assert validation.strouhal_formula(19.7 * 1.5e-5, 1.0) == pytest.approx(0.0, abs=1e-15)
    nu = 2.0 * 0.046 / 5.86e3
    assert validation.strouhal_formula(2.0, 0.046, nu) == pytest.approx(0.198 * (1 - 19.7 / 5.86e3), rel=1e-12)
    assert validation.strouhal_formula(20.0, 0.046, nu) == pytest.approx(0.198 * (1 - 19.7 / 5.86e4), rel=1e-12)


@pytest.mark.parametrize("f", [8.58, 21.49, 86.06])
def test_dominant_frequency_of_known_signals(f):
    dt = 1.0 / (40 * f) * 1.37            # not commensurate with the period
    t = np.arange(int(12 / (f * dt))) * dt
    clean = 1.3 * np.sin(2 * np.pi * f * t + 0.4) + 0.7
    assert validation.dominant_frequency(clean, dt) == pytest.approx(f, rel=2e-3)
    # a second harmonic (the streamwise signature of shedding), a drifting
    # mean (a wake still settling) and noise
    rng = np.random.default_rng(3)
    dirty = clean + 0.5 * np.sin(4 * np.pi * f * t + 1.0) + 0.8 * t / t[-1] + 0.05 * rng.standard_normal(t.size)
    assert validation.dominant_frequency(dirty, dt) == pytest.approx(f, rel=5e-3)


def test_no_oscillation_gives_no_peak():
    assert validation.dominant_frequency(np.linspace(0, 1, 100), 1e-3) == 0.0


def test_cylinder_workload():
    sc = layouts.karman_cylinder(5.0)
    assert (sc.nx, sc.ny, sc.nz, sc.h) == (512, 768, 1, 2e-3)
    solid = int((sc.phi == 0).sum())
    assert abs(solid - np.pi * (sc.D / (2 * sc.h)) ** 2) <= 0.02 * solid
    assert set(np.unique(sc.phi)) == {0.0, 1.0}
    # centred on the channel axis, 0.3 m from the inlet; inflow through y-
    ys, xs = np.nonzero(sc.phi[0] == 0)
    assert ((xs.mean() + 0.5) * sc.h) == pytest.approx(sc.centre[0], abs=sc.h)
    assert ((ys.mean() + 0.5) * sc.h) == pytest.approx(0.3, abs=sc.h)
    p = sc.params()
    assert p["wind_dir_deg"] == 90.0 and p["inflow_loglaw"] == 0 and p["ground_noslip"] == 0
    assert p["fixed_dt"] == 1e-4
