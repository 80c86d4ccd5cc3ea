"""Vortex shedding behind a cylinder (the supplement's solver validation)
through the CUDA step: at a cell Courant number of 1 the measured Strouhal
number matches St = 0.198 (1 - 19.7/Re) within 3 % (measured within 0.1 %
from 2 to 20 m/s, once the street has settled: equal probe amplitudes over
the two halves of the sample); at the supplement's fixed dt = 1e-4 s that
holds at 20 m/s (Courant number 1 there).

At 2 m/s a time-step and grid study (bench.py --karman-study) found St a
smooth function of dt alone: it rises as dt falls (0.198 at 1e-3 s, 0.245
at 1e-4 s, 0.250 at 6.7e-5 s) and barely moves when the cells are refined
1.5 times at a fixed dt (0.245 and 0.248 at 1e-4 s).  So the departure from
the relation at the supplement's dt is time-discretization error of the
split step converging to a limit near 0.25-0.26, about a quarter above the
relation, not interpolation error of the semi-Lagrangian step (which would
shrink under refinement at a fixed Courant number; it grows instead)."""
import pytest

from paper_2204_01117_gb300 import uf, validation

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    uf.build()
    uf.load()


@pytest.mark.parametrize("U, kw", [(5.0, dict(cfl=1.0)), (20.0, dict())])
def test_shedding_frequency_matches_strouhal_relation(U, kw):
    r = validation.shedding_run(U, **kw)
    assert r["amplitude"] > 0.2 * U            # a vortex street, not a steady wake
    a1, a2 = r["amplitude_halves"]
    assert a1 == pytest.approx(a2, rel=0.05), r   # settled: not still growing
    assert r["St"] == pytest.approx(r["St_formula"], rel=0.03), r
    assert r["divergence"] <= 1e-6


@pytest.mark.slow
def test_shedding_at_the_supplements_time_step_2_m_s():
    """U = 2 m/s at dt = 1e-4 s: the frequency does not depend on the grid
    (2 mm and 4/3 mm cells within 2 %), it lies 15-30 % above the relation
    (measured +24.1 % and +25.4 %), and doubling dt lowers it (measured
    +22.0 % at 2e-4 s): the behaviour the study documents."""
    h2 = 2e-3 / 1.5
    a = validation.shedding_run(2.0, dt=1e-4)
    b = validation.shedding_run(2.0, dt=1e-4, nx=768, ny=1152, h=h2)
    c = validation.shedding_run(2.0, dt=2e-4)
    for r in (a, b, c):
        assert r["amplitude"] > 0.2 * 2.0 and r["divergence"] <= 1e-6
        assert r["amplitude_halves"][0] == pytest.approx(r["amplitude_halves"][1], rel=0.05), r
    assert b["St"] == pytest.approx(a["St"], rel=0.02), (a, b)
    for r in (a, b):
        assert 1.15 <= r["St"] / r["St_formula"] <= 1.30, r
    assert c["St"] < a["St"], (a, c)
