"""The fused step kernels against the separate sub-step kernels they replace.

The fused MacCormack advection forms every value with the expressions of
the two-pass form (forward and backward semi-Lagrangian kernels), and the
fused diffusion + drag + BC + right-hand-side kernel with those of its
three kernels (||b||^2 summed in the same order), from the same inputs, so
whole steps agree bit for bit: in FP32 and FP64, on ragged grids, with the
CFL time step (displacements below half a cell: everything from the staged
tiles) and with a fixed time step three times larger (displacements past a
cell: the global-memory fallbacks); each fusion alone and both together."""
import numpy as np
import pytest

from paper_2204_01117_gb300 import layouts, uf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ("u", "v", "w", "p", "k", "omega")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    uf.build()
    uf.load()


def run(sc, precision, unfused, nsteps, **extra):
    g = uf.Grid(sc.nx, sc.ny, sc.nz, precision=precision, **{**sc.params(), **extra})
    g.set_tuning(unfused=unfused)
    g.set_porosity(sc.phi.astype(g.np_dtype))
    g.init_state()
    for _ in range(nsteps):
        g.step()
    out = {n: g.get_state(n) for n in NAMES}
    g.close()
    return out


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("dt_scale", [0.0, 3.0])
@pytest.mark.parametrize("unfused", [uf.UNFUSED_ADVECT, uf.UNFUSED_MOMENTUM, uf.UNFUSED_ALL])
def test_fused_step_equals_sub_step_kernels_bitwise(precision, dt_scale, unfused):
    sc = layouts.urban_block(45, 37, 19, h=2.0, seed=3, wind_dir_deg=135.0)
    extra = {}
    if dt_scale > 0:
        probe = uf.Grid(sc.nx, sc.ny, sc.nz, precision=precision, **sc.params())
        probe.set_porosity(sc.phi.astype(probe.np_dtype))
        probe.init_state()
        dt = probe.step().dt
        probe.close()
        extra["fixed_dt"] = dt_scale * dt
    a = run(sc, precision, 0, 3, **extra)
    b = run(sc, precision, unfused, 3, **extra)
    for n in NAMES:
        assert np.array_equal(a[n], b[n]), n


def test_fused_advection_tuning_roundtrip():
    g = uf.Grid(40, 24, 18, precision="f32")
    g.set_tuning(advect_zc=5)
    t, _ = g.get_tuning()
    assert t["advect_zc"] == 5 and t["unfused"] == 0
    g.set_tuning()
    t, _ = g.get_tuning()
    assert t["advect_zc"] == 16
    with pytest.raises(uf.UFError):
        g.set_tuning(advect_zc=65)
    g.close()


def test_fused_step_with_the_paper_preconditioner():
    """A grid with the approximate-inverse preconditioner (no multigrid
    tail) runs the same fused kernels, and they agree with the sub-step
    kernels bit for bit there too."""
    sc = layouts.urban_block(40, 32, 12, h=2.0, seed=5)
    a = run(sc, "f32", 0, 2, precond="ai1", cg_max_iter=2000)
    b = run(sc, "f32", uf.UNFUSED_ALL, 2, precond="ai1", cg_max_iter=2000)
    for n in NAMES:
        assert np.array_equal(a[n], b[n]), n


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("smoother", ["cheby", "rbgs"])
def test_cluster_vcycle_equals_per_level_kernels_bitwise(precision, smoother):
    """The coarse levels of the V-cycle as per-level launches and as one
    thread-block-cluster launch from level 1, 2 or 3 down; with the
    automatic tail and with the tail at the coarsest level (every other
    level per level).  All give the same three steps bit for bit.  The
    levels (50 x 42 x 15, 25 x 21 x 8, 13 x 11 x 4, ...) are odd in every
    axis."""
    sc = layouts.urban_block(100, 84, 30, h=2.0, seed=4, wind_dir_deg=250.0)
    variants = {"per level": dict(coarse_start=-1), "cluster 1": dict(coarse_start=1),
                "cluster 2": dict(coarse_start=2), "cluster 3": dict(coarse_start=3)}
    for deepest in (False, True):
        out = {}
        for name, kw in variants.items():
            g = uf.Grid(sc.nx, sc.ny, sc.nz, precision=precision, mg_smoother=smoother, **sc.params())
            nl = g.get_tuning()[1]
            assert nl >= 5
            g.set_tuning(tail_level=nl - 1 if deepest else 0, **kw)
            t = g.get_tuning()[0]
            assert t["tail_level"] >= 3
            cs = kw["coarse_start"]
            if cs > 0 and cs < t["tail_level"]:
                assert t["coarse_start"] in (cs, -1)   # -1: the device cannot co-schedule the cluster
            g.set_porosity(sc.phi.astype(g.np_dtype))
            g.init_state()
            for _ in range(3):
                g.step()
            out[name] = {n: g.get_state(n) for n in NAMES}
            g.close()
        for name in variants:
            for n in NAMES:
                assert np.array_equal(out[name][n], out["per level"][n]), (deepest, name, n)
