"""Design loop of Sec. 6 ("Avoiding Heat Pockets in Early Design Stages"):
the region-average objective (uf_objective_ex) against the oracle, its
adjoint gradient (uf_adjoint_run_ex) against finite differences, a few
gradient-descent iterations, and the wind-direction robustness re-runs as
one batch."""
import numpy as np
import pytest

import oracle
from paper_2204_01117_gb300 import uf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NX, NY, NZ, H = 24, 20, 10, 2.0
BOXES = [(14.0, 22.0, 12.0, 20.0), (28.0, 36.0, 20.0, 28.0)]
THETA = np.array([9.0, 0.3, -0.4, 7.0, -0.2, 0.5])
WIDTH = 2.0
PARAMS = dict(h=H, wind_dir_deg=0.0, u_ref=3.0, z_ref=10.0, z0=0.5, inflow_loglaw=1, ground_noslip=1,
              fixed_dt=0.25)
NSTEPS = 6
U_T = 0.55
# pedestrian-level regions: between the buildings, in the wake (an edge on a
# cell centre, x = 37), and one reaching past the outflow and side walls
REGIONS = [(22.0, 28.0, 12.0, 28.0, 0.0, 4.0), (37.0, 46.0, 14.0, 30.0, 0.0, 4.0), (40.0, 60.0, -5.0, 5.0, 0.0, 3.0)]
OBJ = {"kind": "regions", "regions": REGIONS, "u_t": U_T}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    uf.build()
    uf.load()
    oracle.build()


def grid(precision="f64", **kw):
    p = dict(PARAMS)
    p.update(kw)
    return uf.Grid(NX, NY, NZ, precision=precision, **p)


def start_state(g):
    g.design_to_phi(BOXES, THETA, WIDTH)
    g.init_state()
    g.run(4)
    return g.state()


def J_of(g, x0, theta):
    g.design_to_phi(BOXES, theta, WIDTH)
    g.set_fields(x0)
    g.run(NSTEPS)
    return g.objective_ex(OBJ)


def oracle_L(g):
    f = {n: g.get_state(n).astype(np.float64) for n in ("u", "v", "w")}
    return oracle.region_objective(f["u"], f["v"], f["w"], H, REGIONS, U_T)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_region_objective_matches_oracle_on_the_same_state(precision):
    """Cell speeds and sums in FP64 on both sides, from the same stored
    velocities: equal up to the order of the FP64 sums."""
    g = grid(precision)
    start_state(g)
    g.run(3)
    L, means = oracle_L(g)
    assert min(abs(m - U_T) for m in means) > 0.05     # L is not near a cancellation
    assert g.objective_ex(OBJ) == pytest.approx(L, rel=1e-12)
    # a single region, and the comfort band through the same entry point
    one = {"kind": "regions", "regions": REGIONS[1:2], "u_t": 1.0}
    f = {n: g.get_state(n).astype(np.float64) for n in ("u", "v", "w")}
    L1, _ = oracle.region_objective(f["u"], f["v"], f["w"], H, REGIONS[1:2], 1.0)
    assert g.objective_ex(one) == pytest.approx(L1, rel=1e-12)
    assert g.objective_ex({"kind": "comfort", "band": (1.0, 3.0, 4.0, 1.0)}) == g.objective(1.0, 3.0, 4.0, 1.0)


def test_region_objective_after_oracle_run():
    """The whole design evaluation, GPU FP64 against the oracle's run."""
    o = oracle.Oracle(NX, NY, NZ, **PARAMS)
    o.set("phi", oracle.design_to_phi(NX, NY, NZ, H, BOXES, THETA.reshape(-1, 3), WIDTH))
    o.init()
    o.run(4 + NSTEPS)
    ref, _ = oracle.region_objective(o.get("u"), o.get("v"), o.get("w"), H, REGIONS, U_T)
    g = grid()
    x0 = start_state(g)
    assert J_of(g, x0, THETA) == pytest.approx(ref, rel=1e-9)


def test_region_adjoint_theta_gradient_vs_central_fd():
    g = grid()
    x0 = start_state(g)
    g.design_to_phi(BOXES, THETA, WIDTH)
    g.set_fields(x0)
    J, dphi = g.adjoint_run(NSTEPS, ckpt_every=4, objective=OBJ)
    assert J == pytest.approx(J_of(g, x0, THETA), rel=1e-12)
    grad = g.design_vjp(BOXES, THETA, WIDTH, dphi)

    def central(hs):
        return np.array([(J_of(g, x0, THETA + e) - J_of(g, x0, THETA - e)) / (2 * hs)
                         for e in hs * np.eye(THETA.size)])
    f3, f4 = central(1e-3), central(1e-4)
    # a component whose 1e-3 m difference straddles a switch of the
    # piecewise-smooth step takes the 1e-4 m difference
    smooth = np.abs(f3 - f4) <= 1e-4 * np.abs(f4) + 1e-5 * np.abs(f4).max()
    fd = np.where(smooth, f3, f4)
    assert (~smooth).sum() <= 2, (f3, f4)
    floor = 1e-3 * np.abs(fd).max()
    assert np.all(np.abs(grad - fd) <= 1e-3 * np.abs(fd) + floor), (grad, fd)


def test_comfort_through_the_extended_entry_is_the_same_gradient():
    g = grid()
    x0 = start_state(g)
    g.set_fields(x0)
    J1, d1 = g.adjoint_run(NSTEPS, ckpt_every=3)
    g.set_fields(x0)
    J2, d2 = g.adjoint_run(NSTEPS, ckpt_every=3, objective={"kind": "comfort", "band": (1.0, 3.0, 4.0, 1.0)})
    assert J1 == J2
    # the transposed operators scatter with atomics: equal up to the order
    # of floating-point additions
    np.testing.assert_allclose(d1, d2, rtol=1e-12, atol=1e-14 * np.abs(d1).max())


def test_region_objective_autograd_matches_adjoint():
    g = grid()
    x0 = start_state(g)
    theta = torch.tensor(THETA.reshape(-1, 3), dtype=torch.float64, requires_grad=True)
    L = uf.comfort_objective(uf.design_porosity(theta, g, BOXES, WIDTH), g, x0, NSTEPS, ckpt_every=3,
                             objective=OBJ)
    L.backward()
    g.design_to_phi(BOXES, THETA, WIDTH)
    g.set_fields(x0)
    J, dphi = g.adjoint_run(NSTEPS, ckpt_every=3, objective=OBJ)
    assert L.item() == pytest.approx(J, rel=1e-12)
    np.testing.assert_allclose(theta.grad.numpy().ravel(), g.design_vjp(BOXES, THETA, WIDTH, dphi), rtol=1e-9,
                               atol=1e-12)


def test_gradient_descent_lowers_the_region_objective():
    """theta <- clip(theta - lambda dL/dtheta): with a step of 0.3 m on the
    largest component, every iteration lowers L, and the bounds hold."""
    g = grid()
    x0 = start_state(g)
    g.design_to_phi(BOXES, THETA, WIDTH)
    g.set_fields(x0)
    _, dphi = g.adjoint_run(NSTEPS, ckpt_every=3, objective=OBJ)
    g0 = g.design_vjp(BOXES, THETA, WIDTH, dphi)
    step = 0.3 / np.abs(g0).max()
    lower = np.tile([4.0, -1.0, -1.0], 2)
    upper = np.tile([12.0, 1.0, 1.0], 2)
    theta, hist = uf.optimize_design(g, BOXES, THETA, x0, NSTEPS, iterations=4, step_size=step, width=WIDTH,
                                     objective=OBJ, ckpt_every=3, lower=lower, upper=upper)
    Ls = [h[0] for h in hist]
    np.testing.assert_allclose(hist[0][2].ravel(), g0, rtol=1e-12, atol=0)
    assert all(b < a for a, b in zip(Ls, Ls[1:])), Ls
    assert J_of(g, x0, theta.ravel()) < Ls[-1]
    assert np.all(theta.ravel() >= lower) and np.all(theta.ravel() <= upper)


def test_wind_robustness_batch_equals_solo_runs():
    """The +-10 degree re-runs advanced together as one batch give, for each
    direction, the objective of the same design run alone."""
    g = grid("f32")
    phi = g.design_to_phi(BOXES, THETA, WIDTH, set_porosity=False)
    params = dict(PARAMS, nx=NX, ny=NY, nz=NZ)
    params.pop("wind_dir_deg")
    winds = (-10.0, 0.0, 10.0)
    out = uf.wind_robustness(params, phi, winds, 8, objective=OBJ)
    for wd, Lb in zip(winds, out):
        s = grid("f32", wind_dir_deg=wd)
        s.set_porosity(phi.astype(s.np_dtype))
        s.init_state()
        s.run(8)
        assert Lb == s.objective_ex(OBJ), wd
    assert len(set(out)) == 3


@pytest.mark.parametrize("obj, msg", [
    ({"kind": "regions", "regions": np.zeros((0, 6)), "u_t": U_T}, "regions"),
    ({"kind": "regions", "regions": [REGIONS[0]] * 9, "u_t": U_T}, "regions"),
    ({"kind": "regions", "regions": [(100.0, 120.0, 0.0, 10.0, 0.0, 4.0)], "u_t": U_T}, "no cell centre"),
    ({"kind": "regions", "regions": [(10.0, 10.5, 0.0, 10.0, 0.0, 4.0)], "u_t": U_T}, "no cell centre"),
])
def test_region_objective_rejects_bad_regions(obj, msg):
    g = grid("f32")
    g.init_state()
    with pytest.raises(uf.UFError) as ei:
        g.objective_ex(obj)
    assert ei.value.status == uf.UF_ERR_ARG and msg in str(ei.value)
