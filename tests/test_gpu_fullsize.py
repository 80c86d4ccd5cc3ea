"""The design and urban workloads at their stated sizes.

* Design workload (Sec. 4 "Automatic Design Optimization", Sec. 6): 128 x
  128 x 48 cells of 2 m, 12 parametric buildings (height, x and y offset:
  36 parameters), sigmoid design map of one-cell width, fixed time step,
  checkpointed adjoint of the comfort objective against central
  differences of the FP64 forward (see the two tests for what each checks
  and why the 1e-3 m difference is no reference over 200 steps).
* Urban workload: 256 x 256 x 64 cells of 2 m, 40 boxes and 60 canopies,
  500 steps in FP32 (with FP64 reductions) from one FP64 state against the
  FP64 run (held to the FP64 oracle step by step at smaller sizes): every
  field within 1e-3 relative L2, projected divergence <= 1e-6.
"""
import time

import numpy as np
import pytest

from paper_2204_01117_gb300 import layouts, uf

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NAMES = ("u", "v", "w", "p", "k", "omega")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    uf.build()
    uf.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def design_setup(d):
    theta0 = np.asarray(d.theta, dtype=np.float64).reshape(-1)
    g = uf.Grid(d.nx, d.ny, d.nz, precision="f64", **d.params())
    g.design_to_phi(d.boxes, theta0, d.width)
    g.init_state()
    return g, theta0, g.state()          # the start state, held fixed by the gradient


def design_J(g, d, x0, steps):
    def J(theta):
        g.design_to_phi(d.boxes, theta, d.width)
        g.set_fields(x0)
        g.run(steps)
        return g.objective(*BAND)
    return J


def adjoint_grad(g, d, theta0, x0, steps, C):
    g.design_to_phi(d.boxes, theta0, d.width)
    g.set_fields(x0)
    t0 = time.perf_counter()
    J0, dphi = g.adjoint_run(steps, ckpt_every=C, z_lo=BAND[0], z_hi=BAND[1], u_hi=BAND[2], u_lo=BAND[3])
    t = time.perf_counter() - t0
    grad = g.design_vjp(d.boxes, theta0, d.width, dphi)
    g.free_adjoint_workspace()
    return J0, grad, t


BAND = (1.0, 3.0, 4.0, 1.0)


def test_design_workload_gradient_all_36_parameters():
    """The full design grid and parameter set over 20 steps with checkpoints
    every 5 (four recomputed segments), against differences of the FP64
    forward at a 1e-6 m step, within 1e-4 relative (floor 1e-3 of the
    largest component).  The step is only piecewise smooth (Selle clamp,
    drag clamp, limiters, CG iteration counts), so the 1e-3 m difference the
    design workload names is no reference: it differs from the derivative
    by up to 20 % here, while differences from 3e-5 m down agree with each
    other to 1e-6.  The adjoint takes the branches of the forward at theta,
    i.e. the derivative of the smooth piece theta lies on.  Where the
    forward and backward differences at 1e-6 m agree the central one is the
    reference; where they do not, a switch lies within 1e-6 m on one side
    and the adjoint must match one of the two one-sided differences (at
    most four such components, counted and reported)."""
    d = layouts.design_lattice()            # 128 x 128 x 48, 12 buildings
    assert (d.nx, d.ny, d.nz) == (128, 128, 48)
    steps, C, h = 20, 5, 1e-6
    g, theta0, x0 = design_setup(d)
    assert theta0.size == 36
    J = design_J(g, d, x0, steps)
    J0, grad, _ = adjoint_grad(g, d, theta0, x0, steps, C)
    Jc = J(theta0)
    assert J0 == pytest.approx(Jc, rel=1e-12)
    jp = np.array([J(theta0 + h * e) for e in np.eye(theta0.size)])
    jm = np.array([J(theta0 - h * e) for e in np.eye(theta0.size)])
    fwd, bwd, cen = (jp - Jc) / h, (Jc - jm) / h, (jp - jm) / (2 * h)
    floor = 1e-3 * np.abs(cen).max()
    tol = 1e-4 * (np.abs(cen) + floor)
    kink = np.abs(fwd - bwd) > tol
    err = np.where(kink, np.minimum(np.abs(grad - fwd), np.abs(grad - bwd)), np.abs(grad - cen))
    print(f"design workload, 20 steps, C = 5: worst relative error {np.max(err / (np.abs(cen) + floor)):.2e}, "
          f"{int(kink.sum())} of 36 components with a switch within {h:g} m (one-sided reference)")
    assert int(kink.sum()) <= 4, (np.flatnonzero(kink), fwd, bwd)
    assert np.all(err <= tol), (np.flatnonzero(err > tol), grad, cen, fwd, bwd)
    g.close()


def test_design_workload_200_steps_gradient_direction():
    """The stated run: 200 steps, checkpoints every 20.  Over 200 steps the
    discrete map is rough at small scales (kinks of the clamps and limiters,
    jumps from changed CG iteration counts), so no per-component finite
    difference reaches 1e-3: the 1e-3 m differences are reported, not
    bounded.  Checked instead, at the scale of a design-loop step: along the
    normalised adjoint gradient the central difference at 1e-2 m gives the
    gradient's norm within 2 %, and a step of 0.1 m down the gradient lowers
    J while one up raises it."""
    d = layouts.design_lattice()
    assert (d.steps, d.ckpt_every) == (200, 20)
    g, theta0, x0 = design_setup(d)
    J = design_J(g, d, x0, d.steps)
    J0, grad, t_adj = adjoint_grad(g, d, theta0, x0, d.steps, d.ckpt_every)
    gn = np.linalg.norm(grad)
    e = grad / gn
    slope = (J(theta0 + 1e-2 * e) - J(theta0 - 1e-2 * e)) / 2e-2
    f3 = np.array([(J(theta0 + 1e-3 * v) - J(theta0 - 1e-3 * v)) / 2e-3 for v in np.eye(theta0.size)[:6]])
    print(f"design workload, 200 steps: |grad| = {gn:.5g}, central difference along it at 1e-2 m {slope:.5g}, "
          f"adjoint {t_adj:.2f} s; first 6 components adjoint {np.round(grad[:6], 4).tolist()} vs 1e-3 m "
          f"differences {np.round(f3, 4).tolist()}")
    assert slope == pytest.approx(gn, rel=2e-2)
    assert J(theta0 - 0.1 * e) < J0 < J(theta0 + 0.1 * e)
    g.close()


def test_urban_workload_fp32_vs_fp64_500_steps():
    sc = layouts.urban_block(256, 256, 64, seed=0)
    assert sc.steps == 500
    g64 = uf.Grid(sc.nx, sc.ny, sc.nz, precision="f64", **sc.params())
    g64.set_porosity(sc.phi)
    g64.init_state()
    x0 = g64.state()
    g32 = uf.Grid(sc.nx, sc.ny, sc.nz, precision="f32", **sc.params())
    g32.set_porosity(sc.phi.astype(np.float32))
    g32.set_fields({n: x0[n].astype(np.float32) for n in NAMES})
    s64 = g64.run(sc.steps)
    s32 = g32.run(sc.steps)
    errs = {n: rel(g32.get_state(n).astype(np.float64), g64.get_state(n)) for n in NAMES}
    div32 = g32.divergence()
    print(f"urban 256x256x64, 500 steps: FP32 vs FP64 relative L2 {errs}, divergence FP32 {div32:.3e}, "
          f"FP64 {g64.divergence():.3e}, CG iterations last step {s32.cg_iters} / {s64.cg_iters}")
    for n, e in errs.items():
        assert e <= 1e-3, (n, e)
    assert div32 <= 1e-6
    g32.close()
    g64.close()
