"""Discrete adjoint of the RANS step: gradients against finite differences
of the forward runs (GPU FP64 and the FP64 oracle), checkpoint invariance,
precision, the design map and the autograd binding."""
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
BAND = (1.0, 3.0, 4.0, 1.0)


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
    """Developed initial state X0 (held fixed by the gradient)."""
    g.design_to_phi(BOXES, THETA, WIDTH)
    g.init_state()
    g.run(4)
    return g.state()


def fd_reference(J):
    """Central differences of J(theta) with the prescribed 1e-3 m step.  The
    step is piecewise smooth (the Selle clamp of the MacCormack scheme, the
    drag clamp and the eddy-viscosity limiter switch branches), so where the
    1e-3 m difference straddles such a switch it disagrees with the 1e-4 m
    difference; that component takes the 1e-4 m value.  Decided from forward
    runs alone.  Returns (reference, number of components replaced)."""
    def central(hs):
        return np.array([(J(THETA + e) - J(THETA - e)) / (2 * hs) for e in hs * np.eye(THETA.size)])
    f3, f4 = central(1e-3), central(1e-4)
    smooth = np.abs(f3 - f4) <= 1e-4 * np.abs(f4) + 1e-5 * np.abs(f4).max()
    return np.where(smooth, f3, f4), int((~smooth).sum())


def J_of(g, x0, phi=None, theta=None):
    if theta is not None:
        g.design_to_phi(BOXES, theta, WIDTH)
    if phi is not None:
        g.set_porosity(phi.astype(g.np_dtype))
    g.set_fields(x0)
    g.run(NSTEPS)
    return g.objective(*BAND)


def test_design_map_matches_oracle():
    g = grid()
    phi = g.design_to_phi(BOXES, THETA, WIDTH, set_porosity=False)
    ref = oracle.design_to_phi(NX, NY, NZ, H, BOXES, THETA.reshape(-1, 3), WIDTH)
    np.testing.assert_allclose(phi, ref, rtol=0, atol=1e-13)


def test_design_vjp_matches_fd():
    g = grid()
    lam = np.random.default_rng(4).standard_normal((NZ, NY, NX))
    gv = g.design_vjp(BOXES, THETA, WIDTH, lam)
    for q in range(6):
        e = np.zeros(6)
        e[q] = 1e-5
        fp = oracle.design_to_phi(NX, NY, NZ, H, BOXES, (THETA + e).reshape(-1, 3), WIDTH)
        fm = oracle.design_to_phi(NX, NY, NZ, H, BOXES, (THETA - e).reshape(-1, 3), WIDTH)
        fd = np.sum(lam * (fp - fm)) / 2e-5
        assert gv[q] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_adjoint_directional_derivative_in_phi():
    g = grid()
    x0 = start_state(g)
    phi = g.get_state("phi")
    g.set_fields(x0)
    J, dphi = g.adjoint_run(NSTEPS, ckpt_every=4, z_lo=BAND[0], z_hi=BAND[1], u_hi=BAND[2], u_lo=BAND[3])
    assert J > 0
    rng = np.random.default_rng(11)
    for trial in range(3):
        v = rng.standard_normal(phi.shape) * phi * (1 - phi)
        eps = 1e-5
        jp = J_of(g, x0, phi=phi + eps * v)
        jm = J_of(g, x0, phi=phi - eps * v)
        fd = (jp - jm) / (2 * eps)
        ad = float(np.sum(dphi * v))
        assert ad == pytest.approx(fd, rel=1e-4), (trial, ad, fd)


def test_adjoint_theta_gradient_vs_central_fd():
    g = grid()
    x0 = start_state(g)
    g.design_to_phi(BOXES, THETA, WIDTH)
    g.set_fields(x0)
    J, dphi = g.adjoint_run(NSTEPS, ckpt_every=3, z_lo=BAND[0], z_hi=BAND[1], u_hi=BAND[2], u_lo=BAND[3])
    grad = g.design_vjp(BOXES, THETA, WIDTH, dphi)
    fd, replaced = fd_reference(lambda th: J_of(g, x0, theta=th))
    assert replaced <= 2, fd
    floor = 1e-3 * np.abs(fd).max()
    assert np.all(np.abs(grad - fd) <= 1e-3 * np.abs(fd) + floor), (grad, fd)


def test_checkpoint_interval_does_not_change_gradient():
    g = grid()
    x0 = start_state(g)
    outs = []
    for C in (1, 4, NSTEPS):
        g.design_to_phi(BOXES, THETA, WIDTH)
        g.set_fields(x0)
        J, dphi = g.adjoint_run(NSTEPS, ckpt_every=C)
        outs.append((J, dphi))
    for J, dphi in outs[1:]:
        assert J == outs[0][0]
        np.testing.assert_allclose(dphi, outs[0][1], rtol=1e-9, atol=1e-12 * np.abs(outs[0][1]).max())
    # the grid ends at the final state, as after uf_run
    g.set_fields(x0)
    g.run(NSTEPS)
    ref = g.get_state("u")
    g.set_fields(x0)
    g.adjoint_run(NSTEPS, ckpt_every=4)
    np.testing.assert_array_equal(g.get_state("u"), ref)


def test_fp32_adjoint_close_to_fp64():
    grads = {}
    for prec in ("f64", "f32"):
        g = grid(prec)
        g64 = grid("f64")
        x0 = start_state(g64)
        g.design_to_phi(BOXES, THETA, WIDTH)
        g.set_fields(x0)
        J, dphi = g.adjoint_run(NSTEPS, ckpt_every=3)
        grads[prec] = g.design_vjp(BOXES, THETA, WIDTH, dphi)
    rel = np.linalg.norm(grads["f32"] - grads["f64"]) / np.linalg.norm(grads["f64"])
    assert rel <= 2e-3, (rel, grads)


def test_adjoint_matches_oracle_finite_differences():
    """The oracle's central-difference gradient of its own J (FP64, its own
    design map) against the GPU adjoint from the same initial state."""
    op = dict(PARAMS)
    o = oracle.Oracle(NX, NY, NZ, **op)
    o.set("phi", oracle.design_to_phi(NX, NY, NZ, H, BOXES, THETA.reshape(-1, 3), WIDTH))
    o.init()
    o.run(4)
    x0 = o.state()

    def oJ(theta):
        o.set("phi", oracle.design_to_phi(NX, NY, NZ, H, BOXES, theta.reshape(-1, 3), WIDTH))
        o.set_state(x0)
        o.run(NSTEPS)
        return o.objective(*BAND)

    fd, replaced = fd_reference(oJ)
    assert replaced <= 2, fd
    g = grid()
    g.design_to_phi(BOXES, THETA, WIDTH)
    g.set_fields(x0)
    J, dphi = g.adjoint_run(NSTEPS, ckpt_every=4)
    grad = g.design_vjp(BOXES, THETA, WIDTH, dphi)
    assert J == pytest.approx(oJ(THETA), rel=1e-9)
    floor = 1e-3 * np.abs(fd).max()
    assert np.all(np.abs(grad - fd) <= 1e-3 * np.abs(fd) + floor), (grad, fd)


def test_autograd_function():
    """theta -> phi -> J through the two autograd Functions, on device tensors:
    J equals the forward objective, theta.grad the adjoint gradient."""
    g = grid()
    x0 = start_state(g)
    theta = torch.tensor(THETA.reshape(-1, 3), dtype=torch.float64, requires_grad=True)
    phi = uf.design_porosity(theta, g, BOXES, WIDTH)
    assert phi.is_cuda and phi.dtype == torch.float64
    np.testing.assert_allclose(phi.detach().cpu().numpy(), g.design_to_phi(BOXES, THETA, WIDTH, set_porosity=False),
                               rtol=0, atol=0)
    J = uf.comfort_objective(phi, g, x0, NSTEPS, ckpt_every=3, band=BAND)
    J.backward()
    g.design_to_phi(BOXES, THETA, WIDTH)
    g.set_fields(x0)
    J2, dphi = g.adjoint_run(NSTEPS, ckpt_every=3, z_lo=BAND[0], z_hi=BAND[1], u_hi=BAND[2], u_lo=BAND[3])
    ref = g.design_vjp(BOXES, THETA, WIDTH, dphi)
    assert J.item() == pytest.approx(J2, rel=1e-12)
    np.testing.assert_allclose(theta.grad.numpy().ravel(), ref, rtol=1e-9, atol=1e-12)


def test_autograd_phi_gradient_on_device():
    """dJ/dphi from backward lands on the device and equals uf_adjoint_run's."""
    g = grid()
    x0 = start_state(g)
    phi = torch.tensor(g.get_state("phi"), device="cuda", requires_grad=True)
    J = uf.comfort_objective(phi, g, x0, 4, ckpt_every=2, band=BAND)
    (gphi,) = torch.autograd.grad(2.0 * J, phi)
    assert gphi.is_cuda
    g.set_porosity(phi.detach())
    g.set_fields(x0)
    _, dphi = g.adjoint_run(4, ckpt_every=2, z_lo=BAND[0], z_hi=BAND[1], u_hi=BAND[2], u_lo=BAND[3])
    np.testing.assert_allclose(gphi.cpu().numpy(), 2.0 * dphi, rtol=1e-12, atol=0)


def test_adjoint_needs_fixed_dt():
    g = uf.Grid(NX, NY, NZ, precision="f64", h=H)
    g.init_state()
    with pytest.raises(uf.UFError) as ei:
        g.adjoint_run(2)
    assert ei.value.status == uf.UF_ERR_ARG


STATE5 = ("u", "v", "w", "k", "omega")


def _small_grid():
    """8 x 8 x 8, two inflow sides (wind 30 deg), a porous block, FP64 with
    the CG tolerance at 1e-14 so that central differences resolve 1e-9."""
    n = 8
    g = uf.Grid(n, n, n, precision="f64", h=2.0, wind_dir_deg=30.0, u_ref=3.0, z_ref=10.0, z0=0.5, inflow_loglaw=1,
                ground_noslip=1, fixed_dt=0.2, cg_tol=1e-14)
    phi = np.ones((n, n, n))
    phi[0:4, 3:6, 3:6] = 0.5
    g.set_porosity(phi)
    g.init_state()
    g.run(2)
    return g


def _flat(st):
    return np.concatenate([np.asarray(st[n], dtype=np.float64).ravel() for n in STATE5])


def _unflat(x, g):
    out, o = {}, 0
    for n in STATE5:
        m = int(np.prod(g.shapes[n]))
        out[n] = x[o:o + m].reshape(g.shapes[n])
        o += m
    return out


def test_step_vjp_dense_jacobian_transpose_8cubed():
    """Every row of (dX'/dX)^T from uf_step_vjp against every column of the
    central-difference Jacobian of one FP64 step at 8^3 (2752 state values).

    The step is piecewise smooth: a semi-Lagrangian sample is trilinear, so
    linear between lattice planes with a kink where the departure point
    crosses one (a velocity of zero puts it on a plane).  The check runs at
    a generic state: the developed flow plus seeded noise, with every
    velocity at least 1e-4 m/s away from zero, far beyond the 1e-6 steps."""
    g = _small_grid()
    x0 = g.state()
    p0 = x0["p"]
    rng = np.random.default_rng(8)
    for n in ("u", "v", "w"):
        a = x0[n] + 0.02 * rng.standard_normal(x0[n].shape)
        x0[n] = np.where(np.abs(a) < 1e-4, 1e-4, a)
    for n in ("k", "omega"):
        x0[n] = x0[n] * (1.0 + 0.01 * rng.standard_normal(x0[n].shape))
    x = _flat(x0)
    N = x.size

    def step_of(xv):
        g.set_fields(dict(_unflat(xv, g), p=p0))
        g.step(stats=False)
        return _flat(g.state())

    J_fd = np.empty((N, N))
    for j in range(N):
        e = 1e-6 * max(1.0, abs(x[j]))
        xp, xm = x.copy(), x.copy()
        xp[j] += e
        xm[j] -= e
        J_fd[:, j] = (step_of(xp) - step_of(xm)) / (2 * e)
    g.set_fields(x0)
    J_ad = np.empty((N, N))
    for i in range(N):
        lam = np.zeros(N)
        lam[i] = 1.0
        J_ad[i, :] = _flat(g.step_vjp(_unflat(lam, g)))
    scale = np.abs(J_fd).max()
    err = np.abs(J_ad - J_fd)
    assert np.linalg.norm(J_ad - J_fd) <= 1e-7 * np.linalg.norm(J_fd), np.unravel_index(err.argmax(), err.shape)
    assert err.max() <= 1e-6 * scale, (np.unravel_index(err.argmax(), err.shape), err.max(), scale)


def test_step_vjp_dot_product_and_state_untouched():
    """<w, J v> by central differences against <J^T w, v> on the 24 x 20 x 10
    design grid; the grid's state is bitwise unchanged by uf_step_vjp."""
    g = grid()
    x0 = start_state(g)
    g.set_fields(x0)
    before = g.state()
    rng = np.random.default_rng(3)
    x = _flat(x0)
    v = rng.standard_normal(x.size) * (np.abs(x) + 1e-3)
    w = rng.standard_normal(x.size)
    lam_in, lam_phi = g.step_vjp(_unflat(w, g), with_phi=True)
    after = g.state()
    for f in ("u", "v", "w", "p", "k", "omega"):
        np.testing.assert_array_equal(after[f], before[f], err_msg=f)
    eps = 1e-7

    def step_of(xv):
        g.set_fields(dict(_unflat(xv, g), p=x0["p"]))
        g.step(stats=False)
        return _flat(g.state())

    jv = (step_of(x + eps * v) - step_of(x - eps * v)) / (2 * eps)
    lhs = float(np.dot(w, jv))
    rhs = float(np.dot(_flat(lam_in), v))
    assert rhs == pytest.approx(lhs, rel=1e-6), (lhs, rhs)
    # and the porosity part, against a porosity perturbation
    phi = g.get_state("phi")
    dphi = rng.standard_normal(phi.shape) * phi * (1 - phi)

    def step_phi(ph):
        g.set_porosity(ph)
        g.set_fields(x0)
        g.step(stats=False)
        return _flat(g.state())

    jp = (step_phi(phi + 1e-6 * dphi) - step_phi(phi - 1e-6 * dphi)) / 2e-6
    g.set_porosity(phi)
    assert float(np.sum(lam_phi * dphi)) == pytest.approx(float(np.dot(w, jp)), rel=1e-6)
