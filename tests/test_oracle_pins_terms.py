"""Pins of the oracle's k-omega terms, MacCormack limiter, staggered sampling
offsets and strain tensor (Sec. 3: the k and omega equations, P_k, Table 1;
"Discretization and Numerical Integration", which adopts Selle et al.'s
MacCormack scheme).

Each test isolates one term with a closed form that does not come from the
oracle's own code:
  * the upwind difference of a quadratic field (differs from the downwind
    and central differences by one cell),
  * the exact 7-point Laplacian of a quadratic (2 b), which separates the
    sigma* of k from the sigma of omega,
  * the strain of shear, extension, rotation and pure-strain flows,
  * a hand-worked 1D MacCormack step on a spiky field, in dyadic numbers
    (exact in FP64), where the clamp to the forward sample's corners binds,
  * the second-order Taylor closed form of MacCormack for linear fields
    carried by a linear velocity field, which fixes every half-cell offset of
    the cross-component samples.

Most checks difference two runs that share everything but the term under
test, so the other terms of the update cancel exactly.
"""
import numpy as np
import pytest


def grid(oracle_mod, nx, ny, nz, **kw):
    return oracle_mod.Oracle(nx, ny, nz, **kw)


def centres(n, h):
    return (np.arange(n) + 0.5) * h


def cell_field(nx, ny, nz, h, axis, base, b):
    """base + b * (coordinate of the cell centre along axis)^2."""
    c = [centres(nz, h)[:, None, None], centres(ny, h)[None, :, None], centres(nx, h)[None, None, :]][2 - axis]
    return np.broadcast_to(base + b * c ** 2, (nz, ny, nx)).copy(), c


def set_velocity(o, u=0.0, v=0.0, w=0.0):
    o.set("u", u)
    o.set("v", v)
    o.set("w", w)


INTERIOR = (slice(1, -1), slice(1, -1), slice(1, -1))


# ------------------------------------------------- k-omega: upwind advection --

@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_komega_upwind_advection_of_a_quadratic(oracle_mod, axis, sign):
    """Uniform velocity U along one axis carries k = k0 + b x^2.  First-order
    upwind takes the difference towards the side the flow comes from:
    U (k_i - k_{i-1})/h = U b (2 x_i - h) for U > 0 and U b (2 x_i + h) for
    U < 0 (the downwind and central differences give 2 x_i + h and 2 x_i).
    Against a run at rest the update differs by exactly -dt times that; the
    same holds for omega.  Diffusion and the omega sink are switched off
    (nu = sigma = sigma* = beta = 0); the k sink is the same in both runs."""
    nx, ny, nz, h, dt, U = 9, 8, 7, 1.5, 0.2, 1.3
    kw = dict(h=h, nu=0.0, sigma=0.0, sigma_star=0.0, beta=0.0, ground_noslip=0)
    b_k, b_o = 0.01, 0.004
    k0, x = cell_field(nx, ny, nz, h, axis, 0.5, b_k)
    om0, _ = cell_field(nx, ny, nz, h, axis, 0.3, b_o)
    runs = []
    for vel in (sign * U, 0.0):
        o = grid(oracle_mod, nx, ny, nz, **kw)
        comps = [0.0, 0.0, 0.0]
        comps[axis] = vel
        set_velocity(o, *comps)
        o.set("k", k0)
        o.set("omega", om0)
        o.dt = dt
        o.turbulence()
        runs.append((o.get("k"), o.get("omega")))
    off = -h if sign > 0 else h
    upwind = lambda b: np.broadcast_to(sign * U * b * (2 * x + off), (nz, ny, nx))
    dk = runs[0][0] - runs[1][0]
    do = runs[0][1] - runs[1][1]
    np.testing.assert_allclose(dk[INTERIOR], -dt * upwind(b_k)[INTERIOR], rtol=1e-11, atol=0)
    np.testing.assert_allclose(do[INTERIOR], -dt * upwind(b_o)[INTERIOR], rtol=1e-11, atol=0)


# ------------------------------------------------------ k-omega: diffusion --

@pytest.mark.parametrize("axis", [0, 1, 2])
def test_komega_diffusion_separates_sigma_star_and_sigma(oracle_mod, axis):
    """Fluid at rest, k = k0 + b x^2 and omega = w0 + b' x^2: the 7-point
    Laplacian of a quadratic is exactly 2 b, so against a run without
    diffusion (nu = sigma = sigma* = 0) k gains dt (nu + sigma* nu_t) 2 b and
    omega dt (nu + sigma nu_t) 2 b' (Table 1: sigma* = 0.6, sigma = 0.5).
    With k/omega above the viscosity limiter nu_t is the limiter's value
    h^2/(6 dt) - nu; below it, nu_t = k/omega (no strain)."""
    nx, ny, nz, h, dt = 8, 7, 6, 1.0, 0.1
    d = oracle_mod.DEFAULTS
    nu, sig, sig_s = d["nu"], d["sigma"], d["sigma_star"]
    b_k, b_o = 0.02, 0.01
    for k_base, o_base, limited in ((4.0, 1.0, True), (0.1, 2.0, False)):
        k0, _ = cell_field(nx, ny, nz, h, axis, k_base, b_k)
        om0, _ = cell_field(nx, ny, nz, h, axis, o_base, b_o)
        out = []
        for on in (True, False):
            kw = dict(h=h) if on else dict(h=h, nu=0.0, sigma=0.0, sigma_star=0.0)
            o = grid(oracle_mod, nx, ny, nz, **kw)
            set_velocity(o)
            o.set("k", k0)
            o.set("omega", om0)
            o.dt = dt
            o.turbulence()
            out.append((o.get("k"), o.get("omega")))
        if limited:
            assert np.all(k0 / om0 > h * h / (6 * dt) - nu)
            nut = h * h / (6 * dt) - nu
        else:
            assert np.all(k0 / om0 < h * h / (6 * dt) - nu)
            nut = k0 / om0
        dk = out[0][0] - out[1][0]
        do = out[0][1] - out[1][1]
        ek = np.broadcast_to(dt * (nu + sig_s * nut) * 2 * b_k, (nz, ny, nx))
        eo = np.broadcast_to(dt * (nu + sig * nut) * 2 * b_o, (nz, ny, nx))
        np.testing.assert_allclose(dk[INTERIOR], ek[INTERIOR], rtol=1e-10, atol=0)
        np.testing.assert_allclose(do[INTERIOR], eo[INTERIOR], rtol=1e-10, atol=0)


# -------------------------------------------------------- k-omega: sources --

@pytest.mark.parametrize("gamma", [0.02, 0.2])
def test_komega_production_sources_of_shear(oracle_mod, gamma):
    """Shear u = gamma y: S_xy = gamma/2, S_ij S_ij = gamma^2/2 at every cell.
    Against the same k, omega at rest, k gains dt P_k = dt 2 nu_t |S|^2 =
    dt nu_t gamma^2 and omega gains dt 2 alpha |S|^2 = dt alpha gamma^2
    (Sec. 3, Table 1).  nu_t = k / max(omega, C_lim |S| / sqrt(C_mu/2)):
    the small shear leaves omega~ = omega, the large one takes the strain
    branch C_lim gamma / sqrt(C_mu).  k and omega hold the inlet values, so
    advection and diffusion vanish in both runs."""
    nx, ny, nz, h, dt = 6, 9, 5, 2.0, 0.1
    d = oracle_mod.DEFAULTS
    out = []
    for g in (gamma, 0.0):
        o = grid(oracle_mod, nx, ny, nz, h=h, u_ref=5.0)
        y = centres(ny, h)
        set_velocity(o, u=np.broadcast_to((g * y)[None, :, None], (nz, ny, nx + 1)))
        o.set("k", o.inlet_k)
        o.set("omega", o.inlet_omega)
        o.dt = dt
        o.turbulence()
        out.append((o.get("k"), o.get("omega"), o.inlet_k, o.inlet_omega))
    k, om = out[0][2], out[0][3]
    strain_bound = d["C_lim"] * gamma / np.sqrt(d["C_mu"])
    if gamma == 0.02:
        assert om > strain_bound
        nut = k / om
    else:
        assert om < strain_bound
        nut = k * np.sqrt(d["C_mu"]) / (d["C_lim"] * gamma)
    assert nut < h * h / (6 * dt) - d["nu"]
    np.testing.assert_allclose(out[0][0] - out[1][0], dt * nut * gamma ** 2, rtol=1e-11, atol=0)
    np.testing.assert_allclose(out[0][1] - out[1][1], dt * d["alpha"] * gamma ** 2, rtol=1e-11, atol=0)


# ---------------------------------------------------------- strain tensor --

@pytest.mark.parametrize("flow,s2", [
    ("ext_x", 1.0), ("ext_y", 1.0), ("ext_z", 1.0),     # one diagonal entry gamma
    ("rotation", 0.0),                                  # antisymmetric gradient: no strain
    ("pure_strain", 2.0),                               # S_xy = S_yx = gamma
])
def test_strain_of_extension_rotation_and_pure_strain(oracle_mod, flow, s2):
    """S_ij S_ij = s2 gamma^2 for: u = gamma x (S_xx = gamma), v = gamma y,
    w = gamma z; the rotation u = gamma y, v = -gamma x (S = 0); the pure
    strain u = gamma y, v = gamma x (S_xy = S_yx = gamma).  The eddy
    viscosity then reads it back: nu_t = k sqrt(C_mu/2) / (C_lim sqrt(s2)
    gamma) on the strain branch, k/omega without strain."""
    nx, ny, nz, h, g, dt = 7, 6, 5, 1.0, 0.1, 0.01
    d = oracle_mod.DEFAULTS
    o = grid(oracle_mod, nx, ny, nz, h=h)
    xu = np.arange(nx + 1) * h
    yv = np.arange(ny + 1) * h
    zw = np.arange(nz + 1) * h
    yc, xc = centres(ny, h), centres(nx, h)
    U = np.zeros((nz, ny, nx + 1))
    V = np.zeros((nz, ny + 1, nx))
    W = np.zeros((nz + 1, ny, nx))
    if flow == "ext_x":
        U += g * xu[None, None, :]
    elif flow == "ext_y":
        V += g * yv[None, :, None]
    elif flow == "ext_z":
        W += g * zw[:, None, None]
    elif flow == "rotation":
        U += g * yc[None, :, None]
        V -= g * xc[None, None, :]
    else:
        U += g * yc[None, :, None]
        V += g * xc[None, None, :]
    set_velocity(o, U, V, W)
    k, om = 0.5, 0.1
    o.set("k", k)
    o.set("omega", om)
    o.dt = dt
    nut = o.eddy_viscosity()
    if s2 > 0:
        expect = k * np.sqrt(d["C_mu"] / 2) / (d["C_lim"] * np.sqrt(s2) * g)
    else:
        expect = k / om
    np.testing.assert_allclose(nut, expect, rtol=1e-12)


# ------------------------------------------------------ MacCormack limiter --

def _carry_along_x(oracle_mod, vline, c):
    """v(x) (uniform in y, z) carried by the uniform u = 1 m/s at Courant
    number c (h = 1, dt = c); returns v* on an interior row of v faces."""
    nx, ny, nz = len(vline), 4, 3
    o = grid(oracle_mod, nx, ny, nz, h=1.0)
    o.set("u", 1.0)
    o.set("v", np.broadcast_to(np.asarray(vline, dtype=np.float64), (nz, ny + 1, nx)))
    o.set("w", 0.0)
    o.dt = c
    o.advect()
    v = o.get("v")
    # every interior row holds the same values
    assert np.all(v[:, 1:ny, :] == v[0, 1, :])
    return v[0, 1, :]


def test_maccormack_selle_clamp_worked_example(oracle_mod):
    """A 1D step by hand at c = 1/4 on v = (0, 0, 0, 1, 0, 2, 0, 0):
      forward   v^_i = v_{i-1}/4 + 3 v_i/4      = (0, 0, 0, 3/4, 1/4, 3/2, 1/2, 0)
      backward  v_i  = 3 v^_i/4 + v^_{i+1}/4    = (0, 0, 3/16, 5/8, 9/16, 5/4, 3/8, 0)
      corrected v^ + (v - v)/2                  = (0, 0, -3/32, 15/16, -1/32, 15/8, 5/16, 0)
    then clamped to [min, max](v_{i-1}, v_i), the corners of the forward
    sample: faces 2 and 4 bind at 0.  Clamping to the backward sample's
    corners would give 3/4 and 3/2 at faces 3 and 5, reverting to the
    forward value would give 1/4 at face 4, and no limiter -3/32 and -1/32.
    Every number is dyadic, so FP64 reproduces it exactly."""
    got = _carry_along_x(oracle_mod, [0, 0, 0, 1, 0, 2, 0, 0], 0.25)
    expect = np.array([0, 0, 0, 15 / 16, 0, 15 / 8, 5 / 16, 0])
    np.testing.assert_array_equal(got, expect)


@pytest.mark.parametrize("c", [0.25, 0.5, 0.7])
def test_maccormack_result_stays_inside_forward_corners(oracle_mod, c):
    """For 0 < c < 1 the forward sample of face i uses faces i-1 and i: the
    clamped result lies in their range on any data (a maximum principle that
    unlimited MacCormack violates), and it touches a bound somewhere on
    random data, where the unlimited correction overshoots."""
    vline = np.random.default_rng(11).uniform(-1.0, 1.0, 24)
    got = _carry_along_x(oracle_mod, vline, c)
    lo = np.minimum(vline[:-1], vline[1:])
    hi = np.maximum(vline[:-1], vline[1:])
    assert np.all(got[1:] >= lo) and np.all(got[1:] <= hi)
    assert np.any((got[1:] == lo) | (got[1:] == hi))


# ------------------------------------------- staggered cross-component offsets

def test_maccormack_linear_velocity_field_closed_form(oracle_mod):
    """Velocity a(x) = a0 + M x with a generic M (every entry nonzero).  For
    linear data, trilinear samples are exact, and MacCormack with the Euler
    backtrace evaluated at the lattice point gives, for component q at its
    own lattice point x (a = a(x), g = row q of M):
        phi* = phi - dt g.a + dt^2/2 g.M.a
    (forward: phi - dt g.a; the backward sample of that linear field misses
    phi by dt^2 g.M.a; half of it is added back).  The cross-component
    samples enter through a: a half-cell error in any of their offsets moves
    the result by dt M[q][c] M[c][axis] h / 2.  Points two cells from the
    boundary: no sample is clamped; the displacements are 0.3-0.7 of a cell,
    so the Selle clamp does not fire."""
    nx, ny, nz, h, dt = 14, 12, 10, 1.0, 0.5
    a0 = np.array([1.0, 0.9, 0.8])
    M = np.array([[0.011, -0.017, 0.013],
                  [0.019, -0.007, -0.012],
                  [-0.014, 0.016, 0.009]])
    i = lambda n: np.arange(n, dtype=np.float64)
    # physical positions of the three lattices, arrays shaped (z, y, x)
    pos = {
        "u": np.meshgrid((i(nz) + 0.5) * h, (i(ny) + 0.5) * h, i(nx + 1) * h, indexing="ij"),
        "v": np.meshgrid((i(nz) + 0.5) * h, i(ny + 1) * h, (i(nx) + 0.5) * h, indexing="ij"),
        "w": np.meshgrid(i(nz + 1) * h, (i(ny) + 0.5) * h, (i(nx) + 0.5) * h, indexing="ij"),
    }
    def vel(name):
        z, y, x = pos[name]
        X = np.stack([x, y, z], axis=-1)
        return a0 + X @ M.T          # a(x) at every point of that lattice
    o = grid(oracle_mod, nx, ny, nz, h=h)
    for q, name in enumerate("uvw"):
        o.set(name, vel(name)[..., q])
    o.dt = dt
    o.advect()
    for q, name in enumerate("uvw"):
        a = vel(name)
        disp = dt * a / h
        assert np.all((disp > 0.3) & (disp < 0.7))
        g = M[q]
        expect = a[..., q] - dt * (a @ g) + 0.5 * dt * dt * (a @ (g @ M))
        got = o.get(name)
        s = (slice(2, -2),) * 3
        np.testing.assert_allclose(got[s], expect[s], rtol=0, atol=1e-12)
