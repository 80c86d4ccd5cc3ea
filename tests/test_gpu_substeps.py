"""Dot-product tests of every hand-written transpose, one sub-step at a time
(uf_substep), in FP64: <J v, w> = <v, J^T w> with J v from differences of
the sub-step along v and J^T w its transpose.  The difference is the
Richardson combination (4 D(e) - D(2e))/3 of central differences D, whose
e^2 terms cancel, with e per sub-step: large where the map is (bi)linear
(diffusion, projection, and drag in u for fixed phi), small where switches
(limiters, upwind sides, floors) lie close.  The advection's Selle clamp is
active at many faces of a developed flow, so any second step size straddles
some switch; it takes a plain central difference at 1e-6 instead.  Measured
relative gaps: drag 5e-13, diffusion 1e-12, projection 9.5e-12 (the two
solves' tolerance), k-omega 2.2e-11, eddy viscosity 4.8e-11, advection 7e-8
(the difference's own truncation); the bars are 10-20x those."""
import numpy as np
import pytest

from paper_2204_01117_gb300 import uf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NX, NY, NZ, H = 24, 20, 10, 2.0
BOXES = [(14.0, 22.0, 12.0, 20.0), (28.0, 36.0, 20.0, 28.0)]
THETA = np.array([9.0, 0.3, -0.4, 7.0, -0.2, 0.5])
PARAMS = dict(h=H, wind_dir_deg=30.0, u_ref=3.0, z_ref=10.0, z0=0.5, inflow_loglaw=1, ground_noslip=1,
              fixed_dt=0.25)
# step (relative to the state's scale), Richardson or plain central, bar on
# |<Jv, w> - <v, J^T w>| / max(|<Jv, w>|, |<v, J^T w>|)
SCHEME = {"eddy": (1e-5, True, 1e-9), "advect": (1e-6, False, 1e-6), "diffuse": (1e-4, True, 2e-11),
          "drag_bc": (1e-4, True, 1e-11), "project": (1e-4, True, 2e-10), "turb": (1e-6, True, 5e-10)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    uf.build()
    uf.load()


@pytest.fixture(scope="module")
def state():
    g = uf.Grid(NX, NY, NZ, precision="f64", **PARAMS)
    g.design_to_phi(BOXES, THETA, 2.0)
    g.init_state()
    g.run(5)
    x = g.state()
    x["nut"] = g.get_state("nut")
    x["phi"] = g.get_state("phi")
    g.close()
    return x


def direction(name, x, rng):
    a = x[name]
    if name == "phi":
        return rng.standard_normal(a.shape) * a * (1 - a)
    if name in ("k", "omega", "nut"):
        return rng.standard_normal(a.shape) * np.abs(a)
    return rng.standard_normal(a.shape) * (np.abs(a).max() + 1e-30)


@pytest.mark.parametrize("name", list(uf.SUBSTEPS))
def test_substep_transpose_dot_product(name, state):
    g = uf.Grid(NX, NY, NZ, precision="f64", **PARAMS)
    _, ins, outs = uf.SUBSTEPS[name]
    rng = np.random.default_rng(sum(map(ord, name)))
    x = [state[n] for n in ins]
    v = [direction(n, state, rng) for n in ins]
    w = [rng.standard_normal(g.shapes[n]) for n in outs]
    def central(eps):
        fp = g.substep(name, [a + eps * b for a, b in zip(x, v)])
        fm = g.substep(name, [a - eps * b for a, b in zip(x, v)])
        return [(p - m) / (2 * eps) for p, m in zip(fp, fm)]

    eps, richardson, bar = SCHEME[name]
    if richardson:
        d1, d2 = central(2 * eps), central(eps)
        jv = [(4 * b - a) / 3 for a, b in zip(d1, d2)]
    else:
        jv = central(eps)
    jtw = g.substep(name, x, cot=w)
    lhs = sum(float(np.sum(a * b)) for a, b in zip(jv, w))
    rhs = sum(float(np.sum(a * b)) for a, b in zip(v, jtw))
    assert abs(lhs) > 0
    err = abs(lhs - rhs) / max(abs(lhs), abs(rhs))
    print(name, lhs, rhs, err)
    assert err <= bar, (lhs, rhs, err)
    g.close()


def test_substep_forward_matches_the_step(state):
    """Chaining the sub-steps from a state reproduces one uf_step (fixed dt)."""
    g = uf.Grid(NX, NY, NZ, precision="f64", **PARAMS)
    s = state
    nut, = g.substep("eddy", [s["u"], s["v"], s["w"], s["k"], s["omega"]])
    ut = g.substep("advect", [s["u"], s["v"], s["w"]])
    u2 = g.substep("diffuse", ut + [nut])
    u3 = g.substep("drag_bc", u2 + [s["phi"]])
    u1 = g.substep("project", u3)
    k1, o1 = g.substep("turb", u1 + [s["k"], s["omega"]])
    ref = uf.Grid(NX, NY, NZ, precision="f64", **PARAMS)
    ref.set_porosity(s["phi"])
    ref.set_fields({n: s[n] for n in ("u", "v", "w", "k", "omega")})
    ref.step()
    for name, got in zip(("u", "v", "w", "k", "omega"), u1 + [k1, o1]):
        r = ref.get_state(name)
        assert np.linalg.norm(got - r) <= 1e-9 * np.linalg.norm(r), name
    g.close()
    ref.close()


def test_substep_argument_errors():
    g = uf.Grid(8, 8, 4, precision="f64", h=1.0, u_ref=2.0)      # no fixed dt
    z = [np.zeros(g.shapes[n]) for n in ("u", "v", "w")]
    with pytest.raises(uf.UFError) as ei:
        g.substep("advect", z)
    assert ei.value.status == uf.UF_ERR_ARG
