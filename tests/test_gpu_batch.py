"""Batched execution (include/uf.h, "Batched execution") and launch tuning:
every instance of a batch computes bit for bit what it computes alone, for
uneven sizes, wind directions and time-step modes; tuning changes speed,
not results beyond the order of FP64 partial sums."""
import numpy as np
import pytest

import oracle
from paper_2204_01117_gb300 import layouts, uf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS6 = ("u", "v", "w", "p", "k", "omega")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    uf.build()
    uf.load()


def instances():
    """Uneven sizes (ragged tiles), four wind directions, CFL and fixed dt."""
    specs = [(48, 40, 12, 0.0, 0, 3.0), (64, 32, 16, 135.0, 1, 5.0), (33, 45, 9, 300.0, 2, 2.0),
             (40, 24, 20, 90.0, 3, 4.0)]
    out = []
    for i, (nx, ny, nz, deg, seed, speed) in enumerate(specs):
        sc = layouts.scaled_urban_block(nx, ny, nz, seed=seed, wind_dir_deg=deg, u_ref=speed)
        params = dict(nx=nx, ny=ny, nz=nz, **sc.params())
        if i == 3:
            params["fixed_dt"] = 0.3
        out.append((sc, params))
    return out


def solo(sc, params, precision):
    p = dict(params)
    nx, ny, nz = p.pop("nx"), p.pop("ny"), p.pop("nz")
    g = uf.Grid(nx, ny, nz, precision=precision, **p)
    g.set_porosity(sc.phi.astype(g.np_dtype))
    return g


def batch_of(inst, precision):
    b = uf.Batch([p for _, p in inst], precision=precision)
    for (sc, _), g in zip(inst, b.grids):
        g.set_porosity(sc.phi.astype(g.np_dtype))
    return b


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_batch_equals_solo_bitwise(precision):
    inst = instances()
    b = batch_of(inst, precision)
    for g in b.grids:
        g.init_state()
    stats = b.run(5)
    fixed, per_iter = b.launch_counts()
    assert fixed > 0 and per_iter > 0
    for (sc, params), gb, sb in zip(inst, b.grids, stats):
        gs = solo(sc, params, precision)
        gs.init_state()
        ss = gs.run(5)
        assert sb.status == 0 and sb.cg_iters == ss.cg_iters and sb.dt == ss.dt
        for f in FIELDS6:
            np.testing.assert_array_equal(gb.get_state(f), gs.get_state(f), err_msg=f)


def test_batch_runs_continue_and_interleave_with_solo_steps():
    """Parity of the k/omega buffers survives odd run lengths and single
    steps of one instance between batch runs."""
    inst = instances()[:3]
    b = batch_of(inst, "f32")
    solos = [solo(sc, p, "f32") for sc, p in inst]
    for gb, gs in zip(b.grids, solos):
        gb.init_state()
        gs.init_state()
    b.run(3)
    b.grids[1].step()
    b.run(2)
    for i, gs in enumerate(solos):
        gs.run(6 if i == 1 else 5)
        for f in FIELDS6:
            np.testing.assert_array_equal(b.grids[i].get_state(f), gs.get_state(f), err_msg=f"{i} {f}")


def test_batch_instance_matches_oracle():
    sc, params = instances()[1]
    b = batch_of([(sc, params)], "f32")
    o = oracle.Oracle(sc.nx, sc.ny, sc.nz, **sc.params())
    o.set("phi", sc.phi)
    o.init()
    g = b.grids[0]
    g.set_fields(o.state())
    b.run(1)
    o.step()
    for f in FIELDS6:
        ref = o.get(f)
        e = np.linalg.norm(g.get_state(f).astype(np.float64) - ref) / max(np.linalg.norm(ref), 1e-300)
        assert e <= 1e-5, (f, e)


def test_batch_needs_state_for_every_instance():
    inst = instances()[:2]
    b = batch_of(inst, "f32")
    b.grids[0].init_state()
    with pytest.raises(uf.UFError) as ei:
        b.run(1)
    assert ei.value.status == uf.UF_ERR_STATE


def test_tuning_keeps_state_and_results():
    sc, params = instances()[0]
    g = solo(sc, params, "f32")
    g.init_state()
    g.run(2)
    before = g.state()
    t, n_levels = g.get_tuning()
    assert t["tail_level"] >= 1 and all(z >= 2 and z % 2 == 0 for z in t["march_zc"][:t["tail_level"]])
    chosen, ms = g.autotune(reps=2)
    assert ms > 0 and chosen["tail_level"] >= t["tail_level"]
    after = g.state()
    for f in FIELDS6:
        np.testing.assert_array_equal(after[f], before[f], err_msg=f)
    # a different tuning gives the same step up to the order of FP64 sums
    g2 = solo(sc, params, "f32")
    g2.set_fields(before)
    g2.set_tuning(tail_level=n_levels - 1, march_zc=[2] * 16)
    assert g2.get_tuning()[0]["tail_level"] == n_levels - 1
    g.set_tuning()        # back to automatic
    g.run(1)
    g2.run(1)
    for f in FIELDS6:
        a, r = g2.get_state(f).astype(np.float64), g.get_state(f).astype(np.float64)
        assert np.linalg.norm(a - r) <= 1e-5 * max(np.linalg.norm(r), 1e-30), f
    with pytest.raises(uf.UFError):
        g.set_tuning(march_zc=[3])


def test_batch_autotune_then_equals_solo_with_same_tuning():
    inst = instances()
    b = batch_of(inst, "f32")
    classes = b.autotune(reps=1)
    assert 1 <= classes <= len(inst)
    for g in b.grids:
        g.init_state()
    b.run(3)
    for (sc, params), gb in zip(inst, b.grids):
        gs = solo(sc, params, "f32")
        t, _ = gb.get_tuning()
        gs.set_tuning(**t)
        gs.init_state()
        gs.run(3)
        for f in FIELDS6:
            np.testing.assert_array_equal(gb.get_state(f), gs.get_state(f), err_msg=f)


def test_grids_with_different_tails_coexist():
    """The tail kernel's shared-memory limit is per kernel: creating a grid
    with a smaller tail must not break the graphs of an earlier grid with a
    larger one."""
    big = uf.Grid(48, 40, 12, precision="f32")
    small = uf.Grid(24, 20, 8, precision="f32")
    assert big.get_tuning()[0]["tail_level"] >= 1
    big.init_state()
    small.init_state()
    big.run(2)
    small.run(2)
