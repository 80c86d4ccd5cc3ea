"""C-ABI library: builds, loads without a GPU, exports every declared symbol,
and validates descriptions on the host."""
import ctypes

import pytest

from paper_2204_01117_gb300 import uf


@pytest.fixture(scope="module")
def lib():
    uf.build()
    return uf.load()


def test_exports_every_declared_symbol(lib):
    names = uf.declared_functions()
    assert len(names) >= 16
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    for n in ("uf_create_grid", "uf_set_porosity", "uf_step", "uf_run", "uf_objective"):
        assert n in names


def test_default_desc_paper_constants(lib):
    d = uf.default_desc()
    assert (d.C_mu, d.alpha, d.beta, d.sigma, d.sigma_star) == (0.09, 0.52, 0.0708, 0.5, 0.6)
    assert d.C_lim == 7.0 / 8.0
    assert (d.a, d.b, d.e, d.Cd) == (0.62, 2.5, 1e-10, 1.0)
    assert d.precond == uf.PRECOND["mg"] and d.cg_tol == 0.0 and d.cg_max_iter == 200
    assert d.mg_smoother == uf.SMOOTHER["cheby"]
    assert d.ai_omega == 1.65 and d.cfl == 0.5


@pytest.mark.parametrize("bad,msg", [
    (dict(nx=1), "nx"), (dict(h=0.0), "h must"), (dict(precision=7), "precision"),
    (dict(u_ref=0.0), "u_ref"), (dict(precond=9), "preconditioner"), (dict(cg_tol=-1.0), "cg_tol"), (dict(mg_smoother=5), "smoother"),
    (dict(ai_omega=2.0), "ai_omega"), (dict(inflow_loglaw=1, z0=0.0), "log law"),
])
def test_invalid_descriptions_rejected_on_host(lib, bad, msg):
    d = uf.default_desc(**bad)
    assert uf.workspace_bytes(d) == 0
    assert msg in uf.last_error()


def test_workspace_size_scales(lib):
    small = uf.workspace_bytes(uf.default_desc(nx=64, ny=32, nz=16))
    big = uf.workspace_bytes(uf.default_desc(nx=256, ny=256, nz=64))
    f64 = uf.workspace_bytes(uf.default_desc(nx=256, ny=256, nz=64, precision="f64"))
    assert 0 < small < big < f64
    # ~25 cell-sized FP32 arrays plus multigrid levels for the 4.2M-cell grid
    assert 80 * 4194304 < big < 140 * 4194304


def test_null_arguments_are_errors(lib):
    h = ctypes.c_void_p()
    d = uf.default_desc()
    assert lib.uf_create_grid(ctypes.byref(d), None, 0, None, ctypes.byref(h)) == uf.UF_ERR_ARG
    assert lib.uf_step(None, None) == uf.UF_ERR_ARG
    assert lib.uf_destroy(None) == uf.UF_ERR_ARG
    assert lib.uf_last_step_launches(None) == 0


def _descs(*params, precision="f32"):
    arr = (uf.GridDesc * len(params))()
    for i, p in enumerate(params):
        arr[i] = uf.default_desc(precision=precision, **p)
    return arr


def test_batch_workspace_is_sum_of_grids_plus_tables(lib):
    params = [dict(nx=96, ny=96, nz=32), dict(nx=128, ny=64, nz=40, wind_dir_deg=135.0), dict(nx=33, ny=45, nz=9)]
    descs = _descs(*params)
    total = lib.uf_batch_workspace_bytes(len(params), descs)
    grids = sum(uf.workspace_bytes(descs[i]) for i in range(len(params)))
    assert grids < total < grids + len(params) * 256 + 64 * 1024 + 4096 * len(params) + 200 * 1024


@pytest.mark.parametrize("case,msg", [
    ("empty", "batch size"), ("too_many", "batch size"), ("mixed_precision", "precision"),
    ("not_mg", "MG preconditioner"), ("mixed_smoother", "smoother"), ("bad_instance", "instance 1"),
])
def test_batch_descriptions_rejected_on_host(lib, case, msg):
    base = dict(nx=32, ny=16, nz=8)
    if case == "empty":
        n, descs = 0, _descs(base)
    elif case == "too_many":
        n, descs = 65, _descs(*([base] * 65))
    elif case == "mixed_precision":
        descs = _descs(base, base)
        descs[1] = uf.default_desc(precision="f64", **base)
        n = 2
    elif case == "not_mg":
        n, descs = 2, _descs(base, dict(base, precond=uf.PRECOND["ai1"]))
    elif case == "mixed_smoother":
        n, descs = 2, _descs(base, dict(base, mg_smoother=uf.SMOOTHER["rbgs"]))
    else:
        n, descs = 2, _descs(base, dict(base, nx=1))
    assert lib.uf_batch_workspace_bytes(n, descs) == 0
    assert msg in uf.last_error()


def test_batch_null_arguments_are_errors(lib):
    descs = _descs(dict(nx=32, ny=16, nz=8))
    h = ctypes.c_void_p()
    assert lib.uf_batch_create(1, descs, None, 0, None, ctypes.byref(h)) == uf.UF_ERR_ARG
    assert lib.uf_batch_create(1, descs, ctypes.c_void_p(256), 16, None, ctypes.byref(h)) == uf.UF_ERR_NOMEM
    assert lib.uf_batch_run(None, 1, None) == uf.UF_ERR_ARG
    assert lib.uf_batch_grid(None, 0, ctypes.byref(h)) == uf.UF_ERR_ARG
    assert lib.uf_batch_autotune(None, 1, None) == uf.UF_ERR_ARG
    assert lib.uf_get_tuning(None, None, None) == uf.UF_ERR_ARG
    assert lib.uf_set_tuning(None, None) == uf.UF_ERR_ARG
    assert lib.uf_autotune(None, 1, None, None) == uf.UF_ERR_ARG


def test_paper_stop_rule_needs_a_simple_preconditioner(lib):
    assert uf.workspace_bytes(uf.default_desc(precond="mg", cg_stop_rule="paper")) == 0
    assert "App. A.3" in uf.last_error()
    assert uf.workspace_bytes(uf.default_desc(precond="ai2", cg_stop_rule="paper")) > 0
    assert uf.workspace_bytes(uf.default_desc(cg_stop_rule=2)) == 0


def test_checkpoint_calls_declared():
    for name in ("uf_state_bytes", "uf_save_state", "uf_load_state"):
        assert name in uf.declared_functions()
