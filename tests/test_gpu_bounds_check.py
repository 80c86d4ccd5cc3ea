"""The debug build with device-side bounds checks (-DUF_BOUNDS_CHECK).

In that build every global index the kernels form through the index
helpers (the u, v, cell/w lattices and the multigrid levels) is checked
against its array; an index outside it is recorded, the access is redirected
to element 0, and the call returns UF_ERR_BOUNDS.  Here the checked library
runs the main paths (single grids in FP32 and FP64 with every multigrid
transfer and the cluster V-cycle, the unfused sub-step kernels, the other
preconditioners, the adjoint, the batch, the allocation-free solve, the
design map and the mesh resolver) on ragged grids in a child process, which
loads it through UF_LIBRARY; every call must come back clean.
"""
import os
import subprocess
import sys
import textwrap

import pytest

from paper_2204_01117_gb300 import uf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import os, sys
    import numpy as np
    sys.path.insert(0, os.environ["UF_ROOT"])
    import torch
    from paper_2204_01117_gb300 import layouts, uf
    uf.load()
    assert os.path.samefile(uf.CHECKED_LIB_PATH, os.environ["UF_LIBRARY"])
    assert uf.load().uf_bounds_checked() == 1

    def grid(sc, precision, **kw):
        g = uf.Grid(sc.nx, sc.ny, sc.nz, precision=precision, **sc.params(), **kw)
        g.set_porosity(sc.phi.astype(g.np_dtype))
        g.init_state()
        return g

    sc = layouts.urban_block(70, 54, 19, h=2.0, seed=2, wind_dir_deg=200.0)
    for precision in ("f32", "f64"):
        for kw in (dict(), dict(mg_transfer="constant"), dict(mg_smoother="rbgs")):
            g = grid(sc, precision, **kw)
            g.run(3)
            g.close()
    g = grid(sc, "f32")
    g.set_tuning(coarse_start=1)           # the cluster V-cycle, where the device runs it
    g.run(2)
    g.set_tuning(unfused=uf.UNFUSED_ALL)   # the sub-step kernels the fused ones replace
    g.run(2)
    g.close()
    for pc in ("ai1", "ai2", "jacobi"):
        g = grid(sc, "f32", precond=pc, cg_max_iter=4000)
        g.run(1)
        g.close()
    b = np.random.default_rng(0).standard_normal((sc.nz, sc.ny, sc.nx)).astype(np.float32)
    g = uf.Grid(sc.nx, sc.ny, sc.nz, precision="f32")
    g.set_state("p", 0.0)
    g.poisson_solve(b)
    g.close()
    bd = torch.from_numpy(b).cuda()
    pd = torch.zeros_like(bd)
    uf.poisson_solve_static(bd, pd)

    d = layouts.design_lattice(nx=40, ny=36, nz=14, steps=6, ckpt_every=2)
    g = uf.Grid(d.nx, d.ny, d.nz, precision="f32", **d.params())
    theta = np.asarray(d.theta, dtype=np.float64).reshape(-1)
    g.design_to_phi(d.boxes, theta, d.width)
    g.init_state()
    J, dphi = g.adjoint_run(d.steps, ckpt_every=d.ckpt_every)
    g.design_vjp(d.boxes, theta, d.width, dphi)
    g.free_adjoint_workspace()
    g.close()

    insts = [layouts.urban_block(n, m, k, h=2.0, seed=s) for (n, m, k, s) in ((48, 40, 16, 1), (36, 30, 12, 2))]
    bt = uf.Batch([dict(nx=x.nx, ny=x.ny, nz=x.nz, **x.params()) for x in insts], precision="f32")
    for x, gi in zip(insts, bt.grids):
        gi.set_porosity(x.phi.astype(np.float32))
        gi.init_state()
    bt.run(3)
    bt.close()

    tris, objs = layouts.mesh_city(37, 29, 13, 2.0, n_buildings=5, n_trees=3, seed=0)
    g = uf.Grid(37, 29, 13, h=2.0, precision="f32")
    g.mesh_to_phi(tris, objs, sub=3)
    g.close()
    print("clean")
""")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_the_default_build_has_no_bounds_checks():
    uf.build()
    assert uf.load().uf_bounds_checked() == 0


def test_bounds_checked_build_runs_the_main_paths_clean():
    path = uf.build(checked=True)
    env = dict(os.environ, UF_LIBRARY=path, UF_ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0 and "clean" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
