"""uf_poisson_solve_static: the pressure solve for callers that cannot allocate.

Callers embedded in a host application or another framework that owns the
device memory (or must never hit the allocator mid-run) cannot hand the
library a workspace.  The static entry point keeps its scratch in a fixed
array inside the library instead; here it must give the same pressure as the
workspace-based solve (uf_poisson_solve on an AI1-preconditioned grid) and
the FP64 oracle's CG on two calls in a row, through the C ABI, work on the
default arguments of the Python binding, and refuse grids above its stated
size.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2204_01117_gb300 import uf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    uf.build()
    uf.load()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_static_solve_matches_workspace_solve_twice():
    nx, ny, nz, deg = 45, 37, 11, 30.0
    grid = uf.Grid(nx, ny, nz, precision="f32", wind_dir_deg=deg, precond="ai1", cg_tol=1e-7, cg_max_iter=5000)
    stream = torch.cuda.Stream()
    for seed in (1, 2):        # two calls in a row share the same scratch
        b = np.random.default_rng(seed).standard_normal((nz, ny, nx)).astype(np.float32)
        grid.set_state("p", 0.0)
        it_ref, _ = grid.poisson_solve(b)
        ref = grid.get_state("p")
        bd = torch.from_numpy(b).cuda()
        pd = torch.zeros_like(bd)
        torch.cuda.synchronize()
        it, r = uf.poisson_solve_static(bd, pd, wind_dir_deg=deg, tol=1e-7, max_iter=5000, stream=stream)
        assert r <= 1e-7
        assert abs(it - it_ref) <= 2, (it, it_ref)
        assert rel(pd.cpu().numpy(), ref) <= 5e-5


def test_static_solve_matches_oracle_twice():
    """Against the exact discrete solution (the oracle's plain FP64 CG to
    1e-13), within the FP32 solution bound of the other pressure solves."""
    import oracle
    nx, ny, nz, deg = 45, 37, 11, 30.0
    o = oracle.Oracle(nx, ny, nz, wind_dir_deg=deg)
    stream = torch.cuda.Stream()
    for seed in (3, 4):
        b = np.random.default_rng(seed).standard_normal((nz, ny, nx))
        ref, _, _ = o.cg(b, tol=1e-13)
        bd = torch.from_numpy(b.astype(np.float32)).cuda()
        pd = torch.zeros_like(bd)
        torch.cuda.synchronize()
        it, r = uf.poisson_solve_static(bd, pd, wind_dir_deg=deg, tol=1e-7, max_iter=5000, stream=stream)
        assert r <= 1e-7
        assert rel(pd.cpu().numpy(), ref) <= 5e-5, (seed, it)


def test_static_solve_default_stream():
    """No stream argument: the binding runs the solve on a created stream of
    the current device, after the work queued on the current stream."""
    nx, ny, nz = 24, 20, 9
    b = np.random.default_rng(5).standard_normal((nz, ny, nx)).astype(np.float32)
    bd = torch.from_numpy(b).cuda()
    pd = torch.zeros_like(bd)
    pd.fill_(0.0)                      # queued on the current stream before the call
    it, r = uf.poisson_solve_static(bd, pd)
    assert r <= 1e-7 and it > 0
    grid = uf.Grid(nx, ny, nz, precision="f32", wind_dir_deg=0.0, precond="ai1", cg_tol=1e-7, cg_max_iter=5000)
    grid.set_state("p", 0.0)
    grid.poisson_solve(b)
    assert rel(pd.cpu().numpy(), grid.get_state("p")) <= 5e-5


def test_static_solve_rejects_oversize_grid():
    b = torch.zeros((100, 100, 100), dtype=torch.float32, device="cuda")   # 1e6 cells > 800000
    p = torch.zeros_like(b)
    with pytest.raises(uf.UFError) as ei:
        uf.poisson_solve_static(b, p)
    assert ei.value.status == uf.UF_ERR_ARG
    assert "at most 800000" in str(ei.value)
