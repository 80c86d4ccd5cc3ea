"""Checkpoint and resume: a run restored with uf_load_state continues bit
for bit as the uninterrupted run, the pressure history (the extrapolated
guess of the next solve and the pressure held in twice the working
precision) included; restoring only the fields (uf_set_fields) restarts
that history and is not bitwise the same."""
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


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_resume_equals_uninterrupted_run(precision):
    sc = layouts.urban_block(48, 40, 16, h=2.0, seed=2, wind_dir_deg=20.0)
    g = uf.Grid(sc.nx, sc.ny, sc.nz, precision=precision, **sc.params())
    g.set_porosity(sc.phi.astype(g.np_dtype))
    g.init_state()
    g.run(5)
    ck = g.save_checkpoint()
    fields = g.state()
    g.run(7)
    ref = g.state()
    g.load_checkpoint(ck)
    g.run(7)
    for n in NAMES:
        assert np.array_equal(g.get_state(n), ref[n]), n
    # the fields alone restart the pressure history
    g.set_fields(fields)
    g.run(7)
    assert not all(np.array_equal(g.get_state(n), ref[n]) for n in NAMES)
    # an odd number of steps before the save: the k/omega buffer parity
    g.load_checkpoint(ck)
    g.run(3)
    ck2 = g.save_checkpoint()
    g.run(4)
    ref2 = g.state()
    g.load_checkpoint(ck2)
    g.run(4)
    for n in NAMES:
        assert np.array_equal(g.get_state(n), ref2[n]), n
    g.close()


def test_checkpoint_buffer_checks():
    g = uf.Grid(24, 20, 8, precision="f32")
    with pytest.raises(uf.UFError) as e:
        g.save_checkpoint()
    assert e.value.status == uf.UF_ERR_STATE
    g.init_state()
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(uf.UFError) as e:
        uf.check(g.lib.uf_save_state(g._h, small.data_ptr(), 64))
    assert e.value.status == uf.UF_ERR_NOMEM
    g.close()
