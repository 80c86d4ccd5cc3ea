"""Host-side arithmetic of bench.py that the GPU run relies on (no GPU):
the whole-step algorithmic traffic and the source digest of the profiled
kernels."""
import pytest

import bench


def test_step_traffic_sums_bytes_times_launches():
    kernels = {"a": {"bytes_per_launch": 100.0, "launches": 3, "total_ms": 1.0},
               "b": {"bytes_per_launch": 50.0, "launches": 2, "total_ms": 1.0}}
    r = bench.step_traffic(kernels, ms_per_step=1e-3, peak=1.0, cells=4)     # 400 B in 1 us
    assert r["bytes"] == 400.0 and r["bytes_per_cell"] == 100.0
    assert r["achieved"] == pytest.approx(400.0 / 1e-6 / 1e9) and r["frac"] == pytest.approx(r["achieved"])


def test_step_traffic_never_raises():
    assert "error" in bench.step_traffic({"a": {}}, 1.0, 1.0, 1)
    assert "error" in bench.step_traffic({"a": {"bytes_per_launch": 1.0, "launches": 1}}, 0.0, 1.0, 1)


def test_digest_covers_the_profiled_kernel_headers():
    assert len(bench.source_digest()) == 16
    assert set(bench.DIGEST_HEADERS) == {"mg_fused.cuh", "solver_kernels.cuh", "step_kernels.cuh", "uf_device.cuh"}
    # the committed ncu summaries are read (None once the device code has
    # changed since the capture, by design)
    for v in (bench.ncu_traffic("mg_down_cg_L0"), bench.fp64_flops_per_cell("mg_down_cg_L0")):
        assert v is None or v > 0
