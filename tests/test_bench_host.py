"""Host-side arithmetic of bench.py that the GPU run relies on (no GPU):
the whole-step algorithmic traffic and the source digest of the profiled
kernels."""
import os

import pytest

import bench


def test_step_traffic_sums_bytes_times_launches():
    # profiled step with 4 CG iterations: "cg" ran once per iteration, "pre"
    # once per iteration plus one set-up launch, "fix" twice per step
    kernels = {"cg": {"bytes_per_launch": 10.0, "launches": 4}, "pre": {"bytes_per_launch": 1.0, "launches": 5},
               "fix": {"bytes_per_launch": 100.0, "launches": 2}}
    r = bench.step_traffic(kernels, prof_iters=4, mean_iters=2.5, ms_per_step=1e-3, peak=1.0, cells=4)
    fixed, per_iter = 1.0 + 200.0, 11.0
    assert r["fixed_bytes_per_cell"] == fixed / 4 and r["per_cg_iteration_bytes_per_cell"] == per_iter / 4
    assert r["bytes"] == fixed + 2.5 * per_iter
    assert r["achieved"] == (fixed + 2.5 * per_iter) / 1e-6 / 1e9


def test_dominant_kernel_weights_cg_kernels_by_the_mean_iterations():
    # profiled step with 4 CG iterations; the timed steps averaged 2.5: "cg"
    # (0.3 ms per launch, once per iteration) takes 0.75 ms per average step,
    # "fix" (one 1.0 ms launch) 1.0 ms -- although "cg" led the profiled step
    kernels = {"cg": {"total_ms": 1.2, "launches": 4}, "fix": {"total_ms": 1.0, "launches": 1}}
    name, _, ms, share = bench.dominant_kernel(kernels, prof_iters=4, mean_iters=2.5)
    assert name == "fix" and ms == 1.0 and abs(share - 1.0 / 1.75) < 1e-12
    name, _, ms, _ = bench.dominant_kernel(kernels, prof_iters=4, mean_iters=4.0)
    assert name == "cg" and abs(ms - 1.2) < 1e-12


def test_step_traffic_never_raises():
    assert "error" in bench.step_traffic({"a": {}}, 1, 1.0, 1.0, 1.0, 1)
    assert "error" in bench.step_traffic({"a": {"bytes_per_launch": 1.0, "launches": 1}}, 1, 1.0, 0.0, 1.0, 1)


def test_digest_ignores_comments_but_not_code(tmp_path, monkeypatch):
    import shutil
    src = os.path.join(bench.ROOT, "paper_2204_01117_gb300", "csrc")
    dst = tmp_path / "paper_2204_01117_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.DIGEST_HEADERS:
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.source_digest()
    with open(dst / "mg_fused.cuh", "a") as fh:
        fh.write("\n// a note\n/* a block\n   comment */\n")
    assert bench.source_digest() == d0
    with open(dst / "mg_fused.cuh", "a") as fh:
        fh.write("constexpr int an_extra_constant = 1;\n")
    assert bench.source_digest() != d0


def test_digest_covers_the_profiled_kernel_headers():
    assert len(bench.source_digest()) == 16
    assert set(bench.DIGEST_HEADERS) == {"mg_fused.cuh", "solver_kernels.cuh", "step_kernels.cuh", "uf_device.cuh",
                                         "advect_fused.cuh", "momentum_fused.cuh"}
    # the committed ncu summaries are read (None once the device code has
    # changed since the capture, by design)
    for v in (bench.ncu_traffic("mg_down_cg_L0"), bench.ncu_traffic("advect_fused"),
              bench.fp64_flops_per_cell("mg_down_cg_L0")):
        assert v is None or v > 0
