"""Host logic of bench.py that needs no GPU: the recorded DRAM traffic of the
step kernel is reported only while the source it was taken on is unchanged,
and the key is the step kernel's own source (a change to another kernel in
the same header does not void it; a change to the step kernel does)."""
import os
import shutil

import bench


def _copy_csrc(tmp_path):
    src = os.path.join(bench.ROOT, "paper_2203_01316_gb300", "csrc")
    dst = tmp_path / "csrc"
    dst.mkdir()
    for f in ("lbm_device.cuh", "lbm_kernels.cuh"):
        shutil.copy(os.path.join(src, f), dst / f)
    return dst


def test_hash_ignores_other_kernels_and_follows_the_step(tmp_path):
    d = _copy_csrc(tmp_path)
    h0 = bench.kernel_source_hash(str(d))
    assert h0 == bench.kernel_source_hash()
    ker = (d / "lbm_kernels.cuh").read_text()
    # a change to the adjoint kernels (after the step kernel and launch_step)
    tail = ker.replace("// ---- adjoint of the h evolution", "// ---- adjoint of the h evolution (edited)", 1)
    assert tail != ker
    (d / "lbm_kernels.cuh").write_text(tail)
    assert bench.kernel_source_hash(str(d)) == h0
    # a change inside the step kernel
    step = ker.replace("if (type == T_SOLID) return;", "if (type == T_SOLID) { return; }", 1)
    assert step != ker
    (d / "lbm_kernels.cuh").write_text(step)
    assert bench.kernel_source_hash(str(d)) != h0
    # a change to the device collision code
    (d / "lbm_kernels.cuh").write_text(ker)
    dev = (d / "lbm_device.cuh").read_text()
    (d / "lbm_device.cuh").write_text(dev + "\n// edited\n")
    assert bench.kernel_source_hash(str(d)) != h0


def test_recorded_traffic_matches_the_current_step_kernel():
    # profiles/traffic.json was taken on the current step-kernel source
    t = bench.recorded_traffic("k_step_f32_q27_384x128x128")
    assert t is not None and 2.6e9 < t < 2.8e9


def test_clock_summary_parses_samples_and_reasons():
    cs = bench.ClockSampler(0)
    cs.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2062, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1390.2, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = cs.summary()
    assert s["sm_mhz"] == 2062.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    cs.lines = ["0, 1500, 2070, 700.0, 0x8, Active, Not Active, Active, Not Active"]
    assert bench.ClockSampler.summary(cs)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    cs.lines = []
    assert bench.ClockSampler.summary(cs)["reasons"] == ["no samples"]
