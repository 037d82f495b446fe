"""Host arithmetic of the benchmark line, on CPU: the roofline object (dominant phase and every
phase against its ALU peak), the HBM peak lookup and the whole-job rate of replicas."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_roofline_phases_and_dominant_phase(bench):
    info = {"form_flops": 2.0e9, "eval_flops": 3.0e9, "gather_flops": 0.5e9, "direct_flops": 0.1e9}
    # 4 profiled steps; per step: form 0.2 ms, evaluate 0.3 ms, gather 0.05 ms, near 0.1 ms
    prof = {"form": 0.8, "evaluate": 1.2, "gather": 0.2, "near": 0.4, "merge": 0.0, "push": 0.0}
    r = bench.roofline_of(info, prof, 4, 1)
    # split form: the contractions against the 3xTF32 tensor-pipe roofline, FP32 CUDA cores beside it
    tpk, _ = bench.split_tensor_peak_tflops()
    assert r["kernel"] == "evaluate" and r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 3.0e9 / 0.3e-3 / 1e12) < 1e-9
    assert r["peak"] == tpk and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert abs(r["frac_of_fp32_cuda_core"] - r["achieved"] / bench.FP32_PEAK_TFLOPS) < 1e-12
    ph = r["phases"]
    assert set(ph) == {"form", "evaluate", "gather", "near"}          # phases without work are left out
    assert ph["near"]["peak_tflops"] == bench.FP64_PEAK_TFLOPS        # the near field stays FP64
    assert abs(ph["form"]["achieved_tflops"] - 10.0) < 1e-9 and abs(ph["form"]["ms"] - 0.2) < 1e-12
    assert ph["form"]["peak_tflops"] == tpk and "frac_of_fp32_cuda_core" in ph["form"]
    # FP64 form: every phase against the FP64 peak
    r64 = bench.roofline_of(info, prof, 4, 0)
    assert r64["bound"] == "alu" and r64["peak"] == bench.FP64_PEAK_TFLOPS
    assert all(v["peak_tflops"] == bench.FP64_PEAK_TFLOPS for v in r64["phases"].values())
    # FP64_TC in 3D: form and evaluation against the sliced tensor roofline, gather and near field
    # (double-float on the FP32 pipes) against the FP32 instruction rate / 15 per double-float FMA
    spk, _ = bench.sliced_tensor_peak_tflops()
    rtc = bench.roofline_of(dict(info, d=3, n_sliced_jobs=12), prof, 4, 2)
    assert rtc["kernel"] == "evaluate" and rtc["bound"] == "tensor" and rtc["peak"] == spk
    assert rtc["phases"]["gather"]["peak_tflops"] == rtc["phases"]["near"]["peak_tflops"] == bench.DF_PEAK_TFLOPS
    assert abs(bench.DF_PEAK_TFLOPS - bench.FP32_PEAK_TFLOPS / 15) < 1e-12
    assert "frac_of_fp64_alu" in rtc["phases"]["gather"]
    # FP64_TC without sliced stages (2D): FP64 peaks throughout
    r2 = bench.roofline_of(dict(info, d=2, n_sliced_jobs=0), prof, 4, 2)
    assert all(v["peak_tflops"] == bench.FP64_PEAK_TFLOPS for v in r2["phases"].values())


def test_split_tensor_peak(bench, tmp_path, monkeypatch):
    # measured BF16 burst rate x 1/2 (TF32 runs at half the BF16 rate) / 3 products per 3xTF32 product
    f = tmp_path / "peaks.json"
    f.write_text('{"hbm_gbs": 6000.0, "bf16_tflops": 1800.0}')
    monkeypatch.setattr(bench, "PEAKS_FILE", str(f))
    assert bench.split_tensor_peak_tflops() == (300.0, "measured")
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "missing.json"))
    assert bench.split_tensor_peak_tflops() == (1900.0 / 6, "fallback")


def test_error_vs_oracle_row(bench):
    import numpy as np
    u_or = np.ones((3, 8))
    u = np.ones((10, 8))
    u[4, 2] = 1 + 3e-6
    r = bench.error_vs_oracle(u.reshape(-1), np.array([1, 4, 7]), u_or, 1e-6)
    assert abs(r["max_abs_over_max_u"] - 3e-6) < 1e-15 and abs(r["bound"] - 1e-5) < 1e-20 and r["within_bound"]
    assert r["sample_leaves"] == 3


def test_kernel_l1_against_quadrature(bench):
    """max_x of the integral of G over B: free kernel at the centre, periodic kernel over one period
    (image sum), by composite Gauss-Legendre quadrature."""
    import math
    import numpy as np
    x, wq = np.polynomial.legendre.leggauss(200)
    y, wy = 0.5 * x, 0.5 * wq
    for delta in (1e-3, 0.1, 1.0, 4.0):
        free = float((np.exp(-y ** 2 / delta) * wy).sum())
        per = float(sum((np.exp(-(y + n) ** 2 / delta) * wy).sum() for n in range(-12, 13)))
        for d in (1, 2, 3):
            assert abs(bench.kernel_l1(d, delta, False) - free ** d) <= 1e-12 * free ** d
            assert abs(bench.kernel_l1(d, delta, True) - per ** d) <= 1e-12 * per ** d
    assert abs(bench.kernel_l1(3, 1.0, True) - math.pi ** 1.5) < 1e-12


def test_error_vs_oracle_degenerate_scale(bench):
    """Periodic trig density at delta = 1: the exact u is (pi delta)^{3/2} exp(-3 pi^2 delta n_p^2)
    sigma_p, far below rounding, so the error is judged on ||sigma||_inf ||G||_1; a genuinely
    wrong result on that scale still fails."""
    import types
    import numpy as np
    w = types.SimpleNamespace(d=3, delta=1.0, periodic=True, sigma=np.array([[1.0, -1.0]]))
    u_or = np.full((2, 8), 1e-200)
    u = np.full((2, 8), 3e-17)
    r = bench.error_vs_oracle(u.reshape(-1), np.array([0, 1]), u_or, 1e-6, w)
    assert r["max_abs_over_max_u"] > 1 and "degenerate" in r and r["within_bound"]
    u[1, 3] = 1e-3
    assert not bench.error_vs_oracle(u.reshape(-1), np.array([0, 1]), u_or, 1e-6, w)["within_bound"]
    # a non-degenerate row keeps the max |u| scale
    u_or = np.ones((2, 8))
    u = np.ones((2, 8))
    u[0, 0] += 2e-5
    r = bench.error_vs_oracle(u.reshape(-1), np.array([0, 1]), u_or, 1e-6, w)
    assert "degenerate" not in r and not r["within_bound"]


def test_derived_alu_peaks(bench):
    # 152 SMs at 2.07 GHz: 2 FP64 FMA / clock / SM and 128 FP32 lanes, 2 flops per FMA
    assert abs(bench.FP64_PEAK_TFLOPS - 1.25856) < 1e-9
    assert abs(bench.FP32_PEAK_TFLOPS - 80.54784) < 1e-9


def test_clock_sampler_is_live_before_the_region(bench, tmp_path, monkeypatch):
    # a stand-in nvidia-smi: one idle line at once, then a line every 10 ms at 2070 MHz
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 1200, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "while true; do sleep 0.01; "
                    "echo '0, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active'; done\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    import time
    with bench.ClockSampler(0) as cs:
        assert cs.first and cs.first.startswith("0, 1200")   # sampling was live before the region
        time.sleep(0.2)
    sm = cs.summary()
    assert sm["sm_mhz"] == 2070.0 and sm["sm_max_mhz"] == 2070.0 and sm["samples"] >= 3
    assert sm["reasons"] == ["sw_power_cap"] and "note" not in sm
    # only the pre-region line: reported as such
    cs.rows = []
    sm1 = cs.summary()
    assert sm1["sm_mhz"] == 1200.0 and sm1["samples"] == 1 and "before" in sm1["note"]
    # no nvidia-smi at all
    monkeypatch.setenv("PATH", str(tmp_path / "empty"))
    with bench.ClockSampler(0) as cs0:
        pass
    assert cs0.summary()["reasons"] == ["unavailable"]


def test_hbm_peak_lookup(bench, tmp_path, monkeypatch):
    f = tmp_path / "peaks.json"
    f.write_text('{"hbm_gbs": 6000.5}')
    monkeypatch.setattr(bench, "PEAKS_FILE", str(f))
    assert bench.hbm_peak_gbs() == (6000.5, "measured")
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "missing.json"))
    assert bench.hbm_peak_gbs() == (6800.0, "fallback")


def test_whole_job_rate_of_replicas(bench):
    # weak scaling: every rank transforms its own copy each step
    assert bench.whole_job_rate(1000, 10, 4, 2.0) == 4 * 1000 * 10 / 2.0


def test_adaptive_delta_workload_is_the_same_tree(bench):
    # the delta 1e-4 benchmark workload: the adaptive tree and density unchanged, only delta differs
    a, b = bench.workload("adaptive3d"), bench.workload("adaptive3d_d1e-4")
    assert a.delta == 1e-3 and b.delta == 1e-4
    assert (a.tree.level == b.tree.level).all() and (a.tree.coord == b.tree.coord).all()
    assert (a.sigma == b.sigma).all() and a.n_points == b.n_points
