"""Host-side logic of bench.py that needs no GPU: the clock summary keeps only the
nvidia-smi samples inside the timed region and reads the throttle reasons, and the DRAM
traffic figure is reported only while the kernel source matches the hash recorded with
the ncu capture; the serving stream keeps its own arrival times."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _row(mhz, power_cap="Not Active", thermal="Not Active"):
    return ["0", str(mhz), "2070", "900.0", "0x0", "Not Active", "Not Active", thermal, power_cap]


def _clocks(rows, window):
    c = bench.Clocks(0)
    c.proc = object()   # a sampler that ran
    c.rows = rows
    c.window = window
    return c


def test_clock_summary_keeps_samples_inside_the_timed_region():
    rows = [(0.0, _row(1200)), (1.0, _row(2070)), (1.5, _row(2055, power_cap="Active")), (3.0, _row(900))]
    s = _clocks(rows, (0.9, 2.0)).summary()
    assert s["samples"] == 2 and s["window"] == "timed region"
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_short_region_takes_the_nearest_samples():
    rows = [(0.0, _row(1000)), (1.00, _row(2070, thermal="Active")), (1.10, _row(2070)), (5.0, _row(500))]
    s = _clocks(rows, (1.02, 1.04)).summary()
    assert s["window"] == "nearest to the timed region" and s["samples"] == 2
    assert s["sm_mhz"] == 2070.0
    assert s["reasons"] == ["sw_thermal_slowdown"]


def test_clock_summary_without_sampler():
    assert bench.Clocks(0).summary()["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_reported_only_for_the_captured_kernel_source(tmp_path, monkeypatch):
    src = tmp_path / "paper_1802_06738_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    kernel = src / "sigma_kernels.cu"
    kernel.write_text("// kernel v1\n")
    digest = hashlib.sha256(kernel.read_bytes()).hexdigest()
    (tmp_path / "profiles" / "sigma_traffic_medium.md").write_text(
        f"traffic per call (bytes): sandwich->sigma = 1234\n\nkernel source sha256: {digest}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("sandwich->sigma", "medium", "FP32") == 1234.0
    assert bench.ncu_traffic("dense->sigma", "medium", "FP32") is None
    assert bench.ncu_traffic("sandwich->sigma", "large", "FP32") is None     # no capture of that workload
    # the BF16 sandwich class is the tensor-core kernel: its own source decides
    assert bench.ncu_traffic("sandwich->sigma", "medium", "BF16") is None
    tck = src / "sandwich_tc.cu"
    tck.write_text("// tensor-core kernel v1\n")
    (tmp_path / "profiles" / "sigma_traffic_large.md").write_text(
        "traffic per call (bytes): sandwich->sigma = 99\n\nkernel source sha256: "
        + hashlib.sha256(tck.read_bytes()).hexdigest() + "\n")
    assert bench.ncu_traffic("sandwich->sigma", "large", "BF16") == 99.0
    kernel.write_text("// kernel v2\n")
    assert bench.ncu_traffic("sandwich->sigma", "medium", "FP32") is None
    assert bench.ncu_traffic("sandwich->sigma", "large", "BF16") == 99.0


def test_reference_arm_prints_the_same_metric(capsys):
    """The oracle arm uses the GPU arm's metric string; for a workload the oracle cannot
    reach within the run it prints its unavailable line with the reason."""
    import types
    args = types.SimpleNamespace(workload="large", steps=3, warmup=1, gpus=1)
    bench.run_reference(args, 1, 0)
    import json
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert "unavailable" in line and "o=60" in line["config"]["workload"]


def test_roofline_bound_per_precision():
    """The BF16 sandwich class is tensor-bound against the BF16 peak of MEASURED_PEAKS.json
    (sustained); in the FP32 sigma the same class is SIMT work against the FP32 FMA peak."""
    dom = {"name": "sandwich->sigma", "ms": 10.0, "flops": 4e11, "bytes": 1e9, "launches": 2}
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
    dev = {"fp32_fma_tflops": 77.0, "tc_bf16_tflops": 2400.0}
    r = bench.roofline(dom, 1, peaks, dev, {}, "BF16")
    assert r["bound"] == "tensor" and r["peak"] == 1700.0 and abs(r["achieved"] - 40.0) < 1e-9
    assert abs(r["vs_device_tcgen05_bf16"]["frac"] - 40.0 / 2400.0) < 1e-12
    r = bench.roofline(dom, 1, peaks, dev, {}, "FP32")
    assert r["bound"] == "alu" and r["peak"] == 77.0
    g = dict(dom, name="gemm->sigma")
    assert bench.roofline(g, 1, peaks, dev, {}, "BF16")["peak"] == 850.0
    h = dict(dom, name="dense->sigma", flops=1e9)
    r = bench.roofline(h, 1, peaks, dev, {}, "BF16")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"


def test_serving_stream_keeps_the_streams_own_arrival_times():
    """The serving mode submits requests of the 600-request Poisson stream at their own
    arrival times: unfiltered it is the whole stream; a cap on o thins it without
    re-drawing the arrivals."""
    from synthetic import poisson_requests
    whole = poisson_requests(600, 20.0, 5)
    assert bench.serving_stream(600, 40, 20.0) == whole
    thin = bench.serving_stream(40, 14, 20.0)
    assert len(thin) == 40 and all(r["o"] <= 14 for r in thin)
    assert all(r in whole for r in thin)
    ts = [r["t"] for r in thin]
    assert all(a < b for a, b in zip(ts, ts[1:]))


def test_serving_arms_option():
    args = bench.parse(["--mode", "serving", "--arms", "mixed,fp64", "--omax", "40", "--nreq", "600"])
    assert args.arms.split(",") == ["mixed", "fp64"] and args.serve_mixed == "FP32"


def test_fp64_roofline_picks_the_unit_of_the_dominant_class():
    peaks = {"hbm_gbs": 6784.5}
    dev = {"fp64_fma_tflops": 1.06, "cublas_dgemm_tflops": 1.10}
    sw = {"name": "sandwich->sigma", "launches": 3, "ms": 30.0, "bytes": 1e9, "flops": 1e11}
    dn = {"name": "dense->sigma", "launches": 3, "ms": 3.0, "bytes": 1e9, "flops": 1e8}   # below the ridge
    r = bench.fp64_roofline([sw, dn], 3, peaks, dev)
    assert r["kernel"] == "sandwich->sigma" and r["bound"] == "alu" and r["peak"] == 1.06
    assert abs(r["achieved"] - 1e11 / 10e-3 / 1e12) < 1e-12
    r = bench.fp64_roofline([dict(sw, ms=1.0), dict(dn, ms=60.0)], 3, peaks, dev)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and abs(r["frac"] - (1e9 / 20e-3 / 1e9) / 6784.5) < 1e-12
    g = {"name": "gemm->sigma", "launches": 3, "ms": 90.0, "bytes": 1e8, "flops": 1e12}
    assert bench.fp64_roofline([g, sw], 3, peaks, dev)["peak"] == 1.10
    assert "unavailable" in bench.fp64_roofline([dict(sw, ms=0.0)], 3, peaks, dev)
