"""bench.py's host-side bookkeeping (CPU): the roofline entry and the traffic
figures it reads from the committed ncu summaries under profiles/."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2205_11990_gb300 import inputs as I  # noqa: E402


def traffic_lines():
    out = []
    for fn in sorted(os.listdir(bench.PROFILES)):
        if fn.endswith(".md"):
            for line in open(os.path.join(bench.PROFILES, fn)):
                if line.startswith("bench-traffic:"):
                    out.append((fn, line.split()))
    return out


def test_traffic_lines_are_well_formed():
    lines = traffic_lines()
    assert lines, "no bench-traffic line under profiles/"
    workloads = set(I.WORKLOADS) | set(getattr(I, "SPECIES_WORKLOADS", {}))
    for fn, parts in lines:
        assert len(parts) == 4, (fn, parts)
        _, kernel, workload, value = parts
        assert kernel.startswith(("k_", "kb_")), (fn, kernel)
        assert workload in workloads, (fn, workload)
        assert float(value) > 0, (fn, value)


def test_headline_kernel_has_traffic():
    # the headline's dominant class names a kernel whose capture is committed
    kernel = bench.KERNEL_OF_CLASS["qr_factor"]
    t = bench.profile_traffic(kernel, bench.WORKLOAD)
    assert t is not None and t > 0
    assert bench.profile_traffic("no_such_kernel", bench.WORKLOAD) is None


def test_roofline_fraction_and_peak_choice():
    # 2.4 GFLOP of QR work in 50 ms of a 100 ms step: 0.048 TFLOP/s
    prof = {"qr_factor": (50.0, 10, 2.4e9), "gemm": (10.0, 5, 1e9), "apply": (0.1, 1, 1e6)}
    r = bench.roofline(prof, 100.0, 1, bench.WORKLOAD)
    assert r["class"] == "qr_factor" and r["kernel"] == bench.KERNEL_OF_CLASS["qr_factor"]
    assert abs(r["achieved"] - 0.048) < 1e-12
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
    assert abs(r["peak"] - bench.DW_PEAK_GFLOPS / 1e3) < 1e-12  # no probes: the derived roof
    assert abs(r["share_of_step"] - 0.5) < 1e-12
    # a measured dot/update mix above the derived roof replaces it
    r2 = bench.roofline(prof, 100.0, 1, bench.WORKLOAD, probes={"dw_dot": 7.0, "dw_axpy": 3.6})
    assert abs(r2["peak"] - 2.0 / (1.0 / 7.0 + 1.0 / 3.6)) < 1e-12
    # and one below it does not
    r3 = bench.roofline(prof, 100.0, 1, bench.WORKLOAD, probes={"dw_dot": 2.0, "dw_axpy": 1.0})
    assert abs(r3["peak"] - bench.DW_PEAK_GFLOPS / 1e3) < 1e-12
    # a GEMM-dominated window is measured against the FP64 roof
    r4 = bench.roofline({"gemm": (10.0, 5, 1e10)}, 20.0, 1, bench.WORKLOAD)
    assert r4["bound"] == "alu" and abs(r4["peak"] - bench.FP64_PEAK_GFLOPS / 1e3) < 1e-12
