"""The bench's roofline arithmetic on CPU: algorithmic work from the plan and the live kernel time,
the peak from the measured peaks, and the captured DRAM traffic only while the kernel's source
still matches the capture."""
import hashlib
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_karatsuba_roofline_counts_the_sub_products():
    import bench

    plan = {"levels": 3, "h": 256, "groups": 27, "mq": 4608, "kq": 8192}
    n, m, B, ms = 1 << 16, 36473, 8192, 2.0
    r = bench.roofline_for("gemm_karatsuba", B, m, n, ms, plan)
    flops = 2.0 * B * 27 * 4608 * 8192  # 18 live row blocks of 256: every row tile issued
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - flops / (ms / 1e3) / 1e12) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert abs(r["peak"] - 6.0 * bench.measured_peaks()["bf16_tflops"]) < 1e-9
    # the plain product the route replaces, reported beside it
    assert abs(r["equivalent_plain_tflops"] - 2.0 * B * m * n / (ms / 1e3) / 1e12) < 1e-6 * r["achieved"]


def test_karatsuba_roofline_counts_only_issued_rows():
    """At four levels the laser stream's sub-products have 9 live row blocks of 256 in a plan of 10
    (whole pairs of tiles): the tenth gets no MMAs and is not counted."""
    import bench

    plan = {"levels": 4, "h": 256, "groups": 81, "mq": 2560, "kq": 4096}
    n, m, B, ms = 1 << 16, 36473, 8192, 1.8
    r = bench.roofline_for("gemm_karatsuba", B, m, n, ms, plan)
    assert r["rows_issued"] == 2304
    assert abs(r["achieved"] - 2.0 * B * 81 * 2304 * 4096 / (ms / 1e3) / 1e12) < 1e-6 * r["achieved"]


def test_traffic_record_tracks_the_kernel_source():
    import bench

    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)["gemm_pair_kara_kernel"]
    with open(os.path.join(ROOT, "paper_2011_04130_gb300", "csrc", "k_gemm_pair.cu"), "rb") as f:
        current = hashlib.sha256(f.read()).hexdigest()
    got = bench.captured_traffic("gemm_pair_kara_kernel", "k_gemm_pair.cu", rec["blocks"])
    if rec["source_sha256"] == current:
        assert got == rec["dram_bytes"]
    else:
        assert got is None  # a stale capture is never reported
    # scaled by the blocks of the launch
    if got is not None:
        assert bench.captured_traffic("gemm_pair_kara_kernel", "k_gemm_pair.cu", rec["blocks"] // 2) == \
            rec["dram_bytes"] // 2


def test_unknown_route_has_no_roofline():
    import bench

    r = bench.roofline_for("no_such_route", 10, 10, 10, 1.0)
    assert r["bound"] is None and r["frac"] is None


def test_direct_roofline_uses_the_device_sm_count():
    import bench

    caps = {"sms": 100, "sm_max_mhz": 2000.0}
    r = bench.roofline_for("direct", 8, 1000, 4096, 1.0, caps=caps)
    assert r["peak"] == 64 * 32 * 100 * 2000e6 / 1e12
    assert abs(r["achieved"] - 8 * 1000 * 4096 / 1e-3 / 1e12) < 1e-9


def test_transform_routes_report_hbm_and_pipe_fractions():
    import bench

    pk = bench.measured_peaks()
    n, m, B, ms = 1 << 16, 36473, 8192, 10.0
    r = bench.roofline_for("fft64", B, m, n, ms)
    P = 1 << 17
    flops = B // 2 * (10.0 * P * 17 + 6.0 * P)
    assert r["bound"] == "fp64" and abs(r["achieved"] - flops / 1e-2 / 1e12) < 1e-9 * r["achieved"]
    assert abs(r["hbm"]["achieved"] - B * (n + m) / 8 / 1e-2 / 1e9) < 1e-9 * r["hbm"]["achieved"]
    assert abs(r["hbm"]["frac"] - r["hbm"]["achieved"] / pk["hbm_gbs"]) < 1e-12
    r = bench.roofline_for("ntt", B, m, n, ms)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"


def test_fft32_roofline_counts_transforms_and_products():
    import bench

    caps = {"sms": 152, "sm_max_mhz": 2070.0}
    n_t, m, B, ms, S, T = 1 << 16, 36473, 64, 2.0, 4096, 8
    r = bench.roofline_for("fft32_seg", B, m, n_t, ms, {"segment": S, "terms": T}, caps)
    NS, NQ = 16, 9
    per_block = (NS + NQ * 2) * 5.0 * S * 12 + NQ * NS * S * 8.0
    flops = B * per_block + (NQ + NS - 1) * 5.0 * S * 12
    assert r["bound"] == "fp32" and r["segment"] == S and r["terms"] == T
    assert abs(r["achieved"] - flops / 2e-3 / 1e12) < 1e-9 * r["achieved"]
    assert abs(r["peak"] - 2 * 128 * 152 * 2070e6 / 1e12) < 1e-9
