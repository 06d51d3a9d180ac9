"""Host-side pieces of bench.py (no GPU): workload definitions, the flop
models the roofline divides by, and the profile summaries it reads."""
import json
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

WORKLOADS = ["swe2d", "swe2d-friction", "swe2d-wb", "swe2d-limited", "swe1d", "swe1d-limited"]


@pytest.mark.parametrize("name", WORKLOADS)
def test_workload_sizes_and_flops(name):
    wl = bench.Workload(name)
    if wl.dim == 2:
        assert wl.E == (1024, 1024) and wl.N == 3 and wl.M == 3
        assert wl.dof == 1024 * 1024 * 16 * 3
    else:
        assert wl.E == (100000,) and wl.N == 4 and wl.M == 2
    f = wl.local_flops_per_element()
    assert 1000 < f < 20000
    assert wl.label().startswith(wl.system)


def test_limited_flops_add_the_first_order_part():
    from paper_2512_08611_gb300.flops import limiter_local_flops_per_element
    a = bench.Workload("swe2d").local_flops_per_element()
    b = bench.Workload("swe2d-limited").local_flops_per_element()
    assert b - a == limiter_local_flops_per_element("swe2d", 3) > 0


def test_profile_summaries_name_sources_and_traffic():
    """Every summary the bench reads states the hash of the kernel sources it
    was taken on and the DRAM bytes per launch, and gives its commands."""
    names = ["k_local_2d__swe2d_N3.md", "k_local_2d__swe2d_friction_N3.md",
             "k_local_2d__swe2d_wb_N3.md", "k_local_2d__swe2d_N3_limited.md",
             "k_step_1d__swe1d_N4.md", "k_step_1d__swe1d_N4_limited.md",
             "k_step_1d_batch__ensemble256.md"]
    for n in names:
        text = open(os.path.join(ROOT, "profiles", n)).read()
        assert re.search(r"source_sha256:\s*[0-9a-f]{16}", text), n
        m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
        assert m and float(m.group(1)) > 0, n
        assert "ncu " in text and "--clock-control none" in text, n


def test_fp64_peak_is_derived_from_unit_counts():
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(152 * 2 * 2 * 2.070e9 / 1e12)
    peaks = bench.load_peaks()
    if peaks:
        assert peaks.get("hbm_gbs", 0) > 0
