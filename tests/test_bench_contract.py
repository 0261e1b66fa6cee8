"""Host logic of bench.py's JSON line (no GPU): the roofline entry of the
dominant region and the DRAM traffic read from the committed ncu summary."""

import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_tensor_roofline_reports_useful_flop_and_the_issued_passes_apart(bench):
    peaks, _ = bench.measured_peaks()
    kernels = {"assign_tc": {"ms": 2000.0, "work": 6.0e14, "launches": 48},
               "kmeanspp": {"ms": 600.0, "work": 2.0e12, "launches": 3}}
    r = bench.roofline_of(kernels, "dense10m", 3000.0)
    assert r["kernel"] == "assign_tc" and r["bound"] == "tensor"
    useful = 6.0e14 / 2.0 / 1e12                      # TFLOP/s of useful work
    peak = peaks["bf16_tflops_sustained"] * 1.1 / 2.25
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(useful)
    assert r["frac"] == pytest.approx(useful / peak)
    assert r["achieved_issued"] == pytest.approx(bench.TC_PASSES * useful)
    assert r["frac_issued"] == pytest.approx(bench.TC_PASSES * useful /
                                             peaks["bf16_tflops_sustained"])
    assert r["work_per_launch"] == pytest.approx(6.0e14 / 48)
    assert r["ms_share_of_step"] == pytest.approx(2000.0 / 3000.0)
    # the traffic row is used only while the kernel's source is unchanged
    t = bench.ncu_traffic("assign_tc", "dense10m")
    assert r["traffic"] == t
    rows = [ln for ln in open(os.path.join(ROOT, "profiles", "traffic.md"))
            if ln.startswith("| assign_tc | dense10m |")]
    assert len(rows) == 1
    cells = [c.strip() for c in rows[0].strip().strip("|").split("|")]
    if bench.source_hash(cells[2]) == cells[3]:
        assert t == float(cells[4])
    else:
        assert t is None


def test_hbm_roofline_against_the_copy_bandwidth(bench):
    peaks, _ = bench.measured_peaks()
    kernels = {"scan_leaf_cm": {"ms": 4.0, "work": 8.0e9, "launches": 1}}
    r = bench.roofline_of(kernels, "dense10m", 10.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(8.0e9 / 4e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / peaks["hbm_gbs"])
    assert r["traffic"] is None                       # no committed row for it


def test_unknown_traffic_rows_give_none(bench):
    assert bench.ncu_traffic("no_such_kernel", "dense10m") is None
