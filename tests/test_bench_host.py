"""Host-side logic of bench.py (no GPU): the roofline arithmetic of the bench line, the
gate that reports the recorded DRAM traffic only for the sources it was captured on, and
the digest of those sources, which ignores comments so that a comment edit keeps it.
"""
import importlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    try:
        return importlib.import_module("bench")
    finally:
        sys.path.remove(ROOT)


def _peaks(mhz=2000.0):
    # per-unit rates chosen so that every time below is a round number
    rates = {"ffma": 4.0e13, "ffma2": 3.0e13, "ex2": 1.0e13, "lg2": 5.0e12, "rcp": 5.0e12,
             "rsqrt": 5.0e12, "dfma": 5.0e11}
    return {"units": {k: {"ops_per_s": v} for k, v in rates.items()}, "clocks": {"sm_mhz": mhz}}


def test_roofline_fp32_bound(bench):
    work = {"fp32_method": 4.0e11, "fp32_precision": 4.0e10,
            "sfu": {"ex2": 1.0e10, "lg2": 5.0e9, "rcp": 1.0e10, "rsqrt": 5.0e9}}
    r = bench.alu_roofline(work, 0.040, _peaks(), 2000.0)
    # FP32 pipe: the better of scalar and packed FMA, 4e13/s -> 10 ms; SFU 1 + 1 + 2 + 1 ms
    assert r["unit"].startswith("Tops/s (FP32")
    assert r["t_fp32_ms"] == pytest.approx(10.0)
    assert r["t_sfu_ms"] == pytest.approx(5.0)
    assert r["achieved"] == pytest.approx(4.0e11 / 0.040 / 1e12)
    assert r["peak"] == pytest.approx(40.0)
    assert r["frac"] == pytest.approx(0.25)
    assert r["frac_with_precision"] == pytest.approx(0.275)
    # the issue port: FP32 and SFU lane operations share it at the FP32 peak's rate
    assert r["t_issue_fp32_plus_sfu_ms"] == pytest.approx((4.0e11 + 3.0e10) / 4.0e13 * 1e3)
    assert r["frac_issue_fp32_plus_sfu"] == pytest.approx((4.0e11 + 3.0e10) / 4.0e13 / 0.040)
    assert r["frac_issue_fp32_plus_sfu"] >= r["frac"]


def test_roofline_sfu_bound_and_clock_scale(bench):
    work = {"fp32_method": 4.0e10, "fp32_precision": 0.0,
            "sfu": {"ex2": 1.0e11, "lg2": 0.0, "rcp": 0.0, "rsqrt": 0.0}}
    # the probes ran at 2000 MHz, the kernel at 1000 MHz: every rate halves
    r = bench.alu_roofline(work, 0.040, _peaks(2000.0), 1000.0)
    assert r["clock_scale"] == pytest.approx(0.5)
    assert r["unit"].startswith("Tops/s (SFU")
    assert r["t_sfu_ms"] == pytest.approx(20.0)
    assert r["t_fp32_ms"] == pytest.approx(2.0)
    assert r["frac"] == pytest.approx(0.5)


def test_traffic_reported_only_for_its_sources_and_workload(bench, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC", {"digest": "abc", "workload": "c3", "K": 256,
                                           "bytes_per_launch": 1.0e9})
    monkeypatch.setattr(bench, "kernel_digest", lambda read=None: "abc")
    assert bench.traffic_for("c3", 256) == 1.0e9
    assert bench.traffic_for("c2", 256) is None
    assert bench.traffic_for("c3", 64) is None
    monkeypatch.setattr(bench, "kernel_digest", lambda read=None: "def")
    assert bench.traffic_for("c3", 256) is None


def test_digest_ignores_comments_but_not_code(bench):
    files = {}
    for f in bench.KERNEL_SOURCES:
        path = os.path.join("paper_2605_23538_gb300", "csrc", f)
        with open(os.path.join(ROOT, path), encoding="utf-8") as fh:
            files[path] = fh.read()
    base = bench.kernel_digest(lambda p: files[p])
    assert base == bench.kernel_digest()
    first = next(iter(files))
    commented = dict(files)
    commented[first] = "// a new comment line\n" + files[first].replace("\n", "  /* and a block */\n", 1) + "\n\n"
    assert bench.kernel_digest(lambda p: commented[p]) == base
    changed = dict(files)
    changed[first] = files[first] + "\nstatic int an_extra_definition = 1;\n"
    assert bench.kernel_digest(lambda p: changed[p]) != base
