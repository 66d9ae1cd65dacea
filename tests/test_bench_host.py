"""Host logic of the benchmark line: the roofline object (dominant kernel by
its serialised GPU share, algorithmic bytes over the event time, fraction of
the measured peak), the ncu traffic figure withdrawn once the kernel's source
changed, and the clock-sample parser (throttle reasons, median SM clock)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _frames(F, n):
    return [(np.zeros((n, 3), np.float32), None) for _ in range(F)]


def test_roofline_names_the_dominant_kernel_and_computes_the_fraction():
    F, n, steps, C = 8, 1000, 10, bench.C
    nv = np.full(F, n)
    sb = np.full(F, 50_000)
    stages = {"raht_forward_pass0": (10.0, steps), "raht_inverse_pass0": (6.0, steps),
              "rlgr_encode": (9.0, steps), "rlgr_decode": (12.0, steps)}  # decode's event time is the largest
    r = bench.roofline(stages, _frames(F, n), nv, sb, steps, F, 6000.0, "measured")
    assert r["kernel"] == bench.DOMINANT == "raht_forward_pass0"
    alg = 4 * C * (F * n + F * n)  # gathered input rows and written coefficient rows, one launch per step
    assert r["bytes_per_launch"] == alg
    assert np.isclose(r["achieved"], round(alg / (1.0 / 1e3) / 1e9, 1))
    assert np.isclose(r["frac"], round(r["achieved"] / 6000.0, 4), atol=1e-4)
    assert set(r["all"]) == set(stages)
    # without the named kernel the largest event time decides
    del stages["raht_forward_pass0"]
    r2 = bench.roofline(stages, _frames(F, n), nv, sb, steps, F, 6000.0, "measured")
    assert r2["kernel"] == "rlgr_decode"


def test_traffic_is_withdrawn_when_the_source_changed(monkeypatch):
    ent = bench.TRAFFIC["raht_forward_pass0"]
    got = bench.measured_traffic("raht_forward_pass0", 8)
    path = os.path.join(ROOT, "paper_2606_05650_gb300", ent[1])
    import hashlib
    same = hashlib.sha1(open(path, "rb").read()).hexdigest() == ent[2]
    assert (got == int(ent[0] * 8)) if same else got is None
    monkeypatch.setitem(bench.TRAFFIC, "raht_forward_pass0", (ent[0], ent[1], "0" * 40))
    assert bench.measured_traffic("raht_forward_pass0", 8) is None
    assert bench.measured_traffic("no_such_kernel", 8) is None


def test_clock_samples_parse_reasons_and_median():
    cs = bench.ClockSampler(0)

    class _P:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0
    cs.proc = _P()
    cs.lines = ["0, 2070, 2070, 500.1, 0x0, Not Active, Not Active, Not Active, Not Active",
                "0, 2055, 2070, 610.5, 0x4, Not Active, Not Active, Not Active, Active",
                "0, 2070, 2070, 590.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                "garbage"]
    r = cs.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"] and r["power_w_max"] == 610.5


def test_pipeline_fraction():
    # 1,000 frames/s of 1M Gaussians at the stage-minimum bytes against a 6,781 GB/s peak
    v = bench.pipeline_fraction(1000.0, 1_000_000, 6781.4)
    assert np.isclose(v, 1000 * 1e6 * bench.PIPELINE_BYTES_PER_GAUSSIAN / 6781.4e9)
    assert 1900 < bench.PIPELINE_BYTES_PER_GAUSSIAN < 2300  # about 1.25 KB encode + 0.75 KB decode


def test_host_cpu_description():
    h = bench.host_cpu()
    assert h["nproc"] >= 1
    assert "model" not in h or isinstance(h["model"], str)


def test_issue_rate_entry_for_instruction_bound_coders():
    F, n, steps = 16, 1000, 4
    nv = np.full(F, n)
    sb = np.full(F, 50_000)
    stages = {"raht_forward_pass0": (8.0, steps), "rlgr_encode": (7.2, steps)}
    peak = 152 * 4 * 2070e6
    r = bench.roofline(stages, _frames(F, n), nv, sb, steps, F, 6000.0, "measured", peak)
    enc = r["all"]["rlgr_encode"]
    inst = bench.measured_traffic("rlgr_encode", F, bench.INSTR)
    if inst is None:  # counts withdrawn after a source change
        assert "issue" not in enc
        return
    assert inst == int(bench.INSTR["rlgr_encode"][0] * F)
    ms = 7.2 / steps
    assert np.isclose(enc["issue"]["frac"], inst / (ms / 1e3) / peak, atol=1e-4)
    assert "issue" not in r["all"]["raht_forward_pass0"]
    # no peak given: no issue entry
    r0 = bench.roofline(stages, _frames(F, n), nv, sb, steps, F, 6000.0, "measured")
    assert "issue" not in r0["all"]["rlgr_encode"]


def test_stage_roofline_uses_the_per_gaussian_bytes():
    steps, n = 4, 16_000_000
    stages = {"sort": (4 * 1.2, steps), "occupancy": (4 * 0.8, steps), "reconstruction": (0.01, steps)}
    r = bench.stage_roofline(stages, n, steps, 6000.0, 56, 16)
    assert set(r) == {"sort", "occupancy"}  # stages without algorithmic bytes are left out
    assert r["sort"]["bytes_per_step"] == 24 * 6 * n  # six 8-bit passes over 48 code bits
    assert np.isclose(r["sort"]["GBs"], round(24 * 6 * n / 1.2e-3 / 1e9, 1))
    assert np.isclose(r["sort"]["frac"], round(r["sort"]["GBs"] / 6000.0, 4), atol=1e-4)
    assert r["sort"]["branch"] == "serial" and r["occupancy"]["branch"] == "concurrent"
    assert bench.stage_bytes(56, 16)["raht_forward"][0] == 448


def test_latency_legs_pause_the_garbage_collector():
    import gc
    was = gc.isenabled()
    with bench._no_gc():
        assert not gc.isenabled()
    assert gc.isenabled() == was
