"""Host-side pieces of bench.py that need no GPU: the traffic record is
reported only for the kernel sources it was taken on, the plain pipeline's
HBM roofline follows its 28 bytes per combination, the clock summary keeps
the samples of the timed region, and the distinct-fit count skips the
excluded layer."""
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sources_sha():
    h = hashlib.sha256()
    for name in ("svt_kernels.cu", "svt_internal.h"):
        with open(os.path.join(ROOT, "paper_1312_0917_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def test_traffic_record_follows_the_kernel_sources(monkeypatch):
    sha = _sources_sha()
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {
        "stress": {"kernels_sha256": sha, "bytes": 123},
        "scaled": {"kernels_sha256": "0" * 64, "bytes": 456},
    })
    assert bench.measured_traffic("stress") == 123
    assert bench.measured_traffic("scaled") is None     # taken on other sources
    assert bench.measured_traffic("uneven") is None     # no record


def test_committed_traffic_records_name_one_source_state():
    shas = {r["kernels_sha256"] for r in bench.NCU_TRAFFIC.values()}
    assert len(shas) == 1
    assert all(r["bytes"] > 0 for r in bench.NCU_TRAFFIC.values())


def test_plain_hbm_roofline(monkeypatch):
    monkeypatch.setattr(bench, "measured_hbm_gbs", lambda: 1000.0)
    r = bench.plain_hbm(n_fits=10 ** 9, ms=100.0)
    assert r["bytes_per_batch"] == 28 * 10 ** 9
    assert r["achieved_gbs"] == 280.0              # 28 GB in 0.1 s
    assert r["frac"] == 0.28


def test_clock_summary_keeps_the_timed_samples():
    s = bench.ClockSampler(0)
    row = lambda mhz, reason: [  # noqa: E731
        "0", str(mhz), "2070", "900.0", "0x0", "Not Active", "Not Active", reason, "Active"]
    s.rows = [(1.0, row(1000, "Not Active")), (2.0, row(2070, "Not Active")),
              (3.0, row(2060, "Not Active")), (4.0, row(2070, "Not Active")),
              (5.0, row(1200, "Active"))]
    all_ = s.summary()
    assert all_["samples"] == 5 and all_["sm_max_mhz"] == 2070.0
    assert all_["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]
    timed = s.summary(1.5, 4.5)
    assert timed["samples"] == 3 and timed["sm_mhz"] == 2070.0
    assert timed["reasons"] == ["sw_power_cap"]


def test_distinct_fits_skip_the_excluded_layer():
    from paper_1312_0917_gb300 import synth
    b = synth.make_batch("small", seed=0, n_events=20)
    n = b.roads["n"].astype(np.int64)
    excl = b.roads["excl"].astype(np.int64)
    want = 0
    for k in range(len(n)):   # a road with no hit on its excluded layer has no combination
        if n[k][excl[k]] > 0:
            want += int(np.prod([n[k][l] for l in range(5) if l != excl[k]]))
    assert bench.distinct_fits(b) == want
    assert 0 < want <= b.n_fits
