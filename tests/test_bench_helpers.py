"""Host-side arithmetic of the benchmark (no GPU): roofline line, dominant
kernel, whole-job rate, and the recorded DRAM traffic staying tied to the
sources it was measured on."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2106_03636_gb300 import o2tpc  # noqa: E402


def test_every_stage_has_algorithmic_bytes():
    for k in bench.ROOF_KERNELS:
        assert k in bench.STAGE_BYTES and k in o2tpc.STAGES
    tracking = ("ingest", "sort", "neighbours", "clean_starts", "tracklets", "selection", "sector_fit", "merge",
                "refit")
    # per-stage minima add up to 74 B (the sort re-reads the records, the
    # cleaner re-reads the links); the path figure counts each datum once:
    # 64 B, 65 B with the continuous-readout step
    assert abs(sum(bench.STAGE_BYTES[k] for k in tracking) - 74.0) < 1e-9
    assert bench.PATH_BYTES == 65.0


def test_dominant_kernel_and_roofline():
    names = o2tpc.STAGES
    stage = np.zeros(len(names))
    stage[names.index("tl_out")] = 30.0
    stage[names.index("neighbours")] = 25.0
    stage[names.index("tracklets")] = 62.0  # a multi-kernel step is not a candidate
    k, ms = bench.dominant_kernel(stage, names)
    assert (k, ms) == ("tl_out", 30.0)
    r = bench.roofline(stage, names, 242_000_000, 6800.0, "measured")
    assert r["kernel"] == "k_tl_follow<1>" and r["bound"] == "hbm"
    assert abs(r["achieved"] - 12.0 * 242e6 / 0.030 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6800.0) < 1e-12


def test_aggregate_rate_is_whole_job():
    assert bench.aggregate_rate(1e9, 1, 1000.0) == 1e9
    assert bench.aggregate_rate(1e9, 4, 2000.0) == 2e9


def test_recorded_traffic_follows_the_sources(monkeypatch):
    """The traffic the roofline line reports comes from a capture of the
    kernel as it is now: a record carries a hash of the kernel's sources and
    counts only while they hash to it; otherwise the line reports null."""
    import hashlib

    srcs = ["k_track.cu", "o2tpc_internal.cuh"]
    h = hashlib.sha256()
    for f in srcs:
        with open(os.path.join(bench.ROOT, "paper_2106_03636_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    rec = {("k_tl_follow<1>", "full_tf"): {"bytes": 1.0e9, "sources_sha256_16": h.hexdigest()[:16], "sources": srcs},
           ("k_tl_follow<-1>", "full_tf"): {"bytes": 1.0e9, "sources_sha256_16": "0" * 16, "sources": srcs}}
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", rec)
    assert bench.measured_traffic("k_tl_follow<1>", "full_tf") == 1.0e9
    assert bench.measured_traffic("k_tl_follow<-1>", "full_tf") is None
    assert bench.measured_traffic("k_tl_follow<1>", "chunks") is None
