"""Benchmark: TPC clusters/s of the GB300 tracker on a full 50 kHz Pb-Pb Time Frame.

One step = one pass of the whole hot path (ingest, grid + sort, neighbours,
cleaner, start hits, tracklets, selection, sector fits, merger, final refit,
result download) over one synthetic Time Frame of 128 LHC orbits (~250 M
clusters in 12-byte fixed-point records), through the C-ABI.

* ``value``: clusters/s with the input already resident in HBM (the TF is
  submitted with device pointers); CUDA events on the library's stream
  bracket the K timed steps; the 3 GB input is larger than L2, so no flush.
* ``e2e``: the same metric with the input in pinned host memory: the
  host-to-device copy and the result download are inside the timed region.
* ``roofline``: the dominant step, from the library's per-step CUDA events,
  against the measured HBM copy bandwidth.
* ``cpu_baseline``: the FP64 single-threaded oracle on one sector of the same
  Time Frame.
* sub-objects (N = 1): ``full_tpc_1ms`` (the 1 ms, 50-collision frame),
  ``chunks`` (64 uneven chunks: one captured batch vs one chunk at a time,
  the autotuned shapes, FP64 fallbacks) and ``serving`` (Poisson arrivals at
  50 Hz from a pool of Pb-Pb and pp Time Frames: served vs plain, p50 / p99,
  sustained clusters/s, drops); ``n_fp64_fallback`` counts the final-refit
  fallbacks of the full TF.

``--impl reference`` times that oracle as the reference arm instead.
Under torchrun each rank tracks its own Time Frames (replicas; the only
collective is the max-over-ranks of the timings).
"""
from __future__ import annotations

import argparse
import collections
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TPC clusters/s and TF/s at 50 kHz Pb-Pb on 1 GB300 (served vs plain); p99 TF latency"

# Algorithmic HBM bytes per cluster of each step: data the step must read or
# write once per cluster at minimum (16-byte sort records, 8-byte sorted
# coordinates, 4-byte indices, 8-byte ownership words).  The whole path's
# minimum is PATH_BYTES per cluster.
STAGE_BYTES = {
    "ingest": 12.0,        # read the 12-byte packed record
    "sort": 12.0 + 12.0,   # read the record again, write sorted y, zeta + input index
    "neighbours": 8.0 + 8.0,  # read sorted coordinates, write two links
    "clean_starts": 8.0,   # read the links
    "tracklets": 8.0,      # ownership / hit-list words per attached cluster
    "selection": 4.0,      # output cluster index
    "sector_fit": 1.0,
    "merge": 0.5,
    "refit": 0.5,
    "sizes": 0.0,
    "download": 0.0,
    "host_prep": 0.0,
    # the two following passes of the tracklet constructor (single kernels,
    # timed apart): read the coordinates of the clusters they attach and
    # write their indices, >= 8 + 4 bytes per cluster
    "tl_out": 12.0,
    "tl_in": 12.0,
    # continuous readout: per track ~150 B (ends, state, covariance, results)
    # over ~150 clusters per track
    "continuous": 1.0,
}
# DRAM bytes (read + write) per launch that ncu measured for a kernel on a
# workload, valid while the kernel's sources hash to the recorded value;
# otherwise the line says null.
MEASURED_TRAFFIC = {
    # the following passes: one-pass DRAM counters of a single kernel on the
    # 1 ms frame (19.70 M clusters at the same 50 kHz density), scaled by the
    # cluster count (x 241.96 / 19.70) to a launch on the 128-orbit TF
    ("k_tl_follow<1>", "full_tf"): {"bytes": (1256651008 + 318376704) * 241.96 / 19.70,
                                    "sources_sha256_16": "c51eb7e4024de7bf",
                                    "sources": ["k_track.cu", "o2tpc_internal.cuh"]},
    ("k_tl_follow<-1>", "full_tf"): {"bytes": (1249804288 + 240405760) * 241.96 / 19.70,
                                     "sources_sha256_16": "c51eb7e4024de7bf",
                                     "sources": ["k_track.cu", "o2tpc_internal.cuh"]},
}


def measured_traffic(kernel: str, workload: str):
    import hashlib

    rec = MEASURED_TRAFFIC.get((kernel, workload))
    if rec is None:
        return None
    h = hashlib.sha256()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, "paper_2106_03636_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return rec["bytes"] if h.hexdigest()[:16] == rec["sources_sha256_16"] else None


# kernels (or single-kernel steps) the roofline line can name
ROOF_KERNELS = {"tl_out": "k_tl_follow<1>", "tl_in": "k_tl_follow<-1>", "neighbours": "k_neighbours",
                "refit": "k_final_refit", "sort": "k_row_scatter+k_cell_sort", "selection": "k_ownership+k_segments",
                "sector_fit": "k_sector_fit", "merge": "k_merge_*"}
PATH_BYTES = 65.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 7:
                self.rows.append(f)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def make_workload(name: str, seed: int):
    from paper_2106_03636_gb300 import synth

    if name == "full_tf":
        return synth.full_tf(seed=seed), {"workload": "full_tf_128orbits_50kHz_PbPb", "orbits": 128,
                                          "rate_khz": 50.0, "format": "fixed12"}
    if name == "full_tpc_1ms":
        return synth.full_tpc_1ms(seed=seed), {"workload": "full_tpc_50coll_1ms", "format": "float"}
    raise SystemExit(f"unknown workload {name}")


def run_raw(args, rank, world, local):
    """Clusterizer on raw ADC digits: the digits of a 20-collision 1 ms frame
    (fixed point) resident on the device; one step = o2tpc_clusterize over
    all of them.  value = digits per second; the records are then tracked
    once to show the chain (not timed)."""
    import torch
    import torch.distributed as dist

    from paper_2106_03636_gb300 import o2tpc, synth

    tf = synth.full_tpc_1ms(seed=replica_seed(args.seed, rank), n_coll=20, fmt=synth.FMT_FIXED)
    d = synth.digits_from(tf, seed=11)
    arr = {k: torch.from_numpy(np.ascontiguousarray(getattr(d, k))).to(f"cuda:{local}")
           for k in ("sector", "row", "pad", "time", "adc")}
    st = torch.cuda.Stream()
    out = torch.empty((d.n, 12), dtype=torch.uint8, device=f"cuda:{local}")
    dg = o2tpc.o2tpc_digits(n=d.n, sector=arr["sector"].data_ptr(), row=arr["row"].data_ptr(),
                            pad=arr["pad"].data_ptr(), time=arr["time"].data_ptr(), adc=arr["adc"].data_ptr())
    for _ in range(args.warmup):
        rc, nc = o2tpc.o2tpc_clusterize(dg, out.data_ptr(), d.n, st.cuda_stream)
        assert rc == 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(st)
        for _ in range(args.steps):
            rc, nc = o2tpc.o2tpc_clusterize(dg, out.data_ptr(), d.n, st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
    ms = device_max(e0.elapsed_time(e1), world, local) / args.steps
    peak, peak_kind = peaks()
    # algorithmic bytes: read the 9-byte digit once, write a 12-byte record per cluster
    alg = 9.0 * d.n + 12.0 * nc
    with o2tpc.Tracker(device=local) as trk:
        tf2 = synth.TimeFrame(n=nc, fmt=synth.FMT_FIXED, sector=np.zeros(nc, np.uint8), row=np.zeros(nc, np.uint8),
                              packed=np.zeros((1, 12), np.uint8), bz=tf.bz, vdrift=tf.vdrift)
        res = trk.wait(trk.submit(tf2, location=o2tpc.O2TPC_LOC_DEVICE, arrays={"packed": out[:nc]}))
    line = {"metric": "TPC raw digits/s through the clusterizer on 1 GB300", "value": world * d.n / (ms / 1e3),
            "unit": "digits/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "raw_digits_1ms_20coll", "digits": int(d.n), "clusters_in": int(tf.n),
                       "clusters_out": int(nc), "l2": "inputs larger than L2 (no flush)",
                       "parallelism": f"replicas x{world}"},
            "clusters_per_s": world * nc / (ms / 1e3),
            "roofline": {"bound": "hbm", "kernel": "o2tpc_clusterize (k_clu_keys + k_clu_flags + compaction + "
                                                    "k_clu_records)",
                         "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / (ms / 1e3) / 1e9 / peak, "traffic": None, "peak_kind": peak_kind,
                         "bytes_per_digit": alg / d.n},
            "tracked_after": {"status": res["status"], "tracks": res["n_tracks"]},
            "clocks": clk.summary(), "gpu_launches": 9 * args.steps}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(tf, sector: int = 0):
    """The oracle as it stands on one sector of the workload."""
    from types import SimpleNamespace

    import oracle

    sel = tf.packed[:, 9] == sector
    sub = SimpleNamespace(n=int(sel.sum()), fmt=tf.fmt, packed=np.ascontiguousarray(tf.packed[sel]), sector=None,
                          row=None, y=None, z=None, bz=tf.bz, vdrift=tf.vdrift)
    oracle.build()
    t0 = time.perf_counter()
    oracle.run(sub, fields=["trk_off"])
    dt = time.perf_counter() - t0
    return sub.n, dt


def _oracle_sector_job(packed, bz, vdrift):
    """One process of the multi-core oracle run: one sector's clusters."""
    from types import SimpleNamespace

    import oracle

    sub = SimpleNamespace(n=len(packed), fmt=1, packed=packed, sector=None, row=None, y=None, z=None, bz=bz,
                          vdrift=vdrift)
    t0 = time.perf_counter()
    oracle.run(sub, fields=["trk_off"])
    return len(packed), time.perf_counter() - t0


def oracle_baselines(tf):
    """The oracle as it stands, on the GPU machine's host cores: single-threaded
    on the single-sector frame (whole), on one sector of the 1 ms frame and on
    one sector of the benchmark's TF; and the TF's sectors as independent
    processes on all cores at once (one sector per process, as many sectors
    as cores)."""
    import multiprocessing as mp
    from types import SimpleNamespace

    import oracle
    from paper_2106_03636_gb300 import synth

    oracle.build()
    out = {}
    c0 = synth.single_sector()
    t0 = time.perf_counter()
    oracle.run(c0, fields=["trk_off"])
    out["single_sector_whole"] = {"clusters": c0.n, "s": time.perf_counter() - t0}
    c1 = synth.full_tpc_1ms()
    sel = c1.sector == 0
    sub = SimpleNamespace(n=int(sel.sum()), fmt=0, packed=None, sector=np.ascontiguousarray(c1.sector[sel]),
                          row=np.ascontiguousarray(c1.row[sel]), y=np.ascontiguousarray(c1.y[sel]),
                          z=np.ascontiguousarray(c1.z[sel]), bz=c1.bz, vdrift=c1.vdrift)
    t0 = time.perf_counter()
    oracle.run(sub, fields=["trk_off"])
    out["full_tpc_1ms_sector0"] = {"clusters": sub.n, "s": time.perf_counter() - t0}
    nc, dt = cpu_baseline(tf)
    out["full_tf_sector0"] = {"clusters": nc, "s": dt}
    cores = min(os.cpu_count() or 1, 36)
    jobs = [np.ascontiguousarray(tf.packed[tf.packed[:, 9] == s]) for s in range(cores)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_sector_job, [(j, tf.bz, tf.vdrift) for j in jobs])
    wall = time.perf_counter() - t0
    out["full_tf_all_cores"] = {"clusters": int(sum(r[0] for r in res)), "s": wall, "cores": cores,
                                "sectors": cores}
    for v in out.values():
        v["clusters_per_s"] = v["clusters"] / v["s"]
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    import torch  # noqa: F401  (same process layout as the main arm)

    tf, cfg = make_workload(args.workload, args.seed)
    cfg["sample"] = "sector 0 of the Time Frame per step"
    for _ in range(args.warmup):
        cpu_baseline(tf)
    n_tot, t_tot = 0, 0.0
    for _ in range(args.steps):
        n, dt = cpu_baseline(tf)
        n_tot += n
        t_tot += dt
    v = n_tot / t_tot
    line = {"metric": METRIC, "value": v, "unit": "clusters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "clusters/s", "cores": 1, "kind": "oracle",
                             "sample": f"sector 0 of the TF ({n_tot // args.steps} clusters) per step"},
            "e2e": {"value": v, "unit": "clusters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def dominant_kernel(stage, names):
    """The longest single kernel (or single-kernel step) of a step."""
    idx = {nm: i for i, nm in enumerate(names)}
    cand = [(float(stage[idx[k]]), k) for k in ROOF_KERNELS]
    ms, k = max(cand)
    return k, ms


def roofline(stage, names, n, peak, peak_kind, workload=None):
    k, ms = dominant_kernel(stage, names)
    achieved = STAGE_BYTES[k] * n / (ms / 1e3) / 1e9
    traffic = measured_traffic(ROOF_KERNELS[k], workload) if workload else None
    return {"bound": "hbm", "kernel": ROOF_KERNELS[k], "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
            "bytes_per_cluster": STAGE_BYTES[k], "ms_per_launch": ms}


def device_max(ms, world, local, device=None):
    """Max over ranks of a duration (replicas; the only collective).  The
    tensor lives on the rank's GPU (NCCL), or on `device` (gloo on CPU)."""
    if world == 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], device=device or f"cuda:{local}")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def replica_seed(seed: int, rank: int) -> int:
    """Each replica tracks its own Time Frames (weak scaling): seeds differ
    by rank."""
    return seed + 1000 * rank


def aggregate_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return world * units_per_rank / (ms / 1e3)


def measure_chunks(args, rank, world, local, steps, warmup):
    """Uneven sub-Time-Frame chunks (64 chunks, Poisson(20) collisions each, a
    quarter pp-like): plain = one chunk per launch sequence, synchronised per
    chunk; batched = all chunks in one batch (one launch sequence, one CUDA
    graph launch unless --no-graph).  Returns the measurement's fields."""
    import torch
    import torch.distributed as dist

    from paper_2106_03636_gb300 import o2tpc, synth

    chunks = synth.chunk_mix(seed=replica_seed(20210610, rank))
    n = sum(c.n for c in chunks)
    dev = [{"packed": torch.from_numpy(c.packed).to(f"cuda:{local}")} for c in chunks]
    torch.cuda.synchronize()
    tune = 0 if args.no_autotune else o2tpc.O2TPC_FLAG_AUTOTUNE
    plain = o2tpc.Tracker(device=local, flags=o2tpc.O2TPC_FLAG_NO_BATCHING | tune)
    # batched: all chunks in one batch; captured path (one CUDA graph launch) unless --no-graph
    gcap = 0 if args.no_graph else int(n * 1.25)
    batched = o2tpc.Tracker(device=local, max_batch=len(chunks), batch_full_clusters=2**64 - 1, flags=tune,
                            graph_max_clusters=gcap, graph_max_tfs=len(chunks))

    def pass_plain(loc=o2tpc.O2TPC_LOC_DEVICE, arrays=dev):
        out = []
        for c, a in zip(chunks, arrays):
            out.append(plain.wait(plain.submit(c, location=loc, arrays=a)))
        return out

    def pass_batched(loc=o2tpc.O2TPC_LOC_DEVICE, arrays=dev):
        tk = batched.submit_many(chunks, location=loc, arrays=arrays)
        return [batched.wait(t) for t in tk]

    def timed(fn, trk, *a):
        for _ in range(warmup):
            fn(*a)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stage = np.zeros(len(o2tpc.STAGES))
        launches, sizes, captured = 0, set(), set()
        fallback = 0
        e0.record(trk.stream)
        for _ in range(steps):
            rs = fn(*a)
            for r in rs:
                if r["status"] != 0:
                    raise RuntimeError(o2tpc.o2tpc_strerror(r["status"]))
            seen = {}
            for r in rs:  # stages and launches once per batch
                key = (r["stats"]["ms_device"], r["stats"]["batch_size"])
                if key not in seen:
                    seen[key] = r
            for r in seen.values():
                stage += np.asarray(r["stats"]["ms_stage"])
                launches += int(r["stats"]["n_launches"])
                sizes.add(int(r["stats"]["batch_size"]))
                captured.add(int(r["stats"]["captured"]))
                fallback += int(r["stats"]["n_fp64_fallback"])
        e1.record(trk.stream)
        torch.cuda.synchronize()
        ms = device_max(e0.elapsed_time(e1), world, local)
        timed.captured = sorted(captured)
        timed.fallback = fallback // steps
        return ms / steps, stage / steps, launches // steps, sorted(sizes), rs

    ms_p, stage_p, l_p, _, _ = timed(pass_plain, plain)
    ms_b, stage_b, l_b, sizes_b, rs = timed(pass_batched, batched)
    captured_b = timed.captured
    fallback_b = timed.fallback
    if captured_b == [1]:
        # the graph records no per-step events: step times of the same
        # batch on the regular path, for stage_ms and the roofline line
        reg = o2tpc.Tracker(device=local, max_batch=len(chunks), batch_full_clusters=2**64 - 1, flags=tune)
        ms_r, stage_b, _, _, _ = timed(lambda: [reg.wait(t) for t in reg.submit_many(chunks, location=o2tpc.O2TPC_LOC_DEVICE, arrays=dev)], reg)
        reg.close()
    e2e = None
    if not args.no_e2e:
        pin = [{"packed": torch.from_numpy(c.packed).pin_memory()} for c in chunks]
        ms_e, _, _, _, _ = timed(pass_batched, batched, o2tpc.O2TPC_LOC_HOST, pin)
        nt = sum(r["n_tracks"] for r in rs)
        ncl = sum(r["n_cluster_refs"] for r in rs)
        e2e = {"value": world * n / (ms_e / 1e3), "unit": "clusters/s", "h2d_bytes_per_step": 12 * n,
               "d2h_bytes_per_step": 8 * (nt + len(chunks)) + 4 * ncl + nt * 106, "ms_per_step": ms_e,
               "mode": "batched from pinned host memory"}
    peak, peak_kind = peaks()
    names = o2tpc.STAGES
    out = {"value": world * n / (ms_b / 1e3), "unit": "clusters/s", "ms_per_step": ms_b,
           "config": {"workload": "chunks_64x36sectors_poisson20", "chunks": len(chunks), "clusters": int(n),
                      "chunk_clusters_min": int(min(c.n for c in chunks)),
                      "chunk_clusters_max": int(max(c.n for c in chunks)), "format": "fixed12",
                      "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}"},
           "n_fp64_fallback": fallback_b,
           "batched": {"value": world * n / (ms_b / 1e3), "ms_per_step": ms_b, "batch_sizes": sizes_b,
                        "gpu_launches": l_b, "captured_graph": captured_b == [1],
                        "graph_launches_per_step": 1 if captured_b == [1] else 0},
            "plain": {"value": world * n / (ms_p / 1e3), "ms_per_step": ms_p, "gpu_launches": l_p,
                      "stage_ms": {names[i]: round(float(stage_p[i]), 3) for i in range(len(o2tpc.STAGES))}},
            "speedup_batched_vs_plain": ms_p / ms_b,
            "stage_ms_source": "regular path, same batch" if captured_b == [1] else "batched arm",
            "stage_ms": {names[i]: round(float(stage_b[i]), 3) for i in range(len(o2tpc.STAGES))},
            "roofline": roofline(stage_b, names, n, peak, peak_kind),
            "path_roofline": {"bytes_per_cluster": PATH_BYTES, "peak": peak,
                              "frac": n / (ms_b / 1e3) * PATH_BYTES / 1e9 / peak},
            "e2e": e2e, "gpu_launches": l_b,
            "autotune": {"batched": batched.tuning(), "plain": plain.tuning()}}
    plain.close()
    batched.close()
    return out


def run_chunks(args, rank, world, local):
    """The 64-chunk batch as its own bench line."""
    with ClockSampler(local) as clk:
        m = measure_chunks(args, rank, world, local, args.steps, args.warmup)
    line = {"metric": METRIC, "value": m.pop("value"), "unit": m.pop("unit"), "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m.pop("ms_per_step"), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": m.pop("config"),
            "cpu_baseline": None, "clocks": clk.summary()}
    line.update(m)
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_serving(args, rank, local, pool, seconds):
    """Served stream: Time Frames drawn from `pool` arrive as a Poisson
    process at --rate-hz over `seconds` from pinned host memory; at most
    --max-queue are admitted at once (an arrival that finds the server full
    is dropped and counted).  Latency = arrival -> result polled on the
    host.  The same arrival sequence is then replayed 'plain': one TF at a
    time, submitted and waited for, no batching and no overlap.  Returns
    {"served": ..., "plain": ..., "offered": ...}."""
    import torch

    from paper_2106_03636_gb300 import o2tpc

    pin = [{"packed": torch.from_numpy(t.packed).pin_memory()} for t in pool]
    rng = np.random.default_rng(20210611 + rank)
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate_hz, int(args.rate_hz * seconds * 2) + 10))
    arrivals = arrivals[arrivals < seconds]
    picks = rng.integers(0, len(pool), len(arrivals))

    def warm(trk):
        for i in range(min(len(pool), max(args.warmup, 3))):  # device memory pool, pinned result blocks
            trk.wait(trk.submit(pool[i], location=o2tpc.O2TPC_LOC_HOST, arrays=pin[i]))

    def summary(done, dropped, t0):
        lat = np.array([1e3 * (b - a) for a, b, _, _ in done])
        ncl = sum(pool[d[2]].n for d in done)
        wall = max(d[1] for d in done) - t0
        sizes = np.array([d[3] for d in done])
        return {"value": ncl / wall, "tf_per_s": len(done) / wall, "served": int(len(done)), "dropped": int(dropped),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_batch": float(sizes.mean()), "wall_s": wall}

    def served_run():
        # batches of small TFs (up to the GPU-full size) run as one captured graph launch
        trk = o2tpc.Tracker(device=local, max_inflight=args.max_queue,
                            graph_max_clusters=0 if args.no_graph else 1 << 25, graph_max_tfs=16)
        warm(trk)
        done, pending = [], collections.deque()
        n_captured = [0]
        cv = threading.Condition()
        state = {"closed": False}

        def poller():
            while True:
                with cv:
                    cv.wait_for(lambda: pending or state["closed"])
                    if not pending:
                        return
                    tk, t_arr, i = pending.popleft()
                r = trk.wait(tk)
                if r["status"] != 0:
                    raise RuntimeError(o2tpc.o2tpc_strerror(r["status"]))
                done.append((t_arr, time.perf_counter(), i, r["stats"]["batch_size"]))
                n_captured[0] += int(r["stats"]["captured"])

        th = threading.Thread(target=poller, daemon=True)
        th.start()
        dropped = 0
        t0 = time.perf_counter()
        for t_a, i in zip(arrivals, picks):
            now = time.perf_counter() - t0
            if t_a > now:
                time.sleep(t_a - now)
            try:
                tk = trk.submit(pool[i], location=o2tpc.O2TPC_LOC_HOST, arrays=pin[i])
            except o2tpc.O2TPCError as e:
                if e.status != o2tpc.O2TPC_EAGAIN:
                    raise
                dropped += 1
                continue
            with cv:
                pending.append((tk, t0 + t_a, i))
                cv.notify()
        with cv:
            state["closed"] = True
            cv.notify()
        th.join()
        trk.close()
        out = summary(done, dropped, t0)
        out["captured_tfs"] = n_captured[0]
        return out

    def plain_run():
        trk = o2tpc.Tracker(device=local, flags=o2tpc.O2TPC_FLAG_NO_BATCHING)
        warm(trk)
        done, q = [], collections.deque()
        dropped, j = 0, 0
        t0 = time.perf_counter()
        while j < len(arrivals) or q:
            now = time.perf_counter() - t0
            while j < len(arrivals) and arrivals[j] <= now:
                if len(q) < args.max_queue:
                    q.append(j)
                else:
                    dropped += 1
                j += 1
            if not q:
                time.sleep(max(0.0, arrivals[j] - now))
                continue
            a = q.popleft()
            r = trk.wait(trk.submit(pool[picks[a]], location=o2tpc.O2TPC_LOC_HOST, arrays=pin[picks[a]]))
            if r["status"] != 0:
                raise RuntimeError(o2tpc.o2tpc_strerror(r["status"]))
            done.append((t0 + arrivals[a], time.perf_counter(), picks[a], 1))
        trk.close()
        return summary(done, dropped, t0)

    srv = served_run()
    pln = plain_run()
    return {"served": srv, "plain": pln, "offered": int(len(arrivals)), "rate_hz": args.rate_hz,
            "arrival_window_s": seconds, "max_queue": args.max_queue,
            "pool_clusters": [int(t.n) for t in pool], "input": "pinned host memory"}


def measure_full_tpc_1ms(args, rank, world, local, steps: int = 5):
    """The 1 ms full-TPC frame (50 collisions, ~21 M float clusters) resident
    on the device: one frame at a time, synchronised per frame."""
    import torch

    from paper_2106_03636_gb300 import o2tpc, synth

    tf = synth.full_tpc_1ms(seed=replica_seed(20210608, rank))
    dev = {k: torch.from_numpy(getattr(tf, k)).to(f"cuda:{local}") for k in ("sector", "row", "y", "z")}
    torch.cuda.synchronize()
    with o2tpc.Tracker(device=local) as trk:
        for _ in range(3):
            r = trk.wait(trk.submit(tf, location=o2tpc.O2TPC_LOC_DEVICE, arrays=dev))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(trk.stream)
        for _ in range(steps):
            r = trk.wait(trk.submit(tf, location=o2tpc.O2TPC_LOC_DEVICE, arrays=dev))
            if r["status"] != 0:
                raise RuntimeError(o2tpc.o2tpc_strerror(r["status"]))
        e1.record(trk.stream)
        torch.cuda.synchronize()
    ms = device_max(e0.elapsed_time(e1), world, local) / steps
    return {"value": world * tf.n / (ms / 1e3), "unit": "clusters/s", "ms_per_step": ms, "steps": steps,
            "clusters": int(tf.n), "tracks": int(r["n_tracks"]), "n_fp64_fallback": int(r["stats"]["n_fp64_fallback"]),
            "mode": "plain, one frame at a time, input resident in HBM", "format": "float"}


def run_serving(args, rank, world, local):
    """The served stream over the pool of 24 Time Frames (half Pb-Pb with
    10..570 collisions, half pp-like ~3 M clusters) as its own bench line."""
    from paper_2106_03636_gb300 import synth

    pool = synth.serving_pool(seed=replica_seed(20210611, rank))
    with ClockSampler(local) as clk:
        m = measure_serving(args, rank, local, pool, args.serve_seconds)
    srv = m["served"]
    line = {"metric": METRIC, "value": srv["value"], "unit": "clusters/s", "n_gpus": world, "steps": srv["served"],
            "warmup": args.warmup, "ms_per_step": 1e3 * srv["wall_s"] / max(1, srv["served"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving_pool24_poisson", "rate_hz": args.rate_hz,
                       "arrival_window_s": args.serve_seconds, "max_queue": args.max_queue,
                       "pool_clusters": m["pool_clusters"], "format": "fixed12",
                       "input": "pinned host memory", "parallelism": f"replicas x{world}"},
            "offered": m["offered"], "tf_per_s": srv["tf_per_s"], "p50_ms": srv["p50_ms"],
            "p99_ms": srv["p99_ms"], "served": srv, "plain": m["plain"], "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="full_tf", choices=["full_tf", "full_tpc_1ms", "chunks", "serving", "raw"])
    ap.add_argument("--rate-hz", type=float, default=50.0, help="serving: Poisson arrival rate of TFs")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="serving: arrival window")
    ap.add_argument("--max-queue", type=int, default=16, help="serving: TFs admitted at once (more are dropped)")
    ap.add_argument("--no-extras", action="store_true",
                    help="full_tf: skip the 1 ms frame, chunk and serving sub-measurements")
    ap.add_argument("--serve-pool", type=int, default=8, help="full_tf: TFs in the serving sub-measurement's pool")
    ap.add_argument("--serve-extra-seconds", type=float, default=20.0,
                    help="full_tf: arrival window of the serving sub-measurement")
    ap.add_argument("--plain-only", action="store_true",
                    help="time only the one-TF-at-a-time loop, one TF in flight (small device footprint for "
                         "profiling); implies --no-e2e --no-compress --no-extras")
    ap.add_argument("--oracle-configs", action="store_true",
                    help="also time the oracle on the other workloads and on all host cores")
    ap.add_argument("--seed", type=int, default=20210609)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compress", action="store_true", help="skip the compressed-TF measurement")
    ap.add_argument("--trace", action="store_true", help="per-TF stage times on stderr")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes instead of the autotuner's")
    ap.add_argument("--no-graph", action="store_true", help="served and chunks arms on the regular path, not captured")
    ap.add_argument("--torch-memory", action="store_true",
                    help="device buffers from PyTorch's caching allocator (no uploads ahead)")
    ap.add_argument("--inflight", type=int, default=3, help="TFs kept in flight in the served measurement")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "gb300" else args.warmup
    if args.plain_only:
        args.no_e2e = args.no_compress = args.no_extras = True

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    import torch
    import torch.distributed as dist

    if world > 1:
        dist.init_process_group("nccl" if args.impl == "gb300" else "gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
        if world > 1:
            dist.destroy_process_group()
        return

    torch.cuda.set_device(local)
    from paper_2106_03636_gb300 import o2tpc

    if args.workload == "chunks":
        return run_chunks(args, rank, world, local)
    if args.workload == "serving":
        return run_serving(args, rank, world, local)
    if args.workload == "raw":
        return run_raw(args, rank, world, local)

    tf, cfg = make_workload(args.workload, replica_seed(args.seed, rank))
    n = tf.n
    host_in = torch.from_numpy(tf.packed if tf.fmt == 1 else np.zeros(1, np.uint8))
    dev = {}
    if tf.fmt == 1:
        dev["packed"] = host_in.to(f"cuda:{local}")
    else:
        for k in ("sector", "row", "y", "z"):
            dev[k] = torch.from_numpy(getattr(tf, k)).to(f"cuda:{local}")
    torch.cuda.synchronize()

    tune = 0 if args.no_autotune else o2tpc.O2TPC_FLAG_AUTOTUNE
    # plain: one TF at a time on the regular path (per-stage launches, host
    # synchronisations), synchronised per TF
    trk = o2tpc.Tracker(device=local, torch_memory=args.torch_memory, flags=tune)

    def trace(tag, r):
        if args.trace:
            st = r["stats"]["ms_stage"]
            print(f"{tag}: batch {r['stats']['batch_size']} device {r['stats']['ms_device']:.2f} ms, "
                  + ", ".join(f"{o2tpc.STAGES[i]} {st[i]:.2f}" for i in range(len(o2tpc.STAGES))), file=sys.stderr, flush=True)

    def step(t, location, arrays):
        r = t.wait(t.submit(tf, location=location, arrays=arrays))
        if r["status"] != 0:
            raise RuntimeError(o2tpc.o2tpc_strerror(r["status"]))
        trace(f"step loc={location}", r)
        return r

    def timed(t, location, arrays):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stage = np.zeros(len(o2tpc.STAGES))
        launches = 0
        lat = []
        e0.record(t.stream)
        for _ in range(args.steps):
            t0 = time.perf_counter()
            r = step(t, location, arrays)
            lat.append(1e3 * (time.perf_counter() - t0))
            stage += np.asarray(r["stats"]["ms_stage"])
            launches += int(r["stats"]["n_launches"])
        e1.record(t.stream)
        torch.cuda.synchronize()
        ms = device_max(e0.elapsed_time(e1), world, local)
        return ms, stage / args.steps, launches, lat, r

    def served(t, location, arrays, total, inflight):
        """Continuous batching: `inflight` TFs stay queued; the library's
        worker admits them as memory and slots free up.  Latency = submit ->
        result polled."""
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pending = collections.deque()
        t_sub, lat, sizes, capt = {}, [], [], []
        launches = 0.0
        submitted = done = 0
        e0.record(t.stream)
        while done < total:
            while submitted < total and len(pending) < inflight:
                tk = t.submit(tf, location=location, arrays=arrays)
                t_sub[tk] = time.perf_counter()
                pending.append(tk)
                submitted += 1
            tk = pending.popleft()
            r = t.wait(tk)
            if r["status"] != 0:
                raise RuntimeError(o2tpc.o2tpc_strerror(r["status"]))
            lat.append(1e3 * (time.perf_counter() - t_sub.pop(tk)))
            trace(f"served loc={location}", r)
            b = int(r["stats"]["batch_size"])
            sizes.append(b)
            capt.append(int(r["stats"]["captured"]))
            launches += r["stats"]["n_launches"] / b
            done += 1
        e1.record(t.stream)
        torch.cuda.synchronize()
        ms = device_max(e0.elapsed_time(e1), world, local)
        served.captured = capt
        return ms, lat, sizes, int(round(launches))

    for _ in range(args.warmup):
        r = step(trk, o2tpc.O2TPC_LOC_DEVICE, dev)
    n_served = max(1, args.steps)
    pin = None
    if not args.no_e2e:
        pin = {"packed": host_in.pin_memory()} if tf.fmt == 1 else {
            k: torch.from_numpy(getattr(tf, k)).pin_memory() for k in ("sector", "row", "y", "z")}
    with ClockSampler(local) as clk:
        ms, stage, launches, lat, r = timed(trk, o2tpc.O2TPC_LOC_DEVICE, dev)
        if not args.no_e2e:
            step(trk, o2tpc.O2TPC_LOC_HOST, pin)
            ms_h, stage_h, _, lat_h, rh = timed(trk, o2tpc.O2TPC_LOC_HOST, pin)
        tuning = trk.tuning()
        trk.close()  # its memory pool goes before the served context's
        if args.plain_only:  # one TF in flight: the plain loop stands for both
            ms_s, lat_s, sizes_s, launches_s = ms, lat, [1] * args.steps, launches // args.steps
            captured_s = [0] * args.steps
        else:
            # served: its own context; with the captured path every TF is one
            # CUDA graph launch (no host synchronisation inside), the next TF's
            # replay queued behind it while the previous result downloads
            gcap = 0 if args.no_graph else ((n + (1 << 20)) >> 20) << 20
            strk = o2tpc.Tracker(device=local, torch_memory=args.torch_memory, flags=tune, graph_max_clusters=gcap,
                                 graph_max_tfs=1)
            for _ in range(args.warmup):
                step(strk, o2tpc.O2TPC_LOC_DEVICE, dev)
            served(strk, o2tpc.O2TPC_LOC_DEVICE, dev, args.inflight + 1, args.inflight)
            ms_s, lat_s, sizes_s, launches_s = served(strk, o2tpc.O2TPC_LOC_DEVICE, dev, n_served, args.inflight)
            captured_s = served.captured
    clocks = clk.summary()
    ms_step = ms / args.steps
    plain_value = aggregate_rate(n, world, ms_step)
    served_value = aggregate_rate(n * n_served, world, ms_s)
    value = served_value

    # e2e: pinned host input, H2D and result download inside the timed region
    e2e = None
    if not args.no_e2e:
        if args.plain_only:
            ms_hs, lat_hs, sizes_hs = ms_h, lat_h, [1] * args.steps
        else:
            served(strk, o2tpc.O2TPC_LOC_HOST, pin, args.inflight + 1, args.inflight)
            ms_hs, lat_hs, sizes_hs, _ = served(strk, o2tpc.O2TPC_LOC_HOST, pin, n_served, args.inflight)
        h2d = 12 * n if tf.fmt == 1 else 10 * n
        nt, ncl = rh["n_tracks"], rh["n_cluster_refs"]
        # offsets, cluster indices; x, alpha, par, cov, chi2, ndf, sector, flags, zeta_ref,
        # t0 / error / bounds, membrane partner, collision
        d2h = 8 * (nt + 1) + 4 * ncl + nt * (4 * 2 + 20 + 60 + 4 + 4 + 1 + 1 + 4 + 16 + 4 + 4)
        e2e = {"value": world * n * n_served / (ms_hs / 1e3), "unit": "clusters/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "mode": "served from pinned host memory",
               "ms_per_step": ms_hs / n_served, "p50_ms": float(np.percentile(lat_hs, 50)),
               "p99_ms": float(np.percentile(lat_hs, 99)), "batch_sizes": sizes_hs,
               "plain": {"value": world * n / (ms_h / args.steps / 1e3), "ms_per_step": ms_h / args.steps,
                         "p50_ms": float(np.percentile(lat_h, 50)), "p99_ms": float(np.percentile(lat_h, 99)),
                         "stage_ms": {o2tpc.STAGES[i]: round(float(stage_h[i]), 3) for i in range(len(o2tpc.STAGES))}}}
    if not args.plain_only:
        strk.close()
    # the compressed TF (Sec. 2.2) on the same TF: one TF at a time, device input
    compressed = None
    if not args.no_compress:
        ctk = o2tpc.Tracker(device=local, flags=tune | o2tpc.O2TPC_FLAG_COMPRESS)
        for _ in range(2):
            rc = ctk.wait(ctk.submit(tf, location=o2tpc.O2TPC_LOC_DEVICE, arrays=dev))
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = max(3, min(args.steps, 5))
        cst = np.zeros(len(o2tpc.STAGES))
        c0.record(ctk.stream)
        for _ in range(k):
            rc = ctk.wait(ctk.submit(tf, location=o2tpc.O2TPC_LOC_DEVICE, arrays=dev))
            if rc["status"] != 0:
                raise RuntimeError(o2tpc.o2tpc_strerror(rc["status"]))
            cst += np.asarray(rc["stats"]["ms_stage"])
        c1.record(ctk.stream)
        torch.cuda.synchronize()
        cms = device_max(c0.elapsed_time(c1), world, local) / k
        cst /= k
        compressed = {"value": world * n / (cms / 1e3), "unit": "clusters/s", "ms_per_step": cms,
                      "mode": "plain, one TF at a time, tracking + compressed TF",
                      "ctf_bytes": rc["ctf_bytes"], "ctf_bytes_per_cluster": rc["ctf_bytes"] / n,
                      "ratio_vs_12B_records": 12.0 * n / max(1, rc["ctf_bytes"]),
                      "stage_ms_compress": round(float(cst[o2tpc.STAGES.index("compress")]), 3),
                      "compress_clusters_per_s": n / (float(cst[o2tpc.STAGES.index("compress")]) / 1e3)}
        ctk.close()

    peak, peak_kind = peaks()
    names = o2tpc.STAGES
    roof = roofline(stage, names, n, peak, peak_kind, args.workload)
    path_frac = plain_value / world * PATH_BYTES / 1e9 / peak

    # the other workloads of the benchmark, each a sub-object of this line
    extras = {}
    if world == 1 and not args.no_extras:
        with ClockSampler(local) as clk_x:
            extras["full_tpc_1ms"] = measure_full_tpc_1ms(args, rank, world, local)
            extras["chunks"] = measure_chunks(args, rank, world, local, 3, 3)
            from paper_2106_03636_gb300 import synth

            pool = synth.serving_pool(seed=replica_seed(20210611, rank), n_tf=args.serve_pool)
            extras["serving"] = measure_serving(args, rank, local, pool, args.serve_extra_seconds)
            del pool
        extras["clocks"] = clk_x.summary()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and tf.fmt == 1:
        nc0, dt0 = cpu_baseline(tf)
        cpu = {"value": nc0 / dt0, "unit": "clusters/s", "cores": 1, "kind": "oracle",
               "sample": f"sector 0 of the same TF: {nc0} clusters, {dt0:.1f} s"}
        if args.oracle_configs:
            cpu["configs"] = oracle_baselines(tf)

    cfg.update({"clusters": int(n), "tracks": int(r["n_tracks"]), "l2": "inputs larger than L2 (no flush)",
                "mode": ("plain only: one TF at a time" if args.plain_only else
                         f"served: continuous batching, {args.inflight} TFs in flight (TF replayed from memory)"
                         + ("" if args.no_graph else ", captured path (one CUDA graph launch per TF)")),
                "parallelism": f"replicas x{world}"})
    line = {"metric": METRIC, "value": value, "unit": "clusters/s", "n_gpus": world, "steps": n_served,
            "warmup": args.warmup, "ms_per_step": ms_s / n_served, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "tf_per_s": world * n_served / (ms_s / 1e3), "p50_ms": float(np.percentile(lat_s, 50)),
            "p99_ms": float(np.percentile(lat_s, 99)),
            "served": {"value": served_value, "tf_per_s": world * n_served / (ms_s / 1e3),
                       "p50_ms": float(np.percentile(lat_s, 50)), "p99_ms": float(np.percentile(lat_s, 99)),
                       "batch_sizes": sizes_s, "tfs": n_served, "gpu_launches": launches_s,
                       "captured": captured_s},
            "plain": {"value": plain_value, "tf_per_s": world / (ms_step / 1e3), "ms_per_step": ms_step,
                      "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                      "steps": args.steps},
            "stage_ms": {names[i]: round(float(stage[i]), 3) for i in range(len(o2tpc.STAGES))},
            "path_roofline": {"bytes_per_cluster": PATH_BYTES, "frac": path_frac, "peak": peak},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_s, "clocks": clocks,
            "autotune": tuning, "compressed": compressed,
            "n_fp64_fallback": int(r["stats"]["n_fp64_fallback"]), "n_tracks": int(r["n_tracks"])}
    line.update(extras)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
