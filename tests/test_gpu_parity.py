"""CUDA path vs the oracle through the C-ABI (needs a GB300)."""
import numpy as np
import pytest

import oracle
from helpers import float_tf
from parity import assert_criteria, brief, compare_stages, compare_tracks, pool
from paper_2106_03636_gb300 import o2tpc, synth

pytestmark = pytest.mark.gpu

ZUNIT = 0.003125 * 2.58
RESULT_KEYS = ("offsets", "cluster_idx", "par", "cov", "chi2", "ndf", "flags", "zeta_ref", "t0", "t0_err", "t0_lo",
               "t0_hi", "mate", "collision")


@pytest.fixture(scope="module")
def trk():
    t = o2tpc.Tracker(flags=o2tpc.O2TPC_FLAG_KEEP_STAGES)
    yield t
    t.close()


def run_both(trk, tf):
    ticket = trk.submit(tf)
    res = trk.poll(ticket, keep=True)
    assert res["status"] == 0
    o = oracle.run(tf)
    return ticket, res, o


def test_single_sector_parity(trk):
    tf = synth.single_sector()
    ticket, res, o = run_both(trk, tf)
    compare_stages(trk, ticket, o)
    print(brief(compare_tracks(res, o, ZUNIT)))
    trk.release(ticket, res)


def test_single_sector_dense_parity(trk):
    """Ten dense single-sector frames (1500 primaries each, 19x the
    single-sector occupancy), pooled."""
    reps = []
    for seed in range(77, 87):
        tf = synth.single_sector(seed=seed, ntracks=1500)
        ticket, res, o = run_both(trk, tf)
        compare_stages(trk, ticket, o)
        reps.append(compare_tracks(res, o, ZUNIT, check=False))
        trk.release(ticket, res)
    rep = pool(reps)
    print(brief(rep))
    assert_criteria(rep)


@pytest.mark.parametrize("n_coll", [3, 50])
def test_full_tpc_parity(trk, n_coll):
    tf = synth.full_tpc_1ms(n_coll=n_coll)
    ticket, res, o = run_both(trk, tf)
    compare_stages(trk, ticket, o)
    print(brief(compare_tracks(res, o, ZUNIT)))
    trk.release(ticket, res)


def test_fixed_point_parity(trk):
    tf = synth.full_tpc_1ms(seed=5, n_coll=2, fmt=synth.FMT_FIXED)
    ticket, res, o = run_both(trk, tf)
    compare_stages(trk, ticket, o)
    print(brief(compare_tracks(res, o, ZUNIT)))
    trk.release(ticket, res)


def test_tracklets_and_sector_tracks(trk):
    """Tracklet hit lists and sector tracks, not only the final tracks."""
    tf = synth.full_tpc_1ms(seed=9, n_coll=1)
    ticket, res, o = run_both(trk, tf)
    nh = trk.stage(ticket, "tl_nhits")
    assert len(nh) == len(o["tl_nhits"])
    same = np.mean(nh == o["tl_nhits"])
    assert same >= 0.999, same
    th = trk.stage(ticket, "tl_hits")
    eq = 0
    for k in range(len(nh)):
        a = th[k][: nh[k]]
        b = o["tl_hits"][o["tl_off"][k]:o["tl_off"][k + 1]]
        eq += np.array_equal(a, b)
    assert eq / max(1, len(nh)) >= 0.999
    so, oo = trk.stage(ticket, "st_off"), o["st_off"]
    sh = trk.stage(ticket, "st_hits")
    g = {tuple(sh[so[i]:so[i + 1]]) for i in range(len(so) - 1)}
    r = [tuple(o["st_hits"][oo[i]:oo[i + 1]]) for i in range(len(oo) - 1)]
    assert np.mean([x in g for x in r]) >= 0.999
    trk.release(ticket, res)


def test_batch_equals_alone():
    """Each TF's result is the same alone and inside a batch."""
    tfs = [synth.single_sector(seed=s) for s in (1, 2)] + [synth.full_tpc_1ms(seed=3, n_coll=1)]
    with o2tpc.Tracker(flags=o2tpc.O2TPC_FLAG_NO_BATCHING) as a:
        alone = [a.track(tf) for tf in tfs]
    with o2tpc.Tracker(max_batch=8) as b:
        tickets = b.submit_many(tfs)
        mix = [b.poll(t) for t in tickets]
    assert all(m["stats"]["batch_size"] == len(tfs) for m in mix)
    for x, y in zip(alone, mix):
        for k in RESULT_KEYS:
            assert np.array_equal(x[k], y[k]), k


def test_empty_and_tiny_inputs():
    with o2tpc.Tracker() as t:
        e = t.track(float_tf([], [], [], []))
        assert e["status"] == 0 and e["n_tracks"] == 0
        s = t.track(float_tf([0, 0, 0], [10, 11, 12], [0.0, 0.01, 0.02], [100.0, 100.1, 100.2]))
        assert s["status"] == 0 and s["n_tracks"] == 0


def test_invalid_cluster_reported():
    with o2tpc.Tracker() as t:
        r = t.track(float_tf([0, 40], [10, 11], [0.0, 0.0], [1.0, 1.0]))
        assert r["status"] == o2tpc.O2TPC_EINVAL
        r = t.track(float_tf([0], [10], [np.nan], [1.0]))
        assert r["status"] == o2tpc.O2TPC_EINVAL
        ok = t.track(synth.single_sector())
        assert ok["status"] == 0 and ok["n_tracks"] > 10


def test_fp64_fallback_path_agrees():
    tf = synth.single_sector()
    with o2tpc.Tracker() as a:
        r32 = a.track(tf)
    with o2tpc.Tracker(flags=o2tpc.O2TPC_FLAG_FORCE_FP64) as b:
        r64 = b.track(tf)
    assert r64["stats"]["n_fp64_fallback"] == r64["n_tracks"]
    assert np.array_equal(r32["cluster_idx"], r64["cluster_idx"])
    o = oracle.run(tf)
    compare_tracks(r64, o, ZUNIT)


def test_torch_allocator_and_stream():
    torch = pytest.importorskip("torch")
    tf = synth.single_sector()
    with o2tpc.Tracker(torch_memory=True) as t:
        r = t.track(tf)
    o = oracle.run(tf)
    compare_tracks(r, o, ZUNIT)
    assert torch.cuda.memory_allocated() >= 0


def test_uploads_ahead_equal_in_stream_uploads():
    """Host-resident TFs queued behind a running batch are copied ahead on
    the copy stream; their results equal those of the in-stream copy path
    (the caching-allocator context copies in the batch's stream)."""
    pytest.importorskip("torch")
    tfs = [synth.single_sector(seed=s) for s in (4, 5)] + \
          [synth.full_tpc_1ms(seed=6 + k, n_coll=1, ntracks=800, fmt=synth.FMT_FIXED) for k in range(3)] + \
          [synth.single_sector(seed=9)]
    with o2tpc.Tracker(torch_memory=True, flags=o2tpc.O2TPC_FLAG_NO_BATCHING) as a:
        ref = [a.track(tf) for tf in tfs]
    with o2tpc.Tracker(max_batch=1) as b:
        tickets = [b.submit(tf) for tf in tfs]
        got = [b.poll(t) for t in tickets]
    for x, y in zip(ref, got):
        assert y["status"] == 0
        st = y["stats"]["ms_stage"]
        assert np.isfinite(st[12]) and np.isfinite(st[13]) and st[12] >= 0 and st[13] >= 0
        for k in RESULT_KEYS:
            assert np.array_equal(x[k], y[k]), k


def test_submit_many_is_all_or_nothing():
    tfs = [synth.single_sector(seed=s) for s in (11, 12, 13)]
    with o2tpc.Tracker(max_inflight=2) as t:
        with pytest.raises(o2tpc.O2TPCError) as e:
            t.submit_many(tfs)
        assert e.value.status == o2tpc.O2TPC_EAGAIN
        tickets = t.submit_many(tfs[:2])
        rs = [t.wait(k) for k in tickets]
        assert all(r["status"] == 0 and r["n_tracks"] > 10 for r in rs)


def test_launch_shapes_and_autotuner_leave_results_unchanged():
    """The tunable launch shapes (NeighboursFinder hits per block, cell-sort
    threads per row) and the autotuner's choice change no result bit."""
    tf = synth.full_tpc_1ms(seed=21, n_coll=3)
    assert tf.n >= 1 << 20
    keys = RESULT_KEYS
    with o2tpc.Tracker() as a:
        ref = a.track(tf)
        assert a.tuning()["tuned"] is False
    with o2tpc.Tracker(nf_hits_per_block=64, sort_threads_per_row=512, nf_staged=True) as b:
        other = b.track(tf)
    with o2tpc.Tracker(nf_staged=True) as b2:
        staged = b2.track(tf)
    with o2tpc.Tracker(flags=o2tpc.O2TPC_FLAG_AUTOTUNE) as c:
        tuned = c.track(tf)
        t = c.tuning()
    assert t["tuned"] and t["tuned_on_clusters"] == tf.n
    assert t["nf_hits_per_block"] in (64, 128, 256) and t["sort_threads_per_row"] in (128, 256, 512)
    assert all(v > 0 for v in t["nf_ms"] + t["sort_ms"])
    for r in (other, staged, tuned):
        for k in keys:
            assert np.array_equal(ref[k], r[k]), k
    with pytest.raises(o2tpc.O2TPCError):
        o2tpc.Tracker(nf_hits_per_block=100)


def test_captured_path_equals_regular_path():
    """Batches run as one CUDA graph launch (the captured path) give the same
    results as the regular path, on three different batches in a row (the
    replays alternate between two sets of result arrays, so the third reuses
    the first one's); with token capacities every batch overflows and reruns
    on the regular path, again with the same results."""
    keys = RESULT_KEYS
    sets = [synth.chunk_mix(seed=41, n_chunks=5) + [synth.single_sector(seed=42)],
            synth.chunk_mix(seed=43, n_chunks=7), synth.chunk_mix(seed=44, n_chunks=3)]
    with o2tpc.Tracker() as r:
        ref = [[r.poll(t) for t in r.submit_many(s)] for s in sets]
    for flags, captured in ((0, 1), (o2tpc.O2TPC_FLAG_GRAPH_TIGHT, 0)):
        with o2tpc.Tracker(graph_max_clusters=32 << 20, graph_max_tfs=8, flags=flags) as g:
            for s, rs in zip(sets, ref):
                got = [g.poll(t) for t in g.submit_many(s)]
                for x, y in zip(rs, got):
                    assert y["status"] == 0 and y["stats"]["captured"] == captured
                    for k in keys:
                        assert np.array_equal(x[k], y[k]), k


def test_tf_submitted_while_another_is_in_flight():
    """TFs submitted while another TF is on the device (the serving pattern:
    the later ones queue, share batches and run behind it) give the same
    results as each run alone, on the regular and on the captured path."""
    big = synth.full_tpc_1ms(seed=51, n_coll=10)
    later = [synth.single_sector(seed=52), synth.full_tpc_1ms(seed=53, n_coll=1), synth.single_sector(seed=54)]
    with o2tpc.Tracker(flags=o2tpc.O2TPC_FLAG_NO_BATCHING) as a:
        alone = [a.track(tf) for tf in [big] + later]
    for kw in ({}, {"graph_max_clusters": 32 << 20, "graph_max_tfs": 8}):
        with o2tpc.Tracker(max_batch=8, **kw) as t:
            first = t.submit(big)
            in_flight = t.poll(first, timeout_ms=0) is None
            tickets = [t.submit(tf) for tf in later]
            got = [t.poll(first)] + [t.poll(k) for k in tickets]
        assert in_flight, "the first TF had finished before the others were submitted"
        for x, y in zip(alone, got):
            assert y["status"] == 0
            for k in RESULT_KEYS:
                assert np.array_equal(x[k], y[k]), k


def test_float_time_input_parity(trk):
    """Float input with drift time instead of z: bit-exact integer stages and
    the track criteria against the oracle on the same input."""
    tf = synth.float_time_from_fixed(synth.full_tpc_1ms(seed=62, n_coll=2, fmt=synth.FMT_FIXED))
    ticket, res, o = run_both(trk, tf)
    compare_stages(trk, ticket, o)
    print(brief(compare_tracks(res, o, ZUNIT)))
    trk.release(ticket, res)


def test_autotuner_cache_file(tmp_path):
    """The autotuner's choice is written per GPU model and read back by the
    next context, which then counts as tuned without timing anything."""
    path = str(tmp_path / "tune.txt")
    tf = synth.full_tpc_1ms(seed=22, n_coll=3)
    with o2tpc.Tracker(flags=o2tpc.O2TPC_FLAG_AUTOTUNE, tune_cache_path=path) as a:
        a.track(tf)
        first = a.tuning()
    assert first["tuned"]
    name, vals = open(path).read().strip().split("\t")
    assert vals.split() == [str(first["nf_hits_per_block"]), str(int(first["nf_staged"])),
                            str(first["sort_threads_per_row"])]
    with o2tpc.Tracker(flags=o2tpc.O2TPC_FLAG_AUTOTUNE, tune_cache_path=path) as b:
        t = b.tuning()
        assert t["tuned"] and t["tuned_on_clusters"] == 0
        for k in ("nf_hits_per_block", "nf_staged", "sort_threads_per_row"):
            assert t[k] == first[k]


def test_cooperative_search_equals_per_lane_search():
    """The warp-cooperative row search of the following passes picks the
    same hits as the per-lane search: tracklets and tracks bit for bit."""
    tf = synth.full_tpc_1ms(seed=31, n_coll=3)
    out = []
    for flags in (0, o2tpc.O2TPC_FLAG_COOP_SEARCH):
        with o2tpc.Tracker(flags=flags | o2tpc.O2TPC_FLAG_KEEP_STAGES) as t:
            tk = t.submit(tf)
            r = t.poll(tk, keep=True)
            r["tl_nhits"] = t.stage(tk, "tl_nhits")
            r["tl_hits"] = t.stage(tk, "tl_hits")
            r["tl_state"] = t.stage(tk, "tl_state")
            t.release(tk, r)
            out.append(r)
    a, b = out
    assert a["n_tracks"] > 1000
    nh = a["tl_nhits"]
    assert np.array_equal(nh, b["tl_nhits"])
    for i in np.nonzero(nh > 0)[0]:  # slots past a tracklet's hits are never written
        assert np.array_equal(a["tl_hits"][i, :nh[i]], b["tl_hits"][i, :nh[i]]), i
    assert np.array_equal(a["tl_state"][nh > 0], b["tl_state"][nh > 0])
    for k in RESULT_KEYS:
        assert np.array_equal(a[k], b[k]), k
