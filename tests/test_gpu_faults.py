"""Faults made on the host, with no device fault (allocation failures through
the allocator callback), and repeatability of whole results."""
import numpy as np
import pytest

from paper_2106_03636_gb300 import o2tpc, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KEYS = ("offsets", "cluster_idx", "par", "cov", "chi2", "ndf", "flags", "zeta_ref", "t0", "t0_err", "mate",
        "collision")


def test_allocation_failure_reported_and_context_recovers():
    state = {"fail": False, "calls": 0}

    def fail(nbytes):
        state["calls"] += 1
        return state["fail"]

    tf = synth.single_sector(seed=41)
    with o2tpc.Tracker(torch_memory=True, fail_alloc=fail) as t:
        ref = t.track(tf)
        state["fail"] = True
        with pytest.raises(o2tpc.O2TPCError) as e:
            t.track(tf)
        assert e.value.status == o2tpc.O2TPC_ENOMEM
        state["fail"] = False
        again = t.track(tf)
        for k in KEYS:
            assert np.array_equal(ref[k], again[k]), k
    assert state["calls"] > 0


def test_results_repeat_bit_for_bit():
    tf = synth.full_tpc_1ms(seed=42, n_coll=2)
    with o2tpc.Tracker() as t:
        runs = [t.track(tf) for _ in range(5)]
    for r in runs[1:]:
        for k in KEYS:
            assert np.array_equal(runs[0][k], r[k]), k


def test_bounded_wait_that_runs_out_is_reported():
    """The staged NeighboursFinder's slab waits are bounded.  With the
    injected fault the barrier is armed but no copy is issued, so every wait
    runs out (nothing in flight): the blocks read global memory instead, the
    links and tracks are those of the regular run, the batch reports
    stats.events bit 0, and the context goes on working."""
    tf = synth.full_tpc_1ms(seed=43, n_coll=3)
    with o2tpc.Tracker(nf_staged=True, flags=o2tpc.O2TPC_FLAG_KEEP_STAGES) as a:
        tk = a.submit(tf)
        ref = a.poll(tk, keep=True)
        ref_links = [a.stage(tk, nm) for nm in ("up_raw", "dn_raw")]
        a.release(tk, ref)
    assert ref["stats"]["events"] & 1 == 0
    with o2tpc.Tracker(nf_staged=True, debug_inject=1, flags=o2tpc.O2TPC_FLAG_KEEP_STAGES) as b:
        for _ in range(2):  # the context stays usable after a wait ran out
            tk = b.submit(tf)
            got = b.poll(tk, keep=True)
            links = [b.stage(tk, nm) for nm in ("up_raw", "dn_raw")]
            b.release(tk, got)
            assert got["status"] == 0 and got["stats"]["events"] & 1 == 1
            for x, y in zip(ref_links, links):
                assert np.array_equal(x, y)
            for k in KEYS:
                assert np.array_equal(ref[k], got[k]), k


def test_tf_beyond_the_memory_budget_is_refused():
    """A TF whose footprint (160 B per cluster + 64 MB) exceeds mem_budget is
    refused at submission with ETOOBIG (the paper's case for processing a
    TF elsewhere, Sec. 3.1.3); one that fits is tracked."""
    small = synth.single_sector(seed=44)
    big = synth.full_tpc_1ms(seed=45, n_coll=1, ntracks=600)
    budget = 160 * small.n + (64 << 20) + (1 << 20)
    assert 160 * big.n + (64 << 20) > budget
    with o2tpc.Tracker(mem_budget=budget) as t:
        with pytest.raises(o2tpc.O2TPCError) as e:
            t.submit(big)
        assert e.value.status == o2tpc.O2TPC_ETOOBIG
        r = t.track(small)
        assert r["status"] == 0 and r["n_tracks"] > 10


def test_tfs_wait_for_memory_then_run():
    """With a budget that holds one TF, TFs submitted together are admitted
    one at a time as memory frees (batches of one); each result equals the
    result of the same TFs batched together under the default budget."""
    tfs = [synth.single_sector(seed=s) for s in (46, 47, 48)]
    one = 160 * max(t.n for t in tfs) + (64 << 20) + (1 << 20)
    with o2tpc.Tracker(max_batch=8) as a:
        together = [a.poll(tk) for tk in a.submit_many(tfs)]
    assert all(r["stats"]["batch_size"] == 3 for r in together)
    with o2tpc.Tracker(max_batch=8, mem_budget=one) as b:
        tickets = b.submit_many(tfs)
        apart = [b.poll(tk) for tk in tickets]
    assert all(r["status"] == 0 and r["stats"]["batch_size"] == 1 for r in apart)
    for x, y in zip(together, apart):
        for k in KEYS:
            assert np.array_equal(x[k], y[k]), k
