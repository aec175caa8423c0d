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
