"""CUDA path vs the oracle with the two optional refinements (needs a GB300):
the NeighboursFinder with row step 2 (O2TPC_FLAG_ROW_STEP2) on Time Frames
that lost clusters, and the angle-dependent cluster errors
(O2TPC_FLAG_ANGULAR_ERRORS) on clusters smeared that way.  Integer stages
bit-exact, tracks by the same criteria as the default path."""
import numpy as np
import pytest

import oracle
from parity import assert_criteria, brief, compare_stages, compare_tracks, pool
from paper_2106_03636_gb300 import o2tpc, synth

pytestmark = pytest.mark.gpu

ZUNIT = 0.003125 * 2.58


def run_both(flags, tf, **okw):
    with o2tpc.Tracker(flags=flags | o2tpc.O2TPC_FLAG_KEEP_STAGES) as trk:
        tk = trk.submit(tf)
        res = trk.poll(tk, keep=True)
        assert res["status"] == 0
        o = oracle.run(tf, **okw)
        compare_stages(trk, tk, o)
        trk.release(tk, res)
    return res, o


def test_row_step2_parity():
    tf = synth.full_tpc_1ms(seed=71, n_coll=3, row_drop=0.2)
    res, o = run_both(o2tpc.O2TPC_FLAG_ROW_STEP2, tf, row_step2=True)
    # links across a missing row exist and are the oracle's
    plain = oracle.run(tf, fields=["up_raw"])
    assert (o["up_raw"] >= 0).sum() > (plain["up_raw"] >= 0).sum() + 1000
    print(brief(compare_tracks(res, o, ZUNIT)))


# With the angle-dependent errors the out-of-tolerance share of well-posed
# fits is about 0.14 % (12 of 8672 on the 3-collision frame, 11 of them low-pT
# tracks with |q/pT| > 5 / GeV, against 0.04-0.07 % with constant errors):
# this option's parameters are held to 0.2 %; cluster sets and the integer
# stages keep the full criteria.
ANGULAR_BAD_FRAC = 0.002


def test_angular_errors_parity():
    tf = synth.full_tpc_1ms(seed=72, n_coll=3, angular_errors=True)
    res, o = run_both(o2tpc.O2TPC_FLAG_ANGULAR_ERRORS, tf, angular_errors=True)
    print(brief(compare_tracks(res, o, ZUNIT, bad_frac=ANGULAR_BAD_FRAC)))


def test_both_refinements_dense_parity():
    """Dense single-sector frames (1500 primaries) that lost 15 % of their
    clusters, smeared with the angle-dependent errors, both refinements on."""
    flags = o2tpc.O2TPC_FLAG_ROW_STEP2 | o2tpc.O2TPC_FLAG_ANGULAR_ERRORS
    reps = []
    for seed in (91, 92, 93, 94):
        tf = synth.single_sector(seed=seed, ntracks=1500, row_drop=0.15, angular_errors=True)
        res, o = run_both(flags, tf, row_step2=True, angular_errors=True)
        reps.append(compare_tracks(res, o, ZUNIT, check=False))
    rep = pool(reps)
    print(brief(rep))
    assert_criteria(rep, ANGULAR_BAD_FRAC)


def test_refinements_off_by_default():
    """Without the flags the links across missing rows are absent and the
    results equal those of a context that never heard of the options."""
    tf = synth.single_sector(seed=93, row_drop=0.2)
    with o2tpc.Tracker(flags=o2tpc.O2TPC_FLAG_KEEP_STAGES) as t:
        tk = t.submit(tf)
        r = t.poll(tk, keep=True)
        up = t.stage(tk, "up_raw")
        t.release(tk, r)
    o = oracle.run(tf, fields=["up_raw"])
    assert np.array_equal(up, o["up_raw"])
