"""Clusterizer of the CUDA path (o2tpc_clusterize) against the oracle: the
records are integer results and must be bit-identical, on generated raw
digits and on small random digit maps; edge cases; and raw digits -> clusters
-> tracks end to end against the oracle run on the oracle's own clusters."""
import numpy as np
import pytest

import oracle
from parity import brief, compare_tracks
from paper_2106_03636_gb300 import o2tpc, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ZUNIT = 0.003125 * 2.58


def dev(d):
    return {k: torch.from_numpy(np.ascontiguousarray(getattr(d, k))).cuda()
            for k in ("sector", "row", "pad", "time", "adc")}


def run(d, cap=None):
    rc, rec, n = o2tpc.clusterize(dev(d), cap=cap)
    torch.cuda.synchronize()
    return rc, rec.cpu().numpy(), n


@pytest.mark.parametrize("make", [
    lambda: synth.single_sector(seed=5, fmt=synth.FMT_FIXED),
    lambda: synth.full_tpc_1ms(seed=6, n_coll=2, fmt=synth.FMT_FIXED),
])
def test_clusterizer_bit_exact(make):
    d = synth.digits_from(make(), seed=3)
    rc, rec, n = run(d)
    assert rc == o2tpc.O2TPC_OK
    want = oracle.clusterize(d)
    assert n == len(want)
    assert np.array_equal(rec, want)


def test_small_random_maps():
    rng = np.random.default_rng(4)
    for _ in range(5):
        cells = {(int(s), int(r), int(rng.integers(0, 20)), int(rng.integers(0, 20)))
                 for s, r in ((0, 0), (3, 151), (35, 7)) for _ in range(120)}
        rows = sorted((s, r, t, p) for s, r, p, t in cells)
        a = np.array(rows, np.int64)

        class D:
            pass
        d = D()
        d.sector, d.row = a[:, 0].astype(np.uint8), a[:, 1].astype(np.uint8)
        d.time, d.pad = a[:, 2].astype(np.uint32), a[:, 3].astype(np.uint8)
        d.adc = rng.integers(2, 15, len(a)).astype(np.uint16)
        rc, rec, n = run(d)
        assert rc == o2tpc.O2TPC_OK and np.array_equal(rec, oracle.clusterize(d))


def test_edge_cases():
    d = synth.digits_from(synth.single_sector(seed=7, fmt=synth.FMT_FIXED), seed=1)
    rc, rec, n = run(d, cap=3)
    assert rc == o2tpc.O2TPC_ETOOBIG and n == len(oracle.clusterize(d))
    bad = dev(d)
    bad["pad"] = bad["pad"].flip(0).contiguous()
    rc, _, _ = o2tpc.clusterize(bad)
    assert rc == o2tpc.O2TPC_EINVAL
    bad = dev(d)
    bad["sector"][0] = 40
    rc, _, _ = o2tpc.clusterize(bad)
    assert rc == o2tpc.O2TPC_EINVAL
    empty = {k: v[:0] for k, v in dev(d).items()}
    rc, rec, n = o2tpc.clusterize(empty)
    assert rc == o2tpc.O2TPC_OK and n == 0


def test_raw_digits_to_tracks():
    tf = synth.full_tpc_1ms(seed=8, n_coll=3, fmt=synth.FMT_FIXED)
    d = synth.digits_from(tf, seed=2)
    rc, rec_dev, n = o2tpc.clusterize(dev(d))
    assert rc == o2tpc.O2TPC_OK
    rec = rec_dev.cpu().numpy()
    want = oracle.clusterize(d)
    assert np.array_equal(rec, want)
    tf2 = synth.TimeFrame(n=n, fmt=synth.FMT_FIXED, sector=rec[:, 9].copy(), row=rec[:, 8].copy(),
                          packed=np.ascontiguousarray(rec), bz=tf.bz, vdrift=tf.vdrift)
    with o2tpc.Tracker() as t:
        res = t.track(tf2, location=o2tpc.O2TPC_LOC_DEVICE, arrays={"packed": rec_dev.contiguous()})
    assert res["status"] == 0
    print(brief(compare_tracks(res, oracle.run(tf2), ZUNIT)))
