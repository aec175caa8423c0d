"""The library's host decoder of compressed TFs (o2tpc_ctf_decode, no GPU
needed) against the oracle's decoder, on blobs the oracle wrote: the same
cluster sequence, and damaged blobs rejected."""
import numpy as np
import pytest

import oracle
from paper_2106_03636_gb300 import o2tpc, synth


@pytest.mark.parametrize("make", [
    lambda: synth.single_sector(seed=21),
    lambda: synth.full_tpc_1ms(seed=22, n_coll=2, fmt=synth.FMT_FIXED),
    lambda: synth.single_sector(seed=23, sigma_y=0.0, sigma_z=0.0, noise_frac=0.0),
])
def test_host_decoder_equals_oracle_decoder(make):
    tf = make()
    blob = oracle.run(tf, compress=True)["ctf"]
    want = oracle.ctf_decode(blob)
    got = o2tpc.ctf_decode(blob)
    for k, kw in (("sector", "sector"), ("row", "row"), ("y", "y"), ("zeta", "z")):
        assert np.array_equal(got[k], want[kw]), k
    assert np.array_equal(got["track_len"].astype(np.int64), want["track_len"])


def test_empty_and_damaged():
    from helpers import float_tf
    empty = oracle.run(float_tf([], [], [], []), compress=True)["ctf"]
    d = o2tpc.ctf_decode(empty)
    assert len(d["sector"]) == 0 and len(d["track_len"]) == 0
    blob = oracle.run(synth.single_sector(seed=24), compress=True)["ctf"]
    for bad in (blob[:100], blob[: len(blob) - 1], np.concatenate([blob, np.zeros(3, np.uint8)])):
        with pytest.raises(o2tpc.O2TPCError):
            o2tpc.ctf_decode(bad)
    flipped = blob.copy()
    flipped[len(blob) // 2] ^= 0x40
    with pytest.raises(o2tpc.O2TPCError):
        o2tpc.ctf_decode(flipped)


def test_decoded_tf_tracks_like_the_original():
    """Compress, decode to fixed-format records, track again (oracle): the
    kept tracks come back with the same cluster positions."""
    tf = synth.full_tpc_1ms(seed=25, n_coll=2, fmt=synth.FMT_FIXED)
    o = oracle.run(tf, compress=True)
    d = o2tpc.ctf_decode(o["ctf"])
    rec = d["records"]
    # the kept clusters' records equal the input records up to the charge
    tf_pos = {tuple(r) for r in np.concatenate([tf.packed[:, :6], tf.packed[:, 8:10]], axis=1).tolist()}
    dec_pos = [tuple(r) for r in np.concatenate([rec[:, :6], rec[:, 8:10]], axis=1).tolist()]
    assert all(p in tf_pos for p in dec_pos)
    tf2 = synth.TimeFrame(n=len(rec), fmt=synth.FMT_FIXED, sector=rec[:, 9].copy(), row=rec[:, 8].copy(),
                          packed=np.ascontiguousarray(rec), bz=tf.bz, vdrift=tf.vdrift)
    o2 = oracle.run(tf2, fields=["trk_off", "trk_par"])
    kept = np.abs(o["trk_par"][:, 4]) <= 10.0
    n_kept, n2 = int(kept.sum()), len(o2["trk_off"]) - 1
    assert abs(n2 - n_kept) <= 0.02 * n_kept
