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
