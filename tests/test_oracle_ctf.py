"""Pins of the oracle's compressed Time Frame (Sec. 2.2: hit removal, track-model
compression, lossless ANS entropy coding) against what mathematics and the
generator fix, not against the oracle's own formulas:

* the entropy coder is lossless on streams of any length and distribution
  (empty, one symbol, uniform, skewed, around the chunk size),
* its payload lies between the Shannon bound of the stream and the cost of
  the quantised table plus the per-chunk state bytes,
* the frequency tables sum to 4096 and keep every present symbol,
* a TF decodes to exactly its kept clusters: the kept tracks' clusters in
  order (tracks by first input index), then the others in sorted order,
* the removed clusters belong to soft particles (generator truth),
* the straight-line track model predicts noise-free helices to a few units,
* a damaged blob is rejected.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2106_03636_gb300 import synth


def shannon_bytes(a):
    if len(a) == 0:
        return 0.0
    c = np.bincount(a, minlength=256).astype(np.float64)
    p = c[c > 0] / len(a)
    return -len(a) * float(np.sum(p * np.log2(p))) / 8.0


def table_bytes(a, f):
    c = np.bincount(a, minlength=256)
    nz = c > 0
    return float(np.sum(c[nz] * np.log2(4096.0 / f[nz]))) / 8.0


@pytest.mark.parametrize("kind,n", [
    ("empty", 0), ("one", 1), ("const", 50000), ("uniform", 4096), ("uniform", 4097), ("geometric", 100000),
    ("two", 40000), ("sparse", 70000),
])
def test_rans_lossless_and_near_entropy(kind, n):
    rng = np.random.default_rng(hash(kind) % 1000 + n)
    if kind in ("empty", "one", "const"):
        a = np.full(n, 7, np.uint8)
    elif kind == "uniform":
        a = rng.integers(0, 256, n).astype(np.uint8)
    elif kind == "geometric":
        a = np.minimum(rng.geometric(0.3, n), 255).astype(np.uint8)
    elif kind == "two":
        a = (rng.random(n) < 0.01).astype(np.uint8) * 200
    else:
        a = rng.choice(np.array([0, 3, 250], np.uint8), n, p=[0.98, 0.0199, 0.0001])
    blob = oracle.rans_encode(a)
    assert np.array_equal(oracle.rans_decode(blob), a)
    nch = (n + 4095) // 4096
    payload = len(blob) - 8 - 512 - 4 * nch
    f = np.frombuffer(blob[8:520].tobytes(), dtype="<u2")
    assert payload >= shannon_bytes(a) - 1e-6 * n
    assert payload <= table_bytes(a, f) + 6 * nch + 1


def test_normalisation():
    c = np.zeros(256, np.uint64)
    assert np.all(oracle.ctf_normalize(c) == 0)
    c[[10, 20, 30]] = 5
    f = oracle.ctf_normalize(c)
    assert f.sum() == 4096 and list(f[[10, 20, 30]]) == [1366, 1365, 1365]
    rng = np.random.default_rng(3)
    for _ in range(20):
        c = rng.integers(0, 3, 256).astype(np.uint64) * rng.integers(1, 10 ** 6, 256).astype(np.uint64)
        f = oracle.ctf_normalize(c)
        assert f.sum() == 4096
        assert np.array_equal(f > 0, c > 0)


def kept_sequence(tf, o):
    """The cluster sequence the format defines, built here from the oracle's
    tracks and sorted order with plain numpy."""
    sec, row = o["rid"] // 152, o["rid"] % 152
    off, cl, q = o["trk_off"], o["trk_cl"], o["trk_par"][:, 4]
    on = np.zeros(tf.n, bool)
    for t in range(len(q)):
        on[cl[off[t]:off[t + 1]]] = True
    kept = [t for t in range(len(q)) if off[t + 1] > off[t] and abs(q[t]) <= 10.0]
    kept.sort(key=lambda t: cl[off[t]])
    idx = [c for t in kept for c in cl[off[t]:off[t + 1]]]
    lens = [off[t + 1] - off[t] for t in kept]
    idx += [h for h in o["sorted_orig"] if not on[h]]
    idx = np.asarray(idx, np.int64)
    return idx, np.asarray(lens), sec, row


def test_ctf_decodes_to_the_kept_clusters():
    tf = synth.full_tpc_1ms(seed=31, n_coll=2)
    o = oracle.run(tf, compress=True)
    d = oracle.ctf_decode(o["ctf"])
    idx, lens, sec, row = kept_sequence(tf, o)
    assert np.array_equal(d["track_len"], lens)
    assert np.array_equal(d["sector"], sec[idx]) and np.array_equal(d["row"], row[idx])
    assert np.array_equal(d["y"], o["yu"][idx]) and np.array_equal(d["z"], o["zu"][idx])
    # a few bytes per cluster instead of the 12-byte record
    assert len(o["ctf"]) < 3.0 * tf.n
    # the standalone encoder over the same arrays gives the same bytes
    again = oracle.ctf_encode(sec, row, o["yu"], o["zu"], o["trk_off"], o["trk_cl"], o["trk_par"][:, 4],
                              o["sorted_orig"])
    assert np.array_equal(again, o["ctf"])


def test_removed_clusters_are_soft_particles():
    tf = synth.full_tpc_1ms(seed=32, n_coll=2)
    o = oracle.run(tf, compress=True)
    d = oracle.ctf_decode(o["ctf"])
    removed = tf.n - len(d["sector"])
    assert removed > 0
    on_removed = []
    off, cl, q = o["trk_off"], o["trk_cl"], o["trk_par"][:, 4]
    for t in range(len(q)):
        if abs(q[t]) > 10.0:
            on_removed.extend(cl[off[t]:off[t + 1]].tolist())
    assert len(on_removed) == removed
    tt = tf.truth_track[np.asarray(on_removed)]
    pt = tf.truth["pt"][tt[tt >= 0]]
    assert np.mean(pt < 0.12) > 0.9


def test_track_model_on_noise_free_helices():
    """Without smearing, a straight line through the previous two clusters
    misses the next one only by the helix's curvature and the integer
    rounding: the residual streams are nearly constant and cost well under a
    byte per track cluster (about 2.4 with the generator's smearing)."""
    tf = synth.single_sector(seed=11, ntracks=60, sigma_y=0.0, sigma_z=0.0, noise_frac=0.0)
    o = oracle.run(tf, compress=True)
    d = oracle.ctf_decode(o["ctf"])
    ntc = int(d["track_len"].sum())
    assert ntc > 0.9 * tf.n
    assert len(o["ctf"]) - 24 - 10 * 520 < 1.0 * ntc


def test_damaged_blob_rejected():
    tf = synth.single_sector(seed=12)
    o = oracle.run(tf, compress=True)
    blob = o["ctf"]
    with pytest.raises(oracle.OracleError):
        oracle.ctf_decode(blob[: len(blob) // 2])
    bad = blob.copy()
    bad[0] ^= 1
    with pytest.raises(oracle.OracleError):
        oracle.ctf_decode(bad)
