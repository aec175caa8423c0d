"""Pins of the oracle's clusterizer (Sec. 2.2: raw ADC values to hits) against
what plain arithmetic and the generator fix:

* brute force on small random digit maps: a dense-grid formulation of the
  peak rule and the 3 x 3 centre of gravity gives the same records,
* hand-computed cases: a symmetric deposit lands on its cell centre, a
  two-digit deposit on its charge-weighted mean, a plateau of equal maxima
  gives one cluster, a noise-level digit none,
* unsorted input is rejected,
* digits made from a generated TF (charge spread over pads and time bins,
  noise, zero suppression) give back clusters close to the generated ones,
  and the tracker finds nearly the same tracks on them.
"""
import numpy as np
import pytest

import oracle
from paper_2106_03636_gb300 import synth


class D:
    def __init__(self, rows):  # rows: list of (sector, row, pad, time, adc), any order
        rows = sorted(rows, key=lambda r: (r[0], r[1], r[3], r[2]))
        a = np.array(rows, dtype=np.int64).reshape(-1, 5)
        self.sector, self.row, self.pad = a[:, 0].astype(np.uint8), a[:, 1].astype(np.uint8), a[:, 2].astype(np.uint8)
        self.time, self.adc = a[:, 3].astype(np.uint32), a[:, 4].astype(np.uint16)


def rec_fields(r):
    r = np.asarray(r, np.uint8).reshape(-1, 12)
    t64 = r[:, 0:4].copy().view("<u4").ravel()
    p64 = r[:, 4:6].copy().view("<u2").ravel()
    q = r[:, 6:8].copy().view("<u2").ravel()
    return t64, p64, q, r[:, 8], r[:, 9]


def dense_reference(rows, npad=16, ntime=16):
    """Peak rule and centre of gravity on dense per-row grids, cells visited
    in (time, pad) order."""
    out = []
    keys = sorted({(s, r) for s, r, _, _, _ in rows})
    for s, r in keys:
        g = np.zeros((ntime + 2, npad + 2), np.int64)  # one empty cell of margin
        have = np.zeros_like(g, bool)
        for s2, r2, p, t, a in rows:
            if (s2, r2) == (s, r):
                g[t + 1, p + 1] = a
                have[t + 1, p + 1] = True
        for t in range(ntime):
            for p in range(npad):
                a = g[t + 1, p + 1]
                if not have[t + 1, p + 1] or a < 3:
                    continue
                ok = True
                for dt in (-1, 0, 1):
                    for dp in (-1, 0, 1):
                        if (dt, dp) == (0, 0) or not have[t + 1 + dt, p + 1 + dp]:
                            continue
                        b = g[t + 1 + dt, p + 1 + dp]
                        before = (dt, dp) < (0, 0)
                        if (before and not a > b) or (not before and not a >= b):
                            ok = False
                w = g[t:t + 3, p:p + 3] * have[t:t + 3, p:p + 3]
                if not ok:
                    continue
                q = int(w.sum())
                pc = sum(int(w[i, j]) * (64 * (p + j - 1) + 32) for i in range(3) for j in range(3))
                tc = sum(int(w[i, j]) * (64 * (t + i - 1) + 32) for i in range(3) for j in range(3))
                out.append(((2 * tc + q) // (2 * q), (2 * pc + q) // (2 * q), min(q, 65535), r, s))
    return out


@pytest.mark.parametrize("seed", range(8))
def test_brute_force_small_maps(seed):
    rng = np.random.default_rng(seed)
    rows = set()
    for s, r in ((0, 3), (0, 4), (20, 100)):
        for _ in range(60):
            rows.add((s, r, int(rng.integers(0, 16)), int(rng.integers(0, 16))))
    digits = [(s, r, p, t, int(rng.integers(2, 12))) for s, r, p, t in rows]
    got = list(zip(*rec_fields(oracle.clusterize(D(digits)))))
    want = dense_reference(digits)
    assert [tuple(int(v) for v in g) for g in got] == [tuple(w) for w in want]


def test_hand_computed_cases():
    cross = [(1, 2, 7, 5, 20), (1, 2, 6, 5, 6), (1, 2, 8, 5, 6), (1, 2, 7, 4, 6), (1, 2, 7, 6, 6)]
    t, p, q, r, s = rec_fields(oracle.clusterize(D(cross)))
    assert list(t) == [64 * 5 + 32] and list(p) == [64 * 7 + 32] and list(q) == [44] and r[0] == 2 and s[0] == 1
    pair = [(0, 0, 7, 5, 10), (0, 0, 8, 5, 5)]
    t, p, q, _, _ = rec_fields(oracle.clusterize(D(pair)))
    assert list(p) == [501] and list(t) == [352] and list(q) == [15]  # (10*480 + 5*544) / 15 = 501.33
    plateau = [(0, 0, 3, 9, 8), (0, 0, 4, 9, 8)]
    t, p, q, _, _ = rec_fields(oracle.clusterize(D(plateau)))
    assert len(t) == 1 and p[0] == (8 * (64 * 3 + 32) + 8 * (64 * 4 + 32)) // 16
    assert len(oracle.clusterize(D([(0, 0, 3, 9, 2)]))) == 0


def test_unsorted_rejected():
    d = D([(0, 0, 1, 1, 5), (0, 0, 2, 1, 5)])
    d.pad = d.pad[::-1].copy()
    with pytest.raises(oracle.OracleError):
        oracle.clusterize(d)


def test_clusters_from_generated_digits():
    tf = synth.single_sector(seed=5, fmt=synth.FMT_FIXED)
    d = synth.digits_from(tf, seed=9)
    rec = oracle.clusterize(d)
    t64, p64, q, r, s = rec_fields(rec)
    g = tf.packed
    gt, gp = g[:, 0:4].copy().view("<u4").ravel(), g[:, 4:6].copy().view("<u2").ravel()
    gr, gs = g[:, 8], g[:, 9]
    # nearest reconstructed cluster of the same row for every generated one
    close = 0
    for row in np.unique(gr):
        a = np.nonzero(gr == row)[0]
        b = np.nonzero(r == row)[0]
        if len(b) == 0:
            continue
        dp = (gp[a][:, None].astype(np.int64) - p64[b][None, :]) / 64.0
        dt = (gt[a][:, None].astype(np.int64) - t64[b][None, :]) / 64.0
        dist = np.hypot(dp, dt)
        j = dist.argmin(axis=1)
        close += int(np.sum((np.abs(dp[np.arange(len(a)), j]) < 0.3) & (np.abs(dt[np.arange(len(a)), j]) < 0.3)))
    assert close > 0.85 * tf.n
    # the tracker on the clusterized TF finds nearly the same tracks
    tf2 = synth.TimeFrame(n=len(rec), fmt=synth.FMT_FIXED, sector=s.copy(), row=r.copy(),
                          packed=np.ascontiguousarray(rec), bz=tf.bz, vdrift=tf.vdrift)
    o1 = oracle.run(tf, fields=["trk_off"])
    o2 = oracle.run(tf2, fields=["trk_off"])
    n1, n2 = len(o1["trk_off"]) - 1, len(o2["trk_off"]) - 1
    assert abs(n2 - n1) <= 0.1 * n1
    assert o2["trk_off"][-1] > 0.9 * o1["trk_off"][-1]
