"""Pins of the oracle's continuous-readout completion (Sec. 2: tracks are
assigned to collisions after tracking) against what the generator and plain
geometry fix, not against the oracle's own formulas:

* the closest-approach arc length agrees with a brute-force scan of the
  circle, and with the straight line at zero curvature,
* every pair linked across the central membrane joins two pieces of one
  generated particle, and its t0 equals that particle's collision time
  (no vertex assumption is involved),
* most particles seen on both sides of the membrane get linked,
* the vertex t0 of the other tracks has unit pulls against the truth (the
  generator draws z_vertex ~ N(0, 5 cm)),
* the t0 bounds contain the truth,
* with well separated collisions nearly every track goes to its own one,
* the links form a greedy matching of the candidate pairs in (chi2, a, b).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2106_03636_gb300 import synth

COLL = [40.0, 190.0, 340.0, 490.0, 640.0, 790.0]


@pytest.fixture(scope="module")
def run():
    tf = synth.generate(seed=77, t0=COLL, ntracks=[1800] * len(COLL), zvtx_sigma=5.0, name="six_separated")
    o = oracle.run(tf)
    tt = tf.truth_track
    nt = len(o["trk_x"])
    maj = np.full(nt, -1)
    for i in range(nt):
        g = tt[o["trk_cl"][o["trk_off"][i]:o["trk_off"][i + 1]]]
        g = g[g >= 0]
        if len(g):
            v, c = np.unique(g, return_counts=True)
            maj[i] = v[c.argmax()]
    return tf, o, maj


def _circle_scan(x0, y0, snp, k, span=400.0, n=400001):
    """Nearest point to the origin within half a turn either way."""
    if k != 0:
        span = min(span, math.pi / abs(k))
    csp = math.sqrt(1 - snp * snp)
    s = np.linspace(-span, span, n)
    if k == 0:
        px, py = x0 + s * csp, y0 + s * snp
    else:
        phi0 = math.atan2(snp, csp)
        cx, cy = x0 - snp / k, y0 + csp / k
        ph = phi0 + k * s
        px, py = cx + np.sin(ph) / k, cy - np.cos(ph) / k
    j = int(np.argmin(px * px + py * py))
    return s[j], s[1] - s[0]


@pytest.mark.parametrize("x0,y0,snp,k", [
    (100.0, 3.0, 0.1, 0.002), (120.0, -10.0, -0.3, -0.004), (90.0, 5.0, 0.05, 0.0),
    (150.0, 20.0, 0.4, 0.012), (30.0, 1.0, 0.2, 0.03),  # origin inside the circle
    (85.0, -2.0, -0.05, 1e-9),
])
def test_dca_arc_brute_force(x0, y0, snp, k):
    s_ref, ds = _circle_scan(x0, y0, snp, k)
    assert abs(oracle.dca_arc(x0, y0, snp, k) - s_ref) <= 2 * ds
    if k == 0.0:
        csp = math.sqrt(1 - snp * snp)
        assert oracle.dca_arc(x0, y0, snp, k) == pytest.approx(-(x0 * csp + y0 * snp), abs=1e-12)


def test_membrane_links_are_one_particle_with_true_t0(run):
    tf, o, maj = run
    mate = o["trk_mate"]
    a = np.nonzero(mate >= 0)[0]
    assert len(a) >= 40, "too few membrane crossings to pin anything"
    assert np.all(mate[mate[a]] == a)
    assert np.all(o["trk_flags"][a] & 8)
    ok = maj[a] >= 0
    assert np.mean(maj[a][ok] == maj[mate[a]][ok]) >= 0.99
    sides = (o["trk_sector"][a] < 18) != (o["trk_sector"][mate[a]] < 18)
    assert np.all(sides)
    t0_true = tf.truth["t0"][maj[a][ok]]
    d = o["trk_t0"][a][ok] - t0_true
    assert np.median(np.abs(d)) < 0.03 and np.max(np.abs(d)) < 0.2  # us; 0.2 us = 0.5 cm of drift
    # the stated error is honest
    assert np.mean(np.abs(d) < 4 * o["trk_t0err"][a][ok] + 0.01) > 0.95


def test_membrane_link_efficiency(run):
    tf, o, maj = run
    nt = len(o["trk_x"])
    side = (o["trk_sector"] < 18).astype(int)
    by = {}
    for i in range(nt):
        if maj[i] >= 0:
            by.setdefault(int(maj[i]), []).append(i)
    both = [v for v in by.values() if len(v) == 2 and side[v[0]] != side[v[1]]]
    assert len(both) >= 40
    linked = sum(1 for v in both if o["trk_mate"][v[0]] == v[1])
    assert linked / len(both) >= 0.85


def test_vertex_t0_pulls_and_bounds(run):
    tf, o, maj = run
    u = (o["trk_mate"] < 0) & (maj >= 0) & (o["trk_ndf"] > 20)
    d = o["trk_t0"][u] - tf.truth["t0"][maj[u]]
    pull = d / o["trk_t0err"][u]
    # primaries dominate; the 5 cm beam spot sets the width
    assert abs(np.median(pull)) < 0.1
    assert 0.8 < np.std(pull[np.abs(pull) < 5]) < 1.2
    assert np.mean(np.abs(pull) < 3) > 0.97
    ok = maj >= 0
    t0 = tf.truth["t0"][maj[ok]]
    inside = (t0 >= o["trk_t0lo"][ok] - 0.3) & (t0 <= o["trk_t0hi"][ok] + 0.3)
    assert np.mean(inside) > 0.999
    assert np.all(o["trk_t0lo"] <= o["trk_t0hi"])
    # vertex t0 is clamped into the bounds; a membrane t0 may sit below the
    # lower bound by the cluster noise the link tolerates (1 cm of drift)
    u = o["trk_mate"] < 0
    assert np.all((o["trk_t0"][u] >= o["trk_t0lo"][u] - 1e-9) & (o["trk_t0"][u] <= o["trk_t0hi"][u] + 1e-9))
    m = ~u
    assert np.all((o["trk_t0"][m] >= o["trk_t0lo"][m] - 1.0 / tf.vdrift - 1e-9) & (o["trk_t0"][m] <= o["trk_t0hi"][m]))


def test_assignment_to_separated_collisions(run):
    tf, o, maj = run
    ok = maj >= 0
    truth_coll = tf.truth["coll"][maj[ok]]
    assert np.mean(o["trk_coll"][ok] == truth_coll) > 0.99
    # without an interaction record nothing is assigned
    o2 = oracle.run(tf, coll_time=[], fields=["trk_coll", "trk_t0"])
    assert np.all(o2["trk_coll"] == -1)
    np.testing.assert_array_equal(o2["trk_t0"], o["trk_t0"])


def test_links_are_the_greedy_matching(run):
    tf, o, maj = run
    ab, c2 = o["mpair_ab"], o["mpair_chi2"]
    order = np.lexsort((ab[:, 1], ab[:, 0], c2))
    assert np.all(order == np.arange(len(c2))), "candidate pairs come sorted by (chi2, a, b)"
    assert np.all(c2 <= 25.0)
    taken = {}
    for (a, b) in ab:
        if a in taken or b in taken:
            continue
        taken[a] = b
        taken[b] = a
    mate = o["trk_mate"]
    want = np.full(len(mate), -1)
    for k, v in taken.items():
        want[k] = v
    np.testing.assert_array_equal(mate, want)
