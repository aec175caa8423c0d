"""Pins of the oracle's integer stages (grid binning and sort,
NeighboursFinder, NeighboursCleaner, StartHitsFinder):

* sort: permutation + key order + every hit inside the cell rectangle it is
  filed under (an independent statement of what the grid means),
* neighbours: brute force over all pairs of the adjacent rows (no grid),
  including exact-duplicate hits that force metric ties,
* cleaner / starts: link reciprocity and chain-head invariants,
* a hand-worked example (tests/golden/nf_handworked.json).
"""
import json
import os
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
from helpers import float_tf, npads
from paper_2106_03636_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fixed_tf(sector, row, pad64, time64, vdrift=2.58, bz=0.5):
    n = len(sector)
    rec = np.zeros((n, 12), np.uint8)
    rec[:, 0:4] = np.asarray(time64, np.uint32).view(np.uint8).reshape(n, 4)
    rec[:, 4:6] = np.asarray(pad64, np.uint16).view(np.uint8).reshape(n, 2)
    rec[:, 8] = row
    rec[:, 9] = sector
    return SimpleNamespace(n=n, fmt=1, packed=rec, sector=None, row=None, y=None, z=None, bz=bz, vdrift=vdrift)


def dense_tf(seed, n_rows=6, per_row=80, row0=20, dup_frac=0.15, sector=5):
    """Small dense patch: hits of a few adjacent rows concentrated in a
    3 cm x 4 cm region so that windows hold many candidates; some hits are
    exact duplicates of others to force metric ties."""
    rng = np.random.default_rng(seed)
    sec, row, y, z = [], [], [], []
    for r in range(row0, row0 + n_rows):
        yy = rng.uniform(-1.5, 1.5, per_row)
        zz = rng.uniform(10.0, 14.0, per_row)
        nd = int(dup_frac * per_row)
        yy[:nd] = yy[per_row - nd:]
        zz[:nd] = zz[per_row - nd:]
        sec += [sector] * per_row
        row += [r] * per_row
        y += list(yy)
        z += list(zz)
    perm = rng.permutation(len(sec))
    return float_tf(np.array(sec)[perm], np.array(row)[perm], np.array(y)[perm], np.array(z)[perm])


def check_sort_invariants(tf, o):
    n = tf.n
    so = o["sorted_orig"]
    assert np.array_equal(np.sort(so), np.arange(n))          # permutation
    rid, cell = o["sorted_rid"], o["sorted_cell"]
    assert np.array_equal(rid, o["rid"][so])
    assert np.array_equal(o["sorted_y"], o["yu"][so]) and np.array_equal(o["sorted_z"], o["zu"][so])
    key = rid.astype(np.int64) * (1 << 40) + cell.astype(np.int64) * (1 << 20)
    d = np.diff(key)
    assert np.all(d >= 0)                                     # (row, cell) order
    same = d == 0
    assert np.all(np.diff(so)[same] > 0)                      # stable: input order inside a cell
    # per-row counts and row starts
    cnt = np.bincount(rid, minlength=36 * 152)
    assert np.array_equal(cnt, o["row_count"])
    assert np.array_equal(np.concatenate([[0], np.cumsum(cnt)]), o["row_start"])
    # every hit lies inside the rectangle of its cell
    ny, nz, cz, zmin = o["row_ny"][rid], o["row_nz"][rid], o["row_cz"][rid], o["row_zmin"][rid]
    iy, iz = cell % ny, cell // ny
    assert np.all(iz < nz) and np.all(cell >= 0)
    half = np.array([32 * npads(r) for r in range(152)])[rid % 152]
    yrel = o["sorted_y"].astype(np.int64) + half
    lo_ok = (yrel >= iy * 320) | (iy == 0)
    hi_ok = (yrel < (iy + 1) * 320) | (iy == ny - 1)
    assert np.all(lo_ok & hi_ok)
    zrel = o["sorted_z"].astype(np.int64) - zmin
    assert np.all((zrel >= iz * cz) & (zrel < (iz + 1) * cz))
    # the grid covers each row with about 4 hits per cell at most on average
    occ = o["row_count"] > 0
    assert np.all(o["row_ny"][occ] * o["row_nz"][occ] * 4 >= o["row_count"][occ])
    assert np.all(o["row_nz"][occ] * o["row_cz"][occ] >= o["row_zmax"][occ] - o["row_zmin"][occ] + 1)
    # cell starts: hits of cell c are exactly [cell_start[base + c], cell_start[base + c + 1])
    cs = o["cell_start"]
    gcell = o["row_cellbase"][rid] + cell
    idx = np.arange(len(rid))
    assert np.all(cs[gcell] <= idx) and np.all(idx < cs[gcell + 1])
    assert cs[-1] == len(rid)


def brute_neighbours(o):
    y = o["sorted_y"].astype(np.int64)
    z = o["sorted_z"].astype(np.int64)
    rid = o["sorted_rid"]
    n = len(rid)
    up = np.full(n, -1)
    dn = np.full(n, -1)
    for h in range(n):
        r = rid[h] % 152
        if r < 1 or r > 150:
            continue
        U = np.where((rid == rid[h] + 1) & (np.abs(y - y[h]) <= 240) & (np.abs(z - z[h]) <= 248))[0]
        D = np.where((rid == rid[h] - 1) & (np.abs(y - y[h]) <= 240) & (np.abs(z - z[h]) <= 248))[0]
        if len(U) == 0 or len(D) == 0:
            continue
        ey = 2 * y[h] - y[U][:, None] - y[D][None, :]
        ez = 2 * z[h] - z[U][:, None] - z[D][None, :]
        M = 2077 * ey * ey + 1536 * ez * ez
        ok = M <= 16 * 1536 * 2077
        if not ok.any():
            continue
        cand = [(M[i, j], U[i], D[j]) for i, j in zip(*np.nonzero(ok))]
        m, u, d = min(cand)
        up[h], dn[h] = u, d
    return up, dn


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_neighbours_equal_brute_force_dense(seed):
    tf = dense_tf(seed)
    o = oracle.run(tf)
    check_sort_invariants(tf, o)
    up, dn = brute_neighbours(o)
    assert np.array_equal(o["up_raw"], up)
    assert np.array_equal(o["dn_raw"], dn)
    assert (o["up_raw"] >= 0).sum() > 50


def test_neighbours_equal_brute_force_single_sector_slice():
    """A slice of the single-sector workload (rows 0-3 and 148-151 included
    to pin the edge rule: rows 0 and 151 never get links)."""
    tf = synth.single_sector()
    keep = np.isin(tf.row, [0, 1, 2, 3, 70, 71, 72, 148, 149, 150, 151])
    sub = float_tf(tf.sector[keep], tf.row[keep], tf.y[keep], tf.z[keep])
    o = oracle.run(sub)
    check_sort_invariants(sub, o)
    up, dn = brute_neighbours(o)
    assert np.array_equal(o["up_raw"], up) and np.array_equal(o["dn_raw"], dn)
    r = o["sorted_rid"] % 152
    assert np.all(o["up_raw"][(r == 0) | (r == 151)] == -1)


def test_sort_invariants_full_tpc_sample():
    tf = synth.full_tpc_1ms(n_coll=2)
    o = oracle.run(tf, fields=["yu", "zu", "rid", "sorted_orig", "sorted_rid", "sorted_y", "sorted_z",
                               "sorted_cell", "row_count", "row_start", "row_ny", "row_nz", "row_cz",
                               "row_zmin", "row_zmax", "row_cellbase", "cell_start"])
    check_sort_invariants(tf, o)


def check_cleaner_and_starts(o):
    up_r, dn_r, up, dn = o["up_raw"], o["dn_raw"], o["up"], o["dn"]
    n = len(up)
    # cleaned links are a subset of the raw links
    assert np.all((up == -1) | (up == up_r)) and np.all((dn == -1) | (dn == dn_r))
    # reciprocity: up[h] = u  <=>  dn[u] = h
    h = np.nonzero(up >= 0)[0]
    assert np.all(dn[up[h]] == h)
    h = np.nonzero(dn >= 0)[0]
    assert np.all(up[dn[h]] == h)
    # completeness: every reciprocal raw pair survives
    h = np.nonzero(up_r >= 0)[0]
    recip = dn_r[up_r[h]] == h
    assert np.all(up[h[recip]] == up_r[h[recip]])
    # chains are disjoint simple paths (each hit has <= 1 predecessor by construction); starts are
    # exactly the heads of chains with >= 3 hits, in increasing sorted order
    heads = [i for i in range(n) if dn[i] < 0 and up[i] >= 0 and up[up[i]] >= 0]
    assert list(o["starts"]) == heads
    for s in o["starts"]:
        k, seen = s, 0
        while k >= 0:
            seen += 1
            k = up[k]
            assert seen <= 152


@pytest.mark.parametrize("seed", [1, 4])
def test_cleaner_and_start_invariants(seed):
    check_cleaner_and_starts(oracle.run(dense_tf(seed)))


def test_cleaner_and_start_invariants_single_sector():
    check_cleaner_and_starts(oracle.run(synth.single_sector()))


def test_handworked_golden():
    g = json.load(open(os.path.join(GOLDEN, "nf_handworked.json")))
    tf = fixed_tf(g["sector"], g["row"], g["pad64"], g["time64"])
    o = oracle.run(tf)
    so = o["sorted_orig"]

    def to_orig(a):
        return [int(so[v]) if v >= 0 else -1 for v in a]

    inv = np.argsort(so)  # orig -> sorted
    for name in ("up_raw", "dn_raw", "up", "dn"):
        got = to_orig(o[name][inv])
        assert got == g["expected_orig"][name], name
    assert [int(so[s]) for s in o["starts"]] == g["expected_orig"]["starts"]


def test_fixed_point_ingest_matches_format_definition():
    """y_u = pad64 - 32 nPads(row) and zeta_u = time64 for fixed records."""
    rng = np.random.default_rng(7)
    n = 500
    row = rng.integers(0, 152, n)
    sec = rng.integers(0, 36, n)
    pad = np.array([rng.integers(0, 64 * npads(r)) for r in row])
    t64 = rng.integers(0, 1 << 22, n)
    o = oracle.run(fixed_tf(sec, row, pad, t64), fields=["yu", "zu", "rid"])
    assert np.array_equal(o["yu"], pad - np.array([32 * npads(r) for r in row]))
    assert np.array_equal(o["zu"], t64)
    assert np.array_equal(o["rid"], sec * 152 + row)


def test_invalid_input_rejected():
    tf = float_tf([36], [3], [0.0], [1.0])
    with pytest.raises(oracle.OracleError):
        oracle.run(tf)
    tf = float_tf([3], [152], [0.0], [1.0])
    with pytest.raises(oracle.OracleError):
        oracle.run(tf)
    tf = float_tf([3], [10], [np.nan], [1.0])
    with pytest.raises(oracle.OracleError):
        oracle.run(tf)


def test_empty_input():
    tf = float_tf([], [], [], [])
    o = oracle.run(tf)
    assert len(o["sorted_orig"]) == 0 and len(o["trk_x"]) == 0 and o["trk_off"].tolist() == [0]


def test_grid_dimensions_handworked_golden():
    """Grid dimensions (ny, nz, cz, zeta_min) and cell indices of listed hits
    against values worked out by hand (tests/golden/grid_handworked.json):
    a wrong pad count, a wrong cell width, nz off by one or cz rounded the
    wrong way changes at least one of them."""
    g = json.load(open(os.path.join(GOLDEN, "grid_handworked.json")))
    sec, row, pad, tim, listed = [], [], [], [], []
    for r in g["rows"]:
        base = len(sec)
        listed.append(list(range(base, base + len(r["pad64"]))))
        sec += [r["sector"]] * len(r["pad64"])
        row += [r["row"]] * len(r["pad64"])
        pad += r["pad64"]
        tim += r["time64"]
        f = r["fillers"]
        if f:
            k = np.arange(f["count"])
            a, b = (int(v) for v in f["pad64"].replace("(", "").replace(")", "").replace(" k", "").split(" mod "))
            c0, c1 = (int(v) for v in f["time64"].replace(" k", "").split(" + "))
            sec += [r["sector"]] * f["count"]
            row += [r["row"]] * f["count"]
            pad += ((a * k) % b).tolist()
            tim += (c0 + c1 * k).tolist()
    tf = fixed_tf(sec, row, pad, tim)
    o = oracle.run(tf)
    inv = np.argsort(o["sorted_orig"])
    for r, idx in zip(g["rows"], listed):
        rid = r["sector"] * 152 + r["row"]
        e = r["expected"]
        got = (int(o["row_count"][rid]), int(o["row_ny"][rid]), int(o["row_nz"][rid]), int(o["row_cz"][rid]),
               int(o["row_zmin"][rid]))
        assert got == (e["count"], e["ny"], e["nz"], e["cz"], e["zmin"]), (r["name"], got)
        assert [int(o["sorted_cell"][inv[i]]) for i in idx] == e["cells"], r["name"]
    for r in g["empty_rows"]:
        rid = r["sector"] * 152 + r["row"]
        e = r["expected"]
        got = (int(o["row_count"][rid]), int(o["row_ny"][rid]), int(o["row_nz"][rid]))
        assert got == (e["count"], e["ny"], e["nz"]), (r, got)
