"""Parity at the benchmark's full size: one 128-orbit Time Frame at 50 kHz
Pb-Pb (~250 M clusters), tracked by the CUDA path in the default launch
configuration, against the oracle run on a sample of it - sectors 0 and 1
(adjacent on the A side, ~13 M clusters), which the oracle handles alone in
about a minute.

* Sector 0's hits come first in the sorted order, so its sorted indices,
  grid, cell starts, links, start hits and tracklet ids are the same numbers
  on both sides and are compared bit-exactly; its sector tracks must match in
  >= 99.9 % of the cluster sets.
* Through the merger and the final refit: the oracle, restricted to sectors
  0 and 1, merges across their common edge only.  In the full TF a sector
  track can also merge across the two outer edges (sector 0 with 17, sector 1
  with 2), but only if one of its ends lies in the 5 cm border band facing
  that edge.  The oracle's final tracks none of whose sector tracks has an
  end in those two bands are therefore exactly the tracks the full TF must
  contain; they are compared with the GPU's final tracks that lie in sectors
  0 and 1 by the track criteria (identical cluster sets, parameters within
  tolerance, FP64 fallback tracks included).
"""
import numpy as np
import pytest

import oracle
from parity import brief, compare_tracks
from paper_2106_03636_gb300 import o2tpc, synth

pytestmark = pytest.mark.gpu

NROW = 152
ZUNIT = 0.003125 * 2.58
TAN10 = float(np.tan(np.radians(10.0)))
EDGE = 5.0


def sector_subset(res: dict, sector_of_cluster: np.ndarray, sectors) -> dict:
    """The GPU tracks whose clusters all lie in `sectors`."""
    off = res["offsets"].astype(np.int64)
    cl = res["cluster_idx"].astype(np.int64)
    ins = np.isin(sector_of_cluster[cl], list(sectors)).astype(np.int64)
    lens = np.diff(off)
    keep = np.nonzero(np.add.reduceat(ins, off[:-1]) == lens)[0] if len(lens) else np.zeros(0, np.int64)
    new_off = np.concatenate([[0], np.cumsum(lens[keep])]).astype(np.uint64)
    new_cl = np.concatenate([cl[off[t]:off[t + 1]] for t in keep]) if len(keep) else np.zeros(0, np.int64)
    sub = {k: res[k][keep] for k in ("par", "cov", "x", "zeta_ref", "sector", "flags")}
    sub.update(offsets=new_off, cluster_idx=new_cl.astype(np.uint32))
    return sub


def interior_tracks(o: dict, outward: dict) -> dict:
    """Oracle final tracks none of whose sector tracks has an end in a border
    band facing an edge of the sample (outward: sector -> direction, +1 for
    the y > 0 edge)."""
    sts, sin, sout = o["st_sector"], o["st_in"], o["st_out"]

    def facing(i):
        d = outward.get(int(sts[i]))
        if d is None:
            return False
        for st in (sin[i], sout[i]):
            x, y = st[0], st[1]
            if abs(y) >= x * TAN10 - EDGE and (1 if y > 0 else -1) == d:
                return True
        return False

    keep = []
    for t, head in enumerate(o["trk_head"]):
        c, ok = int(head), True
        while c >= 0:
            if facing(c):
                ok = False
                break
            c = int(o["st_next"][c])
        if ok:
            keep.append(t)
    off = o["trk_off"]
    sub = {k: o[k][keep] for k in ("trk_par", "trk_cov", "trk_x", "trk_zref", "trk_sector", "trk_flags", "trk_chi2",
                                   "trk_ndf")}
    sub["trk_off"] = np.concatenate([[0], np.cumsum(np.diff(off)[keep])]).astype(np.int64)
    sub["trk_cl"] = np.concatenate([o["trk_cl"][off[t]:off[t + 1]] for t in keep]).astype(np.int32)
    return sub


def test_full_tf_sectors_0_1_sampled():
    tf = synth.full_tf()
    sector_of_cluster = tf.packed[:, 9].copy()
    with o2tpc.Tracker(flags=o2tpc.O2TPC_FLAG_KEEP_STAGES) as trk:
        tk = trk.submit(tf)
        res = trk.poll(tk, keep=True)
        assert res["status"] == 0 and res["n_tracks"] > 100000
        g = trk.stage(tk, "row_grid")
        n0 = int(g[NROW - 1, 0] + g[NROW - 1, 1])
        c0 = int(g[NROW, 2])
        gpu = {
            "row_grid": g[:NROW].copy(),
            "sorted_orig": trk.stage(tk, "sorted_orig")[:n0].copy(),
            "sorted_yz": trk.stage(tk, "sorted_yz")[:n0].copy(),
            "cell_start": trk.stage(tk, "cell_start")[: c0 + 1].copy(),
        }
        for nm in ("up_raw", "dn_raw", "up", "dn"):
            gpu[nm] = trk.stage(tk, nm)[:n0].copy()
        starts = trk.stage(tk, "starts")
        gpu["starts"] = starts[starts < n0].copy()
        gpu["tl_nhits"] = trk.stage(tk, "tl_nhits")[: len(gpu["starts"])].copy()
        so, sh = trk.stage(tk, "st_off"), trk.stage(tk, "st_hits")
        gpu_st = {tuple(sh[so[i]:so[i + 1]]) for i in range(len(so) - 1) if so[i + 1] > so[i] and sh[so[i]] < n0}
        n_fallback = int(res["stats"]["n_fp64_fallback"])
        trk.release(tk, res)
    gsub = sector_subset(res, sector_of_cluster, (0, 1))
    del res

    o = oracle.run(tf, sector_mask=0b11, fields=[
        "sorted_orig", "sorted_y", "sorted_z", "row_start", "row_count", "row_cellbase", "row_ny", "row_nz",
        "row_cz", "row_zmin", "cell_start", "up_raw", "dn_raw", "up", "dn", "starts", "tl_nhits", "st_off",
        "st_hits", "st_sector", "st_in", "st_out", "st_next", "trk_off", "trk_cl", "trk_x", "trk_par", "trk_cov",
        "trk_sector", "trk_flags", "trk_zref", "trk_head", "trk_chi2", "trk_ndf"])
    # sector 0, integer stages bit for bit
    assert np.array_equal(gpu["sorted_orig"], o["sorted_orig"][:n0]), "sort order"
    assert np.array_equal(gpu["sorted_yz"][:, 0], o["sorted_y"][:n0]), "sorted y"
    assert np.array_equal(gpu["sorted_yz"][:, 1], o["sorted_z"][:n0]), "sorted zeta"
    rg = gpu["row_grid"]
    assert np.array_equal(rg[:, 0], o["row_start"][:NROW]) and np.array_equal(rg[:, 1], o["row_count"][:NROW])
    assert np.array_equal(rg[:, 2], o["row_cellbase"][:NROW])
    assert np.array_equal(rg[:, 3], o["row_ny"][:NROW]) and np.array_equal(rg[:, 4], o["row_nz"][:NROW])
    assert np.array_equal(rg[:, 5], o["row_cz"][:NROW]) and np.array_equal(rg[:, 6], o["row_zmin"][:NROW])
    assert np.array_equal(gpu["cell_start"], o["cell_start"][: c0 + 1]), "cell starts"
    for nm in ("up_raw", "dn_raw", "up", "dn"):
        assert np.array_equal(gpu[nm], o[nm][:n0]), nm
    ostarts = o["starts"][o["starts"] < n0]
    assert np.array_equal(gpu["starts"], ostarts), "start hits"
    same = np.mean(gpu["tl_nhits"] == o["tl_nhits"][: len(ostarts)])
    assert same >= 0.999, same
    oo = o["st_off"]
    ref = [tuple(o["st_hits"][oo[i]:oo[i + 1]]) for i in range(len(oo) - 1) if o["st_sector"][i] == 0]
    st_frac = np.mean([x in gpu_st for x in ref])
    assert st_frac >= 0.999, st_frac

    # sectors 0 and 1 through the merger and the final refit
    osub = interior_tracks(o, {0: -1, 1: +1})
    rep = compare_tracks(gsub, osub, ZUNIT)
    merged = int(np.sum((osub["trk_flags"] & 2) != 0))
    fb = int(np.sum((gsub["flags"] & 1) != 0))
    print(dict(clusters_sector0=n0, sector_tracks_0=len(ref), st_match=st_frac, tl_nhits_same=same,
               oracle_interior_tracks=len(osub["trk_x"]), oracle_tracks=len(o["trk_x"]), merged_interior=merged,
               gpu_tracks_in_01=len(gsub["x"]), fp64_fallback_tf=n_fallback, fp64_fallback_in_01=fb, **brief(rep)))
    assert merged > 100  # the sample holds tracks joined across the 0 / 1 edge
    assert len(osub["trk_x"]) > 0.25 * len(o["trk_x"])  # tracks away from the two outer border bands
