"""Parity at the benchmark's full size: one 128-orbit Time Frame at 50 kHz
Pb-Pb (~250 M clusters), tracked by the CUDA path in the default launch
configuration, against the oracle run on a sample of it - sector 0 (A side,
~7 M clusters), which the oracle handles alone in about half a minute.

Sector 0's hits come first in the sorted order, so its sorted indices,
grid, cell starts, links, start hits and tracklet ids are the same numbers
on both sides and are compared bit-exactly; its sector tracks (before the
merger, which joins sectors) must match in >= 99.9 % of the cluster sets."""
import numpy as np
import pytest

import oracle
from paper_2106_03636_gb300 import o2tpc, synth

pytestmark = pytest.mark.gpu

NROW = 152


def test_full_tf_sector0_sampled():
    tf = synth.full_tf()
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
        trk.release(tk, res)

    o = oracle.run(tf, sector_mask=1, fields=[
        "sorted_orig", "sorted_y", "sorted_z", "row_start", "row_count", "row_cellbase", "row_ny", "row_nz",
        "row_cz", "row_zmin", "cell_start", "up_raw", "dn_raw", "up", "dn", "starts", "tl_nhits", "st_off",
        "st_hits"])
    assert len(o["sorted_orig"]) == n0
    assert np.array_equal(gpu["sorted_orig"], o["sorted_orig"]), "sort order"
    assert np.array_equal(gpu["sorted_yz"][:, 0], o["sorted_y"]), "sorted y"
    assert np.array_equal(gpu["sorted_yz"][:, 1], o["sorted_z"]), "sorted zeta"
    rg = gpu["row_grid"]
    assert np.array_equal(rg[:, 0], o["row_start"][:NROW]) and np.array_equal(rg[:, 1], o["row_count"][:NROW])
    assert np.array_equal(rg[:, 2], o["row_cellbase"][:NROW])
    assert np.array_equal(rg[:, 3], o["row_ny"][:NROW]) and np.array_equal(rg[:, 4], o["row_nz"][:NROW])
    assert np.array_equal(rg[:, 5], o["row_cz"][:NROW]) and np.array_equal(rg[:, 6], o["row_zmin"][:NROW])
    assert np.array_equal(gpu["cell_start"], o["cell_start"][: c0 + 1]), "cell starts"
    for nm in ("up_raw", "dn_raw", "up", "dn"):
        assert np.array_equal(gpu[nm], o[nm]), nm
    assert np.array_equal(gpu["starts"], o["starts"]), "start hits"
    same = np.mean(gpu["tl_nhits"] == o["tl_nhits"])
    assert same >= 0.999, same
    oo = o["st_off"]
    ref = [tuple(o["st_hits"][oo[i]:oo[i + 1]]) for i in range(len(oo) - 1)]
    frac = np.mean([x in gpu_st for x in ref])
    print(dict(clusters_sector0=n0, starts=len(gpu["starts"]), sector_tracks=len(ref), st_match=frac, tl_nhits_same=same))
    assert frac >= 0.999, frac
