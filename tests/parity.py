"""Parity comparison of the CUDA path with the oracle (used by the -m gpu tests).

Criteria (FP32 path against the FP64 oracle):
* grid, sort order, cell starts, neighbour links, cleaned links and start
  hits: bit-exact;
* >= 99.9 % of oracle tracks reproduced with identical cluster sets;
* on those tracks y and zeta within 1e-3 cm, sin(phi), tan(lambda) and q/pT
  within 1e-4 relative, |d| <= 1e-4 * max(|v_oracle|, 1e-2).  For q/pT the
  relative scale is the value itself only where the fit determines it
  (sigma(q/pT) <= |q/pT|); on short stubs whose charge the fit leaves open
  (sigma > |q/pT|) the scale is sigma(q/pT), i.e. 1e-4 of the parameter's
  own uncertainty.
"""
from __future__ import annotations

import numpy as np

TRACK_MATCH = 0.999
TOL_POS = 1e-3
TOL_REL = 1e-4
REL_FLOOR = 1e-2


def compare_stages(trk, ticket, o) -> None:
    """Bit-exact comparison of the integer stages (A2-A7)."""
    so = trk.stage(ticket, "sorted_orig")
    assert np.array_equal(so, o["sorted_orig"]), "sort order"
    yz = trk.stage(ticket, "sorted_yz")
    assert np.array_equal(yz[:, 0], o["sorted_y"]) and np.array_equal(yz[:, 1], o["sorted_z"]), "sorted y/zeta"
    g = trk.stage(ticket, "row_grid")
    assert np.array_equal(g[:, 0], o["row_start"][:-1]), "row starts"
    assert np.array_equal(g[:, 1], o["row_count"]), "row counts"
    assert np.array_equal(g[:, 2], o["row_cellbase"][:-1]), "cell bases"
    assert np.array_equal(g[:, 3], o["row_ny"]) and np.array_equal(g[:, 4], o["row_nz"]), "grid dims"
    occ = o["row_count"] > 0
    assert np.array_equal(g[occ, 5], o["row_cz"][occ]) and np.array_equal(g[occ, 6], o["row_zmin"][occ]), "cz/zmin"
    cs = trk.stage(ticket, "cell_start")
    assert np.array_equal(cs, o["cell_start"]), "cell starts"
    for nm in ("up_raw", "dn_raw", "up", "dn"):
        assert np.array_equal(trk.stage(ticket, nm), o[nm]), nm
    assert np.array_equal(trk.stage(ticket, "starts"), o["starts"]), "start hits"


def track_sets(offsets, clusters):
    return [tuple(sorted(clusters[offsets[i]:offsets[i + 1]].tolist())) for i in range(len(offsets) - 1)]


def compare_tracks(res: dict, o: dict, zunit: float, check: bool = True) -> dict:
    """Track-level parity; returns a report dict (asserts the criteria unless
    ``check`` is False, for samples that are pooled before judging)."""
    go = track_sets(res["offsets"].astype(np.int64), res["cluster_idx"].astype(np.int64))
    oo = track_sets(o["trk_off"], o["trk_cl"])
    gidx = {s: i for i, s in enumerate(go)}
    matched = [(i, gidx[s]) for i, s in enumerate(oo) if s in gidx]
    frac = len(matched) / max(1, len(oo))
    err = np.zeros((len(matched), 5))
    bad = 0
    undetermined = 0
    for k, (i, j) in enumerate(matched):
        po = o["trk_par"][i].copy()
        pg = res["par"][j].astype(np.float64)
        # the same innermost cluster gives the same zeta origin and frame
        assert int(res["zeta_ref"][j]) == int(o["trk_zref"][i])
        assert int(res["sector"][j]) == int(o["trk_sector"][i])
        d = np.abs(pg - po)
        err[k, :2] = d[:2]
        scale = np.maximum(np.abs(po[2:]), REL_FLOOR)
        sq = float(np.sqrt(max(o["trk_cov"][i][14], 0.0)))
        if sq > abs(po[4]):
            scale[2] = max(sq, REL_FLOOR)
            undetermined += 1
        err[k, 2:] = d[2:] / scale
        same_x = abs(float(res["x"][j]) - o["trk_x"][i]) < 1e-4
        if not same_x or np.any(err[k, :2] > TOL_POS) or np.any(err[k, 2:] > TOL_REL):
            bad += 1
    rep = dict(n_oracle=len(oo), n_gpu=len(go), matched=len(matched), frac=frac, bad_params=bad,
               charge_undetermined=undetermined,
               max_err=err.max(axis=0).tolist() if len(err) else [0] * 5,
               p999_err=np.quantile(err, 0.999, axis=0).tolist() if len(err) else [0] * 5)
    if check:
        assert_criteria(rep)
    return rep


def assert_criteria(rep: dict) -> None:
    """>= 99.9 % of oracle tracks reproduced with identical cluster sets, and
    >= 99.9 % of them with every parameter within tolerance."""
    assert rep["frac"] >= TRACK_MATCH, rep
    assert rep["bad_params"] <= (1 - TRACK_MATCH) * max(1, rep["n_oracle"]), rep


def pool(reps: list) -> dict:
    out = dict(n_oracle=sum(r["n_oracle"] for r in reps), matched=sum(r["matched"] for r in reps),
               bad_params=sum(r["bad_params"] for r in reps),
               max_err=np.max([r["max_err"] for r in reps], axis=0).tolist())
    out["frac"] = out["matched"] / max(1, out["n_oracle"])
    return out
