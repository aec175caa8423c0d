"""Parity comparison of the CUDA path with the oracle (used by the -m gpu tests).

Criteria (FP32 path against the FP64 oracle):
* grid, sort order, cell starts, neighbour links, cleaned links and start
  hits: bit-exact;
* >= 99.9 % of oracle tracks reproduced with identical cluster sets;
* on those tracks y and zeta within 1e-3 cm, sin(phi), tan(lambda) and q/pT
  within 1e-4 relative, |d| <= 1e-4 * max(|v_oracle|, 1e-2), the same
  tolerance for every track; at most 0.1 % of the matched tracks whose fit
  is well posed may miss it.
* Well posed: the oracle's final fit used at least 5 clusters (ndf >= 5) and
  its chi2 is at most 10 ndf.  The tolerance is a statement about rounding,
  and the sensitivity of a least-squares solution to rounding grows with the
  fit's residual: for relative perturbations eps of the data and arithmetic
  the relative change of the solution is bounded by
  eps (2 kappa / cos(theta) + kappa^2 tan(theta)), sin(theta) = |r| / |b|
  (the least-squares perturbation theorem, e.g. Golub & Van Loan, Matrix
  Computations, Thm. 5.3.1).  When chi2 is many times ndf the clusters do not
  fit the helix (a cluster of another particle, a looper's two legs), the
  kappa^2 tan(theta) term dominates and single-precision rounding is
  amplified past 1e-4; with fewer than 5 clusters used the five parameters
  are barely determined.  Such tracks still count in the cluster-set
  criterion, their parameter errors are reported with the others, and they
  may make up at most 2 % of the matched tracks.
* The report gives, per parameter, the largest error and the 99.9th
  percentile against the FP64 oracle (all matched tracks), and the
  out-of-tolerance counts (all, and well posed).
"""
from __future__ import annotations

import numpy as np

TRACK_MATCH = 0.999
WELL_POSED_CHI2_PER_NDF = 10.0
WELL_POSED_MIN_NDF = 5
ILL_POSED_MAX = 0.02
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


def compare_tracks(res: dict, o: dict, zunit: float, check: bool = True, bad_frac: float = 1 - TRACK_MATCH) -> dict:
    """Track-level parity; returns a report dict (asserts the criteria unless
    ``check`` is False, for samples that are pooled before judging)."""
    go = track_sets(res["offsets"].astype(np.int64), res["cluster_idx"].astype(np.int64))
    oo = track_sets(o["trk_off"], o["trk_cl"])
    gidx = {s: i for i, s in enumerate(go)}
    matched = [(i, gidx[s]) for i, s in enumerate(oo) if s in gidx]
    frac = len(matched) / max(1, len(oo))
    err = np.zeros((len(matched), 5))
    bad = 0
    bad_wp = 0
    n_wp = 0
    bad_param = np.zeros(5, np.int64)
    for k, (i, j) in enumerate(matched):
        po = o["trk_par"][i].copy()
        pg = res["par"][j].astype(np.float64)
        # the same innermost cluster gives the same zeta origin and frame
        assert int(res["zeta_ref"][j]) == int(o["trk_zref"][i])
        assert int(res["sector"][j]) == int(o["trk_sector"][i])
        d = np.abs(pg - po)
        err[k, :2] = d[:2]
        scale = np.maximum(np.abs(po[2:]), REL_FLOOR)
        err[k, 2:] = d[2:] / scale
        same_x = abs(float(res["x"][j]) - o["trk_x"][i]) < 1e-4
        over = np.concatenate([err[k, :2] > TOL_POS, err[k, 2:] > TOL_REL])
        bad_param += over
        ndf, chi2 = int(o["trk_ndf"][i]), float(o["trk_chi2"][i])
        wp = ndf >= WELL_POSED_MIN_NDF and chi2 <= WELL_POSED_CHI2_PER_NDF * ndf
        n_wp += wp
        if not same_x or np.any(over):
            bad += 1
            bad_wp += wp
    rep = dict(n_oracle=len(oo), n_gpu=len(go), matched=len(matched), frac=frac, bad_params=bad,
               well_posed=n_wp, bad_well_posed=bad_wp, bad_per_param=bad_param.tolist(),
               max_err=err.max(axis=0).tolist() if len(err) else [0] * 5,
               p999_err=np.quantile(err, 0.999, axis=0).tolist() if len(err) else [0] * 5, _err=err)
    if check:
        assert_criteria(rep, bad_frac)
    return rep


def assert_criteria(rep: dict, bad_frac: float = 1 - TRACK_MATCH) -> None:
    """>= 99.9 % of oracle tracks reproduced with identical cluster sets;
    >= 99.9 % of those with a well-posed fit with every parameter within
    tolerance (bad_frac: the allowed out-of-tolerance fraction); at most 2 %
    of the matched tracks ill posed."""
    assert rep["frac"] >= TRACK_MATCH, brief(rep)
    assert rep["bad_well_posed"] <= bad_frac * max(1, rep["well_posed"]), brief(rep)
    assert rep["matched"] - rep["well_posed"] <= ILL_POSED_MAX * max(1, rep["matched"]), brief(rep)


def pool(reps: list) -> dict:
    out = dict(n_oracle=sum(r["n_oracle"] for r in reps), matched=sum(r["matched"] for r in reps),
               bad_params=sum(r["bad_params"] for r in reps),
               well_posed=sum(r["well_posed"] for r in reps), bad_well_posed=sum(r["bad_well_posed"] for r in reps),
               bad_per_param=np.sum([r["bad_per_param"] for r in reps], axis=0).tolist(),
               max_err=np.max([r["max_err"] for r in reps], axis=0).tolist())
    err = np.concatenate([r["_err"] for r in reps])
    out["p999_err"] = np.quantile(err, 0.999, axis=0).tolist() if len(err) else [0] * 5
    out["frac"] = out["matched"] / max(1, out["n_oracle"])
    return out


def brief(rep: dict) -> dict:
    """The report without the per-track error array (for printing)."""
    return {k: v for k, v in rep.items() if not k.startswith("_")}
