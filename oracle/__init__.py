"""FP64 single-threaded CPU oracle of the TPC Time-Frame tracker.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The oracle is a
plain C program (``o2tpc_oracle.c``) that shares no code with the CUDA path;
this module builds it with gcc and exposes it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "o2tpc_oracle.c")
CTF_SRC = os.path.join(HERE, "o2tpc_ctf.c")
CLU_SRC = os.path.join(HERE, "o2tpc_clu.c")
LIBDIR = os.path.join(HERE, "_lib")
SO = os.path.join(LIBDIR, "liboracle.so")


def build(force: bool = False) -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    deps = [SRC, CTF_SRC, CLU_SRC, os.path.join(HERE, "o2tpc_oracle.h")]
    if force or not os.path.exists(SO) or any(os.path.getmtime(d) > os.path.getmtime(SO) for d in deps):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", SO + ".tmp", SRC, CTF_SRC, CLU_SRC, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stdout + r.stderr)
        os.replace(SO + ".tmp", SO)
    return SO


class _Input(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("format", ctypes.c_int32),
        ("sector", ctypes.c_void_p),
        ("row", ctypes.c_void_p),
        ("y", ctypes.c_void_p),
        ("z", ctypes.c_void_p),
        ("time", ctypes.c_void_p),
        ("packed", ctypes.c_void_p),
        ("bz", ctypes.c_double),
        ("vdrift", ctypes.c_double),
        ("sector_mask", ctypes.c_uint64),
        ("reverse_tracklet_order", ctypes.c_int32),
        ("coll_time", ctypes.c_void_p),
        ("n_coll", ctypes.c_int64),
        ("compress", ctypes.c_int32),
        ("row_step2", ctypes.c_int32),
        ("angular_errors", ctypes.c_int32),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_run.restype = ctypes.c_void_p
        lib.oracle_run.argtypes = [ctypes.POINTER(_Input), ctypes.POINTER(ctypes.c_int32)]
        lib.oracle_free.restype = None
        lib.oracle_free.argtypes = [ctypes.c_void_p]
        lib.oracle_get.restype = ctypes.c_int64
        lib.oracle_get.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p),
                                   ctypes.POINTER(ctypes.c_int32)]
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_propagate.restype = ctypes.c_int32
        lib.oracle_propagate.argtypes = [dp, dp, dp, ctypes.c_double, ctypes.c_double]
        lib.oracle_update.restype = ctypes.c_int32
        lib.oracle_update.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, dp]
        lib.oracle_rotate.restype = ctypes.c_int32
        lib.oracle_rotate.argtypes = [dp, dp, dp, ctypes.c_double]
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_ctf_encode.restype = ctypes.c_int64
        lib.oracle_ctf_encode.argtypes = [ctypes.c_int64, i32p, i32p, i32p, i32p, ctypes.c_int64, i64p, i32p, dp,
                                          i32p, ctypes.c_int64, ctypes.POINTER(u8p)]
        lib.oracle_ctf_decode.restype = ctypes.c_int64
        lib.oracle_ctf_decode.argtypes = [u8p, ctypes.c_int64] + [ctypes.POINTER(i32p)] * 4 + [
            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(i64p)]
        lib.oracle_ctf_normalize.restype = None
        lib.oracle_ctf_normalize.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint16)]
        lib.oracle_rans_encode.restype = ctypes.c_int64
        lib.oracle_rans_encode.argtypes = [u8p, ctypes.c_int64, ctypes.POINTER(u8p)]
        lib.oracle_rans_decode.restype = ctypes.c_int64
        lib.oracle_rans_decode.argtypes = [u8p, ctypes.c_int64, ctypes.POINTER(u8p)]
        lib.oracle_buffer_free.restype = None
        lib.oracle_buffer_free.argtypes = [ctypes.c_void_p]
        lib.oracle_clusterize.restype = ctypes.c_int64
        lib.oracle_clusterize.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 5 + [ctypes.POINTER(u8p)]
        lib.oracle_dca_arc.restype = ctypes.c_double
        lib.oracle_dca_arc.argtypes = [ctypes.c_double] * 4
        lib.oracle_fit_points.restype = ctypes.c_int32
        lib.oracle_fit_points.argtypes = [ctypes.c_int32, dp, dp, dp, ctypes.c_double, dp, dp]
        _lib = lib
    return _lib


_DT = {0: np.int32, 1: np.int64, 2: np.float64, 3: np.uint8}

FIELDS = [
    "yu", "zu", "rid", "sorted_orig", "sorted_rid", "sorted_y", "sorted_z", "sorted_cell",
    "row_count", "row_zmin", "row_zmax", "row_ny", "row_nz", "row_cz", "row_start", "row_cellbase",
    "cell_start", "up_raw", "dn_raw", "up", "dn", "starts", "tl_nhits", "tl_kept", "tl_zref", "tl_off",
    "tl_hits", "tl_state", "st_sector", "st_tracklet", "st_zref", "st_off", "st_hits", "st_in", "st_out",
    "st_next", "st_prev", "pair_ab", "pair_chi2", "trk_off", "trk_cl", "trk_x", "trk_alpha", "trk_par",
    "trk_cov", "trk_chi2", "trk_ndf", "trk_sector", "trk_flags", "trk_zref", "trk_head", "trk_nseg",
    "trk_t0", "trk_t0err", "trk_t0lo", "trk_t0hi", "trk_mate", "trk_coll", "mpair_ab", "mpair_chi2", "ctf",
]


class OracleError(RuntimeError):
    pass


def _vp(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def run(tf, sector_mask: int = 0, reverse_tracklet_order: bool = False, fields=None, coll_time=None,
        compress: bool = False, row_step2: bool = False, angular_errors: bool = False) -> dict:
    """Runs the oracle on a ``synth.TimeFrame``-like object (attributes n,
    fmt, sector, row, y, z, packed, bz, vdrift, and optionally coll_time,
    the TF's interaction times in us).  ``coll_time`` overrides the TF's;
    ``compress`` also builds the compressed TF (field ``ctf``, bytes);
    ``row_step2`` lets the NeighboursFinder link across one missing pad row;
    ``angular_errors`` makes the cluster errors grow with the track angles.
    Returns a dict of numpy arrays (copies) named as in ``FIELDS``."""
    lib = _load()
    inp = _Input()
    inp.n = tf.n
    inp.format = tf.fmt
    keep = []
    if tf.fmt == 0:
        names = ("sector", "row", "y", "z") if getattr(tf, "z", None) is not None else ("sector", "row", "y", "time")
        for nm in names:
            a = np.ascontiguousarray(getattr(tf, nm))
            keep.append(a)
            setattr(inp, nm, _vp(a))
    else:
        a = np.ascontiguousarray(tf.packed)
        keep.append(a)
        inp.packed = _vp(a)
    inp.bz = tf.bz
    inp.vdrift = tf.vdrift
    inp.sector_mask = sector_mask
    inp.reverse_tracklet_order = int(reverse_tracklet_order)
    inp.compress = int(compress)
    inp.row_step2 = int(row_step2)
    inp.angular_errors = int(angular_errors)
    ct = coll_time if coll_time is not None else getattr(tf, "coll_time", None)
    if ct is not None and len(ct):
        ct = np.ascontiguousarray(np.asarray(ct, dtype=np.float64))
        keep.append(ct)
        inp.coll_time = _vp(ct)
        inp.n_coll = len(ct)
    st = ctypes.c_int32()
    h = lib.oracle_run(ctypes.byref(inp), ctypes.byref(st))
    if st.value != 0 or not h:
        raise OracleError(f"oracle rejected the input (status {st.value})")
    out = {}
    try:
        for nm in (fields or FIELDS):
            p = ctypes.c_void_p()
            t = ctypes.c_int32()
            n = lib.oracle_get(h, nm.encode(), ctypes.byref(p), ctypes.byref(t))
            if n < 0:
                raise KeyError(nm)
            dt = _DT[t.value]
            if n == 0:
                out[nm] = np.zeros(0, dt)
            else:
                buf = (ctypes.c_char * (n * np.dtype(dt).itemsize)).from_address(p.value)
                out[nm] = np.frombuffer(buf, dtype=dt).copy()
    finally:
        lib.oracle_free(h)
    for nm in ("tl_state", "st_in", "st_out"):
        if nm in out:
            out[nm] = out[nm].reshape(-1, 21)
    if "trk_par" in out:
        out["trk_par"] = out["trk_par"].reshape(-1, 5)
    if "trk_cov" in out:
        out["trk_cov"] = out["trk_cov"].reshape(-1, 15)
    for nm in ("pair_ab", "mpair_ab"):
        if nm in out:
            out[nm] = out[nm].reshape(-1, 2)
    return out


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def propagate(x: float, p5, c15, x2: float, bz: float):
    lib = _load()
    xx = np.array([x], np.float64)
    p = np.array(p5, np.float64)
    c = np.array(c15, np.float64)
    rc = lib.oracle_propagate(_dptr(xx), _dptr(p), _dptr(c), x2, bz)
    return rc, xx[0], p, c


def update(p5, c15, ym: float, zm: float):
    lib = _load()
    p = np.array(p5, np.float64)
    c = np.array(c15, np.float64)
    chi = np.zeros(1, np.float64)
    rc = lib.oracle_update(_dptr(p), _dptr(c), ym, zm, _dptr(chi))
    return rc, p, c, chi[0]


def rotate(x: float, p5, c15, dalpha: float):
    lib = _load()
    xx = np.array([x], np.float64)
    p = np.array(p5, np.float64)
    c = np.array(c15, np.float64)
    rc = lib.oracle_rotate(_dptr(xx), _dptr(p), _dptr(c), dalpha)
    return rc, xx[0], p, c


def fit_points(x, y, z, bz: float, seed_p5, c15_init=None):
    lib = _load()
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    p = np.array(seed_p5, np.float64)
    c = np.zeros(15, np.float64) if c15_init is None else np.array(c15_init, np.float64)
    rc = lib.oracle_fit_points(len(x), _dptr(x), _dptr(y), _dptr(z), bz, _dptr(p), _dptr(c))
    return rc, p, c


def dca_arc(x0: float, y0: float, snp: float, k: float) -> float:
    """Signed transverse arc length from (x0, y0), sin(phi) = snp, curvature
    k = dphi/ds, to the closest approach to the origin."""
    return float(_load().oracle_dca_arc(x0, y0, snp, k))


def _take(lib, ptr, n, dtype):
    out = np.ctypeslib.as_array(ptr, shape=(n,)).copy() if n > 0 else np.zeros(0, dtype)
    lib.oracle_buffer_free(ctypes.cast(ptr, ctypes.c_void_p))
    return out.astype(dtype, copy=False)


def rans_encode(sym) -> np.ndarray:
    """One byte stream through the CTF's entropy coder (table, chunk sizes,
    payloads)."""
    lib = _load()
    a = np.ascontiguousarray(np.asarray(sym, dtype=np.uint8))
    out = ctypes.POINTER(ctypes.c_uint8)()
    n = lib.oracle_rans_encode(a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), len(a), ctypes.byref(out))
    return _take(lib, out, n, np.uint8)


def rans_decode(blob):
    lib = _load()
    a = np.ascontiguousarray(np.asarray(blob, dtype=np.uint8))
    out = ctypes.POINTER(ctypes.c_uint8)()
    n = lib.oracle_rans_decode(a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), len(a), ctypes.byref(out))
    if n < 0:
        raise OracleError("malformed rANS stream")
    return _take(lib, out, n, np.uint8)


def ctf_normalize(count) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(np.asarray(count, dtype=np.uint64))
    assert len(c) == 256
    f = np.zeros(256, np.uint16)
    lib.oracle_ctf_normalize(c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                             f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)))
    return f


def ctf_encode(sector, row, y, z, trk_off, trk_cl, trk_qpt, sorted_orig) -> np.ndarray:
    """The compressed TF of the given clusters (integer units) and tracks."""
    lib = _load()
    i32 = lambda v: np.ascontiguousarray(np.asarray(v, dtype=np.int32))
    sector, row, y, z, trk_cl, sorted_orig = map(i32, (sector, row, y, z, trk_cl, sorted_orig))
    trk_off = np.ascontiguousarray(np.asarray(trk_off, dtype=np.int64))
    trk_qpt = np.ascontiguousarray(np.asarray(trk_qpt, dtype=np.float64))
    P = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))
    out = ctypes.POINTER(ctypes.c_uint8)()
    n = lib.oracle_ctf_encode(len(sector), P(sector, ctypes.c_int32), P(row, ctypes.c_int32), P(y, ctypes.c_int32),
                              P(z, ctypes.c_int32), len(trk_off) - 1, P(trk_off, ctypes.c_int64),
                              P(trk_cl, ctypes.c_int32), P(trk_qpt, ctypes.c_double),
                              P(sorted_orig, ctypes.c_int32), len(sorted_orig), ctypes.byref(out))
    return _take(lib, out, n, np.uint8)


def ctf_decode(blob) -> dict:
    """The cluster sequence of a compressed TF: sector, row, y, zeta arrays
    and the kept tracks' cluster counts (the tracks come first)."""
    lib = _load()
    a = np.ascontiguousarray(np.asarray(blob, dtype=np.uint8))
    ptrs = [ctypes.POINTER(ctypes.c_int32)() for _ in range(4)]
    nt = ctypes.c_int64()
    lens = ctypes.POINTER(ctypes.c_int64)()
    n = lib.oracle_ctf_decode(a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), len(a), *[ctypes.byref(p) for p in ptrs],
                              ctypes.byref(nt), ctypes.byref(lens))
    if n < 0:
        raise OracleError("malformed compressed TF")
    out = {k: _take(lib, p, n, np.int32) for k, p in zip(("sector", "row", "y", "z"), ptrs)}
    out["track_len"] = _take(lib, lens, nt.value, np.int64)
    return out


def clusterize(digits) -> np.ndarray:
    """12-byte cluster records (uint8 [n, 12]) of sorted raw digits (an object
    with sector, row, pad, time, adc arrays)."""
    lib = _load()
    arrs = [np.ascontiguousarray(np.asarray(getattr(digits, k), dtype=t)) for k, t in
            (("sector", np.uint8), ("row", np.uint8), ("pad", np.uint8), ("time", np.uint32), ("adc", np.uint16))]
    out = ctypes.POINTER(ctypes.c_uint8)()
    n = lib.oracle_clusterize(len(arrs[0]), *[a.ctypes.data for a in arrs], ctypes.byref(out))
    if n < 0:
        lib.oracle_buffer_free(ctypes.cast(out, ctypes.c_void_p))
        raise OracleError("digits not sorted or out of range")
    return _take(lib, out, 12 * n, np.uint8).reshape(-1, 12)
