"""Seeded synthetic TPC Time Frames (the input recipe).

The paper's benchmark inputs are ALICE Time Frames in raw format (Sec. 3.2);
none ship with it, so these seeded generators stand in for them, with the
shapes of the workloads the tracker is measured on:

* ``single_sector``  - one sector, one collision at t = 0, 80 primaries,
  float y/z, ~13 k clusters.
* ``full_tpc_1ms``   - 36 sectors, 50 collisions at uniform times over 1 ms,
  2900 primaries each, float y/z, ~22 M clusters.
* ``full_tf``        - one Time Frame of 128 LHC orbits at a 50 kHz Pb-Pb
  interaction rate (Poisson collision times, falling minimum-bias
  multiplicity), 12-byte fixed-point records, ~250 M clusters.
* ``chunk_mix``      - uneven sub-Time-Frame chunks (Poisson-many collisions,
  a quarter pp-like), for batched launches.
* ``serving_pool``   - Time Frames of mixed size for a served stream: half
  Pb-Pb with a uniform number of collisions (10..570), half pp-like with
  2000 collisions at dN/deta = 6 (~3 M clusters).

Physics of every primary: pT ~ 0.05 GeV + Exp(0.6 GeV), |eta| < 0.9,
charge +-1, helix in Bz = 0.5 T, one cluster per crossed pad row, Gaussian
smearing sigma_y = 0.1 cm, sigma_z = 0.15 cm, plus 10 % uniform noise
clusters.  All random draws are seeded; the per-track draws are
counter-based inside ``o2gen.c``.  Options: ``angular_errors`` adds the
pad-length term (L tan phi)^2 / 12 and (L tan lambda)^2 / 12 (L = 160/151
cm) to the smearing variances; ``row_drop`` loses each track cluster with
that probability (missing pad rows).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

from .. import _build

VDRIFT = 2.58          # cm/us
BZ = 0.5               # T
ORBIT_US = 88.924      # LHC orbit
TF_ORBITS = 128
PBPB_RATE_KHZ = 50.0
# Scale factor on the falling multiplicity shape that brings the expected
# Time Frame to ~250 M clusters (solved once from measured clusters/track).
FULL_TF_MULT_SCALE = 3.6

FMT_FLOAT = 0
FMT_FIXED = 1


class _GenParams(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_coll", ctypes.c_int32),
        ("t0", ctypes.POINTER(ctypes.c_double)),
        ("ntracks", ctypes.POINTER(ctypes.c_int32)),
        ("pt_mean", ctypes.c_double),
        ("pt_min", ctypes.c_double),
        ("eta_min", ctypes.c_double),
        ("eta_max", ctypes.c_double),
        ("sector_only", ctypes.c_int32),
        ("zvtx_sigma", ctypes.c_double),
        ("sigma_y", ctypes.c_double),
        ("sigma_z", ctypes.c_double),
        ("noise_frac", ctypes.c_double),
        ("bz", ctypes.c_double),
        ("vdrift", ctypes.c_double),
        ("t_window", ctypes.c_double),
        ("nthreads", ctypes.c_int32),
        ("angular_errors", ctypes.c_int32),
        ("row_drop", ctypes.c_double),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build_gen()
        lib = ctypes.CDLL(path)
        lib.o2gen_run.restype = ctypes.c_void_p
        lib.o2gen_run.argtypes = [ctypes.POINTER(_GenParams), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_int64)]
        lib.o2gen_copy.restype = None
        lib.o2gen_copy.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 7
        lib.o2gen_truth.restype = None
        lib.o2gen_truth.argtypes = [ctypes.c_void_p] * 4
        lib.o2gen_free.restype = None
        lib.o2gen_free.argtypes = [ctypes.c_void_p]
        pp = ctypes.POINTER(ctypes.c_void_p)
        lib.o2dig_run.restype = ctypes.c_int64
        lib.o2dig_run.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int32] + [pp] * 5
        lib.o2dig_free.restype = None
        lib.o2dig_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class TimeFrame:
    """One Time Frame of clusters in submission order.

    ``fmt`` FMT_FLOAT: ``sector``, ``row`` (uint8), ``y``, ``z`` (float32;
    z is the apparent z for a collision at t = 0, side * (250 - v_d t)), or
    ``time`` (float32 drift time in us) instead of ``z``.
    ``fmt`` FMT_FIXED: ``packed`` (uint8 [n, 12]) records.
    ``truth_track`` is the generating track id (-1 noise); ``truth`` holds
    per-track pt, eta, phi0, zv, t0, q, coll.
    """
    n: int
    fmt: int
    sector: np.ndarray
    row: np.ndarray
    y: np.ndarray | None = None
    z: np.ndarray | None = None
    time: np.ndarray | None = None
    packed: np.ndarray | None = None
    truth_track: np.ndarray | None = None
    truth: dict = field(default_factory=dict)
    coll_time: np.ndarray | None = None
    bz: float = BZ
    vdrift: float = VDRIFT
    name: str = ""


def generate(*, seed: int, t0, ntracks, fmt: int = FMT_FLOAT, sector_only: int = -1,
             zvtx_sigma: float = 0.0, sigma_y: float = 0.1, sigma_z: float = 0.15,
             noise_frac: float = 0.1, bz: float = BZ, vdrift: float = VDRIFT,
             t_window: float | None = None, pt_mean: float = 0.6, pt_min: float = 0.05,
             eta_min: float = -0.9, eta_max: float = 0.9, with_truth: bool = True, nthreads: int | None = None,
             name: str = "", angular_errors: bool = False, row_drop: float = 0.0) -> TimeFrame:
    lib = _load()
    t0 = np.ascontiguousarray(np.asarray(t0, dtype=np.float64))
    ntracks = np.ascontiguousarray(np.asarray(ntracks, dtype=np.int32))
    assert t0.shape == ntracks.shape
    if t_window is None:
        t_window = float(t0.max(initial=0.0)) + 250.0 / vdrift + 1.0
    P = _GenParams()
    P.seed = seed
    P.n_coll = len(t0)
    P.t0 = t0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    P.ntracks = ntracks.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    P.pt_mean, P.pt_min, P.eta_min, P.eta_max = pt_mean, pt_min, eta_min, eta_max
    P.sector_only = sector_only
    P.zvtx_sigma, P.sigma_y, P.sigma_z = zvtx_sigma, sigma_y, sigma_z
    P.noise_frac, P.bz, P.vdrift, P.t_window = noise_frac, bz, vdrift, t_window
    P.nthreads = nthreads or max(1, min(32, os.cpu_count() or 1))
    P.angular_errors = int(angular_errors)
    P.row_drop = row_drop
    n = ctypes.c_int64()
    nt = ctypes.c_int64()
    h = lib.o2gen_run(ctypes.byref(P), ctypes.byref(n), ctypes.byref(nt))
    try:
        n = n.value
        tf = TimeFrame(n=n, fmt=fmt, sector=np.empty(n, np.uint8), row=np.empty(n, np.uint8),
                       bz=bz, vdrift=vdrift, name=name)
        # the interaction record of the TF: the collision times, ascending
        # (the truth's collision index points into it)
        tf.coll_time = t0.copy() if np.all(np.diff(t0) >= 0) else None
        if fmt == FMT_FLOAT:
            tf.y = np.empty(n, np.float32)
            tf.z = np.empty(n, np.float32)
        else:
            tf.packed = np.empty((n, 12), np.uint8)
        if with_truth:
            tf.truth_track = np.empty(n, np.int32)
        lib.o2gen_copy(h, _ptr(tf.sector), _ptr(tf.row), _ptr(tf.y), _ptr(tf.z), None,
                       _ptr(tf.packed), _ptr(tf.truth_track))
        if with_truth:
            d5 = np.empty((nt.value, 5), np.float64)
            q = np.empty(nt.value, np.int32)
            coll = np.empty(nt.value, np.int32)
            lib.o2gen_truth(h, _ptr(d5), _ptr(q), _ptr(coll))
            tf.truth = dict(pt=d5[:, 0], eta=d5[:, 1], phi0=d5[:, 2], zv=d5[:, 3], t0=d5[:, 4], q=q, coll=coll)
    finally:
        lib.o2gen_free(h)
    return tf


# --------------------------------------------------------------- workloads
def single_sector(seed: int = 20210607, ntracks: int = 80, t0: float = 0.0, **kw) -> TimeFrame:
    """1 sector (s = 0, side A), one collision at ``t0`` (default 0), z_vtx = 0,
    float y/z.

    The primaries are drawn with 0 < eta < 0.9 and phi inside the sector so
    that they head into the one simulated sector.  With t0 = 0 the clusters
    next to the end plate arrive at the very start of the readout window and
    those whose smeared time falls before it are lost (a Time-Frame edge)."""
    kw.setdefault("name", "single_sector")
    kw.setdefault("eta_min", 0.0)
    return generate(seed=seed, t0=[t0], ntracks=[ntracks], sector_only=0, zvtx_sigma=0.0, **kw)


def full_tpc_1ms(seed: int = 20210608, n_coll: int = 50, ntracks: int = 2900, **kw) -> TimeFrame:
    """36 sectors, ``n_coll`` collisions at U(0, 1 ms), z_vtx ~ N(0, 5 cm)."""
    rng = np.random.default_rng(seed)
    t0 = np.sort(rng.uniform(0.0, 1000.0, n_coll))
    kw.setdefault("name", f"full_tpc_1ms_{n_coll}coll")
    return generate(seed=seed, t0=t0, ntracks=np.full(n_coll, ntracks), zvtx_sigma=5.0,
                    t_window=1000.0, **kw)


def falling_multiplicity(rng: np.random.Generator, n: int) -> np.ndarray:
    """dN/deta per collision with pdf proportional to 1/(m + 50) on [0, 2000]."""
    u = rng.uniform(0.0, 1.0, n)
    return 50.0 * np.power(41.0, u) - 50.0


def full_tf(seed: int = 20210609, orbits: int = TF_ORBITS, rate_khz: float = PBPB_RATE_KHZ,
            mult_scale: float = FULL_TF_MULT_SCALE, fmt: int = FMT_FIXED, **kw) -> TimeFrame:
    """One Time Frame: ``orbits`` LHC orbits, Poisson collision times at
    ``rate_khz``, falling minimum-bias multiplicity scaled by ``mult_scale``."""
    rng = np.random.default_rng(seed)
    t_len = orbits * ORBIT_US
    times = []
    t = rng.exponential(1000.0 / rate_khz)
    while t < t_len:
        times.append(t)
        t += rng.exponential(1000.0 / rate_khz)
    t0 = np.asarray(times)
    m = falling_multiplicity(rng, len(t0))
    ntr = np.rint(mult_scale * 1.8 * m).astype(np.int32)
    kw.setdefault("name", f"full_tf_{orbits}orbits")
    kw.setdefault("with_truth", False)
    return generate(seed=seed, t0=t0, ntracks=ntr, zvtx_sigma=5.0, t_window=t_len, fmt=fmt, **kw)


def chunk_mix(seed: int = 20210610, n_chunks: int = 64, mean_coll: float = 20.0,
              chunk_us: float = 400.0, fmt: int = FMT_FIXED, **kw) -> list[TimeFrame]:
    """Uneven sub-Time-Frame chunks: Poisson(mean_coll) collisions each; a
    quarter of the chunks are pp-like (dN/deta = 6)."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_chunks):
        ncoll = max(1, int(rng.poisson(mean_coll)))
        t0 = np.sort(rng.uniform(0.0, chunk_us, ncoll))
        if c % 4 == 3:
            ntr = np.full(ncoll, int(round(6 * 1.8)), np.int32)
        else:
            ntr = np.rint(1.8 * falling_multiplicity(rng, ncoll)).astype(np.int32)
        out.append(generate(seed=seed * 1000 + c, t0=t0, ntracks=ntr, zvtx_sigma=5.0,
                            t_window=chunk_us, fmt=fmt, with_truth=False, name=f"chunk{c}", **kw))
    return out



def serving_pool(seed: int = 20210611, n_tf: int = 24, orbits: int = TF_ORBITS, coll_min: int = 10,
                 coll_max: int = 570, pp_coll: int = 2000, pp_dndeta: float = 6.0,
                 mult_scale: float = FULL_TF_MULT_SCALE, fmt: int = FMT_FIXED, **kw) -> list[TimeFrame]:
    """A pool of Time Frames to replay as a served stream.  Even entries are
    Pb-Pb (collision count uniform on [coll_min, coll_max], collision times
    uniform over the frame, falling multiplicity scaled like ``full_tf``), odd
    entries pp-like (``pp_coll`` collisions of dN/deta = ``pp_dndeta``)."""
    rng = np.random.default_rng(seed)
    t_len = orbits * ORBIT_US
    out = []
    for i in range(n_tf):
        if i % 2 == 0:
            k = int(rng.integers(coll_min, coll_max + 1))
            t0 = np.sort(rng.uniform(0.0, t_len, k))
            ntr = np.rint(mult_scale * 1.8 * falling_multiplicity(rng, k)).astype(np.int32)
            name = f"pbpb{i}_{k}coll"
        else:
            t0 = np.sort(rng.uniform(0.0, t_len, pp_coll))
            ntr = np.full(pp_coll, int(round(pp_dndeta * 1.8)), np.int32)
            name = f"pp{i}"
        out.append(generate(seed=seed * 1000 + i, t0=t0, ntracks=ntr, zvtx_sigma=5.0, t_window=t_len, fmt=fmt,
                            with_truth=False, name=name, **kw))
    return out


def float_time_from_fixed(tf: TimeFrame) -> TimeFrame:
    """The same clusters as a fixed-point TF, in float format with drift time
    instead of z: y = y_u / 160 cm and time = time64 / 320 us, which quantize
    back to the same integer units."""
    rec = tf.packed
    t64 = rec[:, 0:4].copy().view(np.uint32).ravel()
    pad = rec[:, 4:6].copy().view(np.uint16).ravel().astype(np.int64)
    row = rec[:, 8].copy()
    sector = rec[:, 9].copy()
    npads = np.floor(2.0 * (85.0 + row.astype(np.float64) * 160.0 / 151.0) * math.tan(math.radians(10.0)) / 0.4)
    yu = pad - 32 * npads.astype(np.int64)
    return TimeFrame(n=tf.n, fmt=FMT_FLOAT, sector=sector, row=row, y=(yu / 160.0).astype(np.float32),
                     time=(t64.astype(np.float64) / 320.0).astype(np.float32), bz=tf.bz, vdrift=tf.vdrift,
                     name=tf.name + "_time", coll_time=tf.coll_time)


@dataclass
class Digits:
    """Zero-suppressed raw ADC digits, sorted by (sector, row, time, pad)."""
    n: int
    sector: np.ndarray
    row: np.ndarray
    pad: np.ndarray
    time: np.ndarray
    adc: np.ndarray
    name: str = ""


def digits_from(tf: TimeFrame, seed: int = 1, sigma_pad: float = 0.7, sigma_time: float = 0.8,
                noise: float = 0.6, threshold: int = 2) -> Digits:
    """Raw ADC digits of a fixed-format TF's clusters (see o2digits.c):
    Gaussian charge spread over 5 x 5 pad x time cells, summed, noise added,
    rounded, zero-suppressed below ``threshold``."""
    assert tf.fmt == FMT_FIXED
    lib = _load()
    ptrs = [ctypes.c_void_p() for _ in range(5)]
    rec = np.ascontiguousarray(tf.packed)
    nd = lib.o2dig_run(tf.n, rec.ctypes.data, seed, sigma_pad, sigma_time, noise, threshold,
                       *[ctypes.byref(p) for p in ptrs])
    out = []
    for p, dt in zip(ptrs, (np.uint8, np.uint8, np.uint8, np.uint32, np.uint16)):
        if nd > 0:
            buf = (ctypes.c_char * (nd * np.dtype(dt).itemsize)).from_address(p.value)
            out.append(np.frombuffer(buf, dtype=dt).copy())
        else:
            out.append(np.zeros(0, dt))
        lib.o2dig_free(p)
    return Digits(n=int(nd), sector=out[0], row=out[1], pad=out[2], time=out[3], adc=out[4],
                  name=tf.name + "_digits")
