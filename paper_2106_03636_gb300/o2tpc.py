"""ctypes binding of the C-ABI in ``include/o2tpc.h`` (argument marshalling only).

Every step of the tracker runs in ``libo2tpc.so``; this module only loads it,
declares the structures and calls the entry points under their C names.  The
``Tracker`` helper wraps the create / submit / poll / release cycle and can
route the library's device allocations through PyTorch's caching allocator
and run it on a ``torch.cuda.Stream``.  There is no CPU fallback: without the
built library every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

O2TPC_OK = 0
O2TPC_PENDING = 1
O2TPC_EINVAL = -1
O2TPC_ENOMEM = -2
O2TPC_EAGAIN = -3
O2TPC_ETOOBIG = -4
O2TPC_ECUDA = -5
O2TPC_ETIMEOUT = -6
O2TPC_ENOTFOUND = -7

O2TPC_FMT_FLOAT = 0
O2TPC_FMT_FIXED = 1
O2TPC_LOC_HOST = 0
O2TPC_LOC_DEVICE = 1

O2TPC_FLAG_KEEP_STAGES = 1 << 0
O2TPC_FLAG_AUTOTUNE = 1 << 3
O2TPC_FLAG_GRAPH_TIGHT = 1 << 4
O2TPC_FLAG_COMPRESS = 1 << 5
O2TPC_FLAG_NO_BATCHING = 1 << 1
O2TPC_FLAG_FORCE_FP64 = 1 << 2
O2TPC_FLAG_COOP_SEARCH = 1 << 6
O2TPC_FLAG_ROW_STEP2 = 1 << 7
O2TPC_FLAG_ANGULAR_ERRORS = 1 << 8

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class o2tpc_config(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int32),
        ("mem_budget", ctypes.c_uint64),
        ("max_inflight", ctypes.c_int32),
        ("max_batch", ctypes.c_int32),
        ("bz_tesla", ctypes.c_double),
        ("vdrift_cm_us", ctypes.c_double),
        ("flags", ctypes.c_uint32),
        ("dev_alloc", ALLOC_FN),
        ("dev_free", FREE_FN),
        ("alloc_user", ctypes.c_void_p),
        ("stream", ctypes.c_void_p),
        ("batch_full_clusters", ctypes.c_uint64),
        ("nf_hits_per_block", ctypes.c_int32),
        ("sort_threads_per_row", ctypes.c_int32),
        ("graph_max_clusters", ctypes.c_uint64),
        ("graph_max_tfs", ctypes.c_int32),
        ("nf_staged", ctypes.c_int32),
        ("tune_cache_path", ctypes.c_char_p),
        ("debug_inject", ctypes.c_uint32),
    ]


class o2tpc_tuning(ctypes.Structure):
    _fields_ = [
        ("tuned", ctypes.c_int32),
        ("nf_hits_per_block", ctypes.c_int32),
        ("nf_staged", ctypes.c_int32),
        ("sort_threads_per_row", ctypes.c_int32),
        ("tuned_on_clusters", ctypes.c_int32),
        ("nf_ms", ctypes.c_float * 6),
        ("sort_ms", ctypes.c_float * 3),
    ]


class o2tpc_tf(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64),
        ("format", ctypes.c_int32),
        ("location", ctypes.c_int32),
        ("sector", ctypes.c_void_p),
        ("row", ctypes.c_void_p),
        ("y", ctypes.c_void_p),
        ("z", ctypes.c_void_p),
        ("time", ctypes.c_void_p),
        ("packed", ctypes.c_void_p),
        ("user_tag", ctypes.c_uint64),
        ("coll_time", ctypes.c_void_p),
        ("n_coll", ctypes.c_uint64),
    ]


class o2tpc_stats(ctypes.Structure):
    _fields_ = [
        ("n_clusters", ctypes.c_uint64),
        ("n_tracklets", ctypes.c_uint64),
        ("n_sector_tracks", ctypes.c_uint64),
        ("n_tracks", ctypes.c_uint64),
        ("n_fp64_fallback", ctypes.c_uint64),
        ("batch_size", ctypes.c_uint32),
        ("ms_queue", ctypes.c_float),
        ("ms_batch", ctypes.c_float),
        ("ms_device", ctypes.c_float),
        ("n_launches", ctypes.c_uint64),
        ("ms_stage", ctypes.c_float * 18),
        ("captured", ctypes.c_uint32),
        ("events", ctypes.c_uint32),
    ]

STAGES = ("ingest", "sort", "neighbours", "clean_starts", "tracklets", "selection", "sector_fit", "merge",
          "refit", "sizes", "download", "host_prep", "upload", "upload_wait", "tl_out", "tl_in", "continuous",
          "compress")


class o2tpc_result(ctypes.Structure):
    _fields_ = [
        ("n_tracks", ctypes.c_uint64),
        ("offsets", ctypes.POINTER(ctypes.c_uint64)),
        ("cluster_idx", ctypes.POINTER(ctypes.c_uint32)),
        ("x", ctypes.POINTER(ctypes.c_float)),
        ("alpha", ctypes.POINTER(ctypes.c_float)),
        ("par", ctypes.POINTER(ctypes.c_float)),
        ("cov", ctypes.POINTER(ctypes.c_float)),
        ("chi2", ctypes.POINTER(ctypes.c_float)),
        ("ndf", ctypes.POINTER(ctypes.c_int32)),
        ("sector", ctypes.POINTER(ctypes.c_uint8)),
        ("flags", ctypes.POINTER(ctypes.c_uint8)),
        ("zeta_ref", ctypes.POINTER(ctypes.c_uint32)),
        ("t0", ctypes.POINTER(ctypes.c_float)),
        ("t0_err", ctypes.POINTER(ctypes.c_float)),
        ("t0_lo", ctypes.POINTER(ctypes.c_float)),
        ("t0_hi", ctypes.POINTER(ctypes.c_float)),
        ("mate", ctypes.POINTER(ctypes.c_int32)),
        ("collision", ctypes.POINTER(ctypes.c_int32)),
        ("ctf", ctypes.POINTER(ctypes.c_uint8)),
        ("ctf_bytes", ctypes.c_uint64),
        ("stats", o2tpc_stats),
        ("user_tag", ctypes.c_uint64),
        ("status", ctypes.c_int32),
    ]


class o2tpc_digits(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64),
        ("sector", ctypes.c_void_p),
        ("row", ctypes.c_void_p),
        ("pad", ctypes.c_void_p),
        ("time", ctypes.c_void_p),
        ("adc", ctypes.c_void_p),
    ]


class o2tpc_ctf_clusters(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64),
        ("n_tracks", ctypes.c_uint64),
        ("sector", ctypes.POINTER(ctypes.c_int32)),
        ("row", ctypes.POINTER(ctypes.c_int32)),
        ("y", ctypes.POINTER(ctypes.c_int32)),
        ("zeta", ctypes.POINTER(ctypes.c_int32)),
        ("track_len", ctypes.POINTER(ctypes.c_uint32)),
    ]


class O2TPCError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {o2tpc_strerror(status)} ({status})")


_lib = None


def load(build: bool = True) -> ctypes.CDLL:
    """Loads the in-tree ``libo2tpc.so`` (building it first if asked)."""
    global _lib
    if _lib is None:
        path = _build.build_tpc() if build else _build.TPC_SO
        if not os.path.exists(path):
            raise RuntimeError(f"libo2tpc.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        lib.o2tpc_create.restype = ctypes.c_int
        lib.o2tpc_create.argtypes = [ctypes.POINTER(o2tpc_config), ctypes.POINTER(vp)]
        lib.o2tpc_submit_tf.restype = ctypes.c_int
        lib.o2tpc_submit_tf.argtypes = [vp, ctypes.POINTER(o2tpc_tf), ctypes.POINTER(ctypes.c_uint64)]
        lib.o2tpc_submit_many.restype = ctypes.c_int
        lib.o2tpc_submit_many.argtypes = [vp, ctypes.POINTER(o2tpc_tf), ctypes.c_uint32,
                                          ctypes.POINTER(ctypes.c_uint64)]
        lib.o2tpc_poll.restype = ctypes.c_int
        lib.o2tpc_poll.argtypes = [vp, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(ctypes.POINTER(o2tpc_result))]
        lib.o2tpc_result_release.restype = None
        lib.o2tpc_result_release.argtypes = [vp, ctypes.POINTER(o2tpc_result)]
        lib.o2tpc_destroy.restype = ctypes.c_int
        lib.o2tpc_destroy.argtypes = [vp]
        lib.o2tpc_strerror.restype = ctypes.c_char_p
        lib.o2tpc_strerror.argtypes = [ctypes.c_int32]
        lib.o2tpc_sort_tf_static.restype = ctypes.c_int
        lib.o2tpc_sort_tf_static.argtypes = [ctypes.POINTER(o2tpc_tf), ctypes.c_double, vp, vp, vp, vp,
                                             ctypes.c_uint64, vp]
        lib.o2tpc_get_tuning.restype = ctypes.c_int
        lib.o2tpc_get_tuning.argtypes = [vp, ctypes.POINTER(o2tpc_tuning)]
        lib.o2tpc_clusterize.restype = ctypes.c_int
        lib.o2tpc_clusterize.argtypes = [ctypes.POINTER(o2tpc_digits), vp, ctypes.c_uint64,
                                         ctypes.POINTER(ctypes.c_uint64), vp]
        lib.o2tpc_ctf_decode.restype = ctypes.c_int
        lib.o2tpc_ctf_decode.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(o2tpc_ctf_clusters)]
        lib.o2tpc_ctf_records.restype = ctypes.c_int
        lib.o2tpc_ctf_records.argtypes = [ctypes.POINTER(o2tpc_ctf_clusters), vp]
        lib.o2tpc_ctf_free.restype = None
        lib.o2tpc_ctf_free.argtypes = [ctypes.POINTER(o2tpc_ctf_clusters)]
        lib.o2tpc_get_stage.restype = ctypes.c_int
        lib.o2tpc_get_stage.argtypes = [vp, ctypes.c_uint64, ctypes.c_char_p, vp, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_uint64)]
        _lib = lib
    return _lib


# ------------------------------------------------------- C names, 1:1
def o2tpc_create(cfg: o2tpc_config | None):
    out = ctypes.c_void_p()
    rc = load().o2tpc_create(ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(out))
    return rc, out


def o2tpc_submit_tf(ctx, tf: o2tpc_tf):
    t = ctypes.c_uint64()
    rc = load().o2tpc_submit_tf(ctx, ctypes.byref(tf), ctypes.byref(t))
    return rc, t.value


def o2tpc_submit_many(ctx, tfs: list):
    arr = (o2tpc_tf * len(tfs))(*tfs)
    t = (ctypes.c_uint64 * len(tfs))()
    rc = load().o2tpc_submit_many(ctx, arr, len(tfs), t)
    return rc, list(t)


def o2tpc_get_tuning(ctx):
    t = o2tpc_tuning()
    rc = load().o2tpc_get_tuning(ctx, ctypes.byref(t))
    return rc, t


def o2tpc_poll(ctx, ticket: int, timeout_ms: int):
    out = ctypes.POINTER(o2tpc_result)()
    rc = load().o2tpc_poll(ctx, ticket, timeout_ms, ctypes.byref(out))
    return rc, out


def o2tpc_result_release(ctx, res) -> None:
    load().o2tpc_result_release(ctx, res)


def o2tpc_destroy(ctx) -> int:
    return load().o2tpc_destroy(ctx)


def o2tpc_strerror(status: int) -> str:
    return load().o2tpc_strerror(status).decode()


def o2tpc_get_stage(ctx, ticket: int, name: str, dst, capacity: int):
    need = ctypes.c_uint64()
    rc = load().o2tpc_get_stage(ctx, ticket, name.encode(), dst, capacity, ctypes.byref(need))
    return rc, need.value


O2TPC_STATIC_MAX_CLUSTERS = 262144


def o2tpc_sort_tf_static(tf: o2tpc_tf, vdrift: float, sorted_orig, sorted_yz, row_grid, cell_start,
                         cell_capacity: int, stream) -> int:
    """Allocation-free binning + sort of one TF: every pointer is a device
    buffer the caller owns; nothing is allocated by the call."""
    return load().o2tpc_sort_tf_static(ctypes.byref(tf), vdrift, sorted_orig, sorted_yz, row_grid, cell_start,
                                       cell_capacity, stream)


def o2tpc_clusterize(digits: o2tpc_digits, records, cap: int, stream):
    n = ctypes.c_uint64()
    rc = load().o2tpc_clusterize(ctypes.byref(digits), records, cap, ctypes.byref(n), stream)
    return rc, n.value


def clusterize(arrays: dict, stream=None, cap: int | None = None):
    """Clusterizer over device tensors ``sector, row, pad, time, adc``
    (sorted digits); returns (status, records as a uint8 [n, 12] device
    tensor).  ``stream``: a torch.cuda.Stream (default: the current one)."""
    import torch

    n = int(arrays["adc"].numel())
    cap = n if cap is None else cap
    out = torch.empty((max(cap, 1), 12), dtype=torch.uint8, device=arrays["adc"].device)
    d = o2tpc_digits(n=n, sector=_ptr(arrays["sector"]), row=_ptr(arrays["row"]), pad=_ptr(arrays["pad"]),
                     time=_ptr(arrays["time"]), adc=_ptr(arrays["adc"]))
    st = stream if stream is not None else torch.cuda.current_stream()
    rc, nc = o2tpc_clusterize(d, out.data_ptr(), cap, st.cuda_stream)
    return rc, (out[:nc] if rc == O2TPC_OK else out[:0]), nc


def ctf_decode(blob) -> dict:
    """Host decoder of a compressed TF (numpy uint8 array): the cluster
    sequence as numpy arrays (sector, row, y, zeta), as fixed-format records
    (records, uint8 [n, 12]) and the kept tracks' cluster counts (track_len).
    Raises O2TPCError on a damaged blob."""
    a = np.ascontiguousarray(np.asarray(blob, dtype=np.uint8))
    c = o2tpc_ctf_clusters()
    rc = load().o2tpc_ctf_decode(a.ctypes.data, len(a), ctypes.byref(c))
    if rc != O2TPC_OK:
        raise O2TPCError(rc, "o2tpc_ctf_decode")
    try:
        n, nt = int(c.n), int(c.n_tracks)
        out = {k: _np(getattr(c, k), n, np.int32) for k in ("sector", "row", "y", "zeta")}
        out["track_len"] = _np(c.track_len, nt, np.uint32)
        rec = np.zeros((max(n, 1), 12), np.uint8)
        rc = load().o2tpc_ctf_records(ctypes.byref(c), rec.ctypes.data)
        if rc != O2TPC_OK:
            raise O2TPCError(rc, "o2tpc_ctf_records")
        out["records"] = rec[:n]
    finally:
        load().o2tpc_ctf_free(ctypes.byref(c))
    return out


# ---------------------------------------------------------- helpers
def _ptr(a) -> int | None:
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _np(ptr, n, dtype, shape=None):
    if n == 0:
        return np.zeros(shape if shape else 0, dtype)
    a = np.ctypeslib.as_array(ptr, shape=(n,)).copy()
    return a.reshape(shape) if shape else a


def result_to_dict(r: o2tpc_result) -> dict:
    """Copies a result into numpy arrays."""
    n = int(r.n_tracks)
    off = _np(r.offsets, n + 1, np.uint64)
    ncl = int(off[-1]) if n else 0
    return dict(
        n_tracks=n, offsets=off, cluster_idx=_np(r.cluster_idx, ncl, np.uint32),
        x=_np(r.x, n, np.float32), alpha=_np(r.alpha, n, np.float32),
        par=_np(r.par, 5 * n, np.float32, (n, 5)), cov=_np(r.cov, 15 * n, np.float32, (n, 15)),
        chi2=_np(r.chi2, n, np.float32), ndf=_np(r.ndf, n, np.int32), sector=_np(r.sector, n, np.uint8),
        flags=_np(r.flags, n, np.uint8), zeta_ref=_np(r.zeta_ref, n, np.uint32),
        t0=_np(r.t0, n, np.float32), t0_err=_np(r.t0_err, n, np.float32), t0_lo=_np(r.t0_lo, n, np.float32),
        t0_hi=_np(r.t0_hi, n, np.float32), mate=_np(r.mate, n, np.int32), collision=_np(r.collision, n, np.int32),
        ctf=_np(r.ctf, int(r.ctf_bytes), np.uint8),
        status=int(r.status), user_tag=int(r.user_tag),
        stats={k: (list(getattr(r.stats, k)) if k == "ms_stage" else getattr(r.stats, k))
               for k, _ in o2tpc_stats._fields_},
    )


def make_tf(tf, location: int = O2TPC_LOC_HOST, arrays: dict | None = None, user_tag: int = 0,
            coll_time=None) -> o2tpc_tf:
    """Builds an ``o2tpc_tf`` from a ``synth.TimeFrame`` (host numpy arrays)
    or from ``arrays`` (numpy or torch tensors, host or device).  The
    interaction times come from ``coll_time``, else ``arrays["coll_time"]``,
    else the TF's ``coll_time`` (host, ascending us; an empty array: none);
    the returned struct keeps them alive in its ``_coll`` attribute."""
    src = arrays if arrays is not None else {k: getattr(tf, k, None) for k in ("sector", "row", "y", "z", "time",
                                                                            "packed")}
    t = o2tpc_tf()
    t.n = int(tf.n)
    t.format = int(tf.fmt)
    t.location = location
    if t.format == O2TPC_FMT_FIXED:
        t.packed = _ptr(src["packed"])
    else:
        t.sector, t.row, t.y = (_ptr(src[k]) for k in ("sector", "row", "y"))
        if src.get("z") is not None:
            t.z = _ptr(src["z"])
        else:
            t.time = _ptr(src["time"])
    t.user_tag = user_tag
    ct = coll_time if coll_time is not None else (arrays or {}).get("coll_time", getattr(tf, "coll_time", None))
    if ct is not None and len(ct):
        ct = np.ascontiguousarray(np.asarray(ct, dtype=np.float64))
        t._coll = ct
        t.coll_time = ct.ctypes.data
        t.n_coll = len(ct)
    return t


class Tracker:
    """One context on one GPU, running on its own ``torch.cuda.Stream``.

    ``torch_memory``: allocate the library's device buffers from PyTorch's
    caching allocator (host-resident inputs are then copied in the batch's
    stream); otherwise the library's own memory pool and copy stream serve
    them and uploads of queued TFs overlap earlier batches.  ``fail_alloc``
    (with ``torch_memory``): called with each request's size; True makes that
    allocation fail (fault tests).  ``debug_inject``: o2tpc_config.debug_inject
    (bit 0: the staged NeighboursFinder's waits run out with no copy in
    flight)."""

    def __init__(self, device: int = 0, bz: float = 0.5, vdrift: float = 2.58, flags: int = 0,
                 mem_budget: int = 0, max_inflight: int = 0, max_batch: int = 0, torch_memory: bool = False,
                 batch_full_clusters: int = 0, nf_hits_per_block: int = 0, sort_threads_per_row: int = 0,
                 graph_max_clusters: int = 0, graph_max_tfs: int = 0, nf_staged: bool = False,
                 tune_cache_path: str | None = None, fail_alloc=None, debug_inject: int = 0):
        self.cfg = o2tpc_config()
        self.cfg.device = device
        self.cfg.bz_tesla = bz
        self.cfg.vdrift_cm_us = vdrift
        self.cfg.flags = flags
        self.cfg.mem_budget = mem_budget
        self.cfg.max_inflight = max_inflight
        self.cfg.max_batch = max_batch
        self.cfg.batch_full_clusters = batch_full_clusters
        self.cfg.nf_hits_per_block = nf_hits_per_block
        self.cfg.sort_threads_per_row = sort_threads_per_row
        self.cfg.graph_max_clusters = graph_max_clusters
        self.cfg.graph_max_tfs = graph_max_tfs
        self.cfg.nf_staged = int(nf_staged)
        self._cache_path = tune_cache_path.encode() if tune_cache_path else None
        self.cfg.tune_cache_path = self._cache_path
        self.cfg.debug_inject = debug_inject
        self._keep = []
        import torch

        # the context runs on this stream (CUDA events for timing go on it)
        self.stream = torch.cuda.Stream(device=device)
        self.cfg.stream = self.stream.cuda_stream
        if torch_memory:
            dev = device
            st = self.stream

            def _alloc(nbytes, user):
                if fail_alloc is not None and fail_alloc(int(nbytes)):
                    return None
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                except Exception:
                    return None

            def _free(p, user):
                torch.cuda.caching_allocator_delete(p)

            self._keep = [ALLOC_FN(_alloc), FREE_FN(_free)]
            self.cfg.dev_alloc, self.cfg.dev_free = self._keep
        rc, self.ctx = o2tpc_create(self.cfg)
        if rc != O2TPC_OK:
            raise O2TPCError(rc, "o2tpc_create")
        self._pending = {}

    def submit(self, tf, location: int = O2TPC_LOC_HOST, arrays: dict | None = None, user_tag: int = 0,
               coll_time=None) -> int:
        t = make_tf(tf, location, arrays, user_tag, coll_time)
        rc, ticket = o2tpc_submit_tf(self.ctx, t)
        if rc != O2TPC_OK:
            raise O2TPCError(rc, "o2tpc_submit_tf")
        self._pending[ticket] = (tf, arrays, t)  # inputs are borrowed until polled
        return ticket

    def submit_many(self, tfs, location: int = O2TPC_LOC_HOST, arrays: list | None = None) -> list[int]:
        """Queues all ``tfs`` at once (they share a batch as far as the limits
        allow); ``arrays``: one dict per TF for device or pinned inputs."""
        arrays = arrays if arrays is not None else [None] * len(tfs)
        ts = [make_tf(tf, location, a) for tf, a in zip(tfs, arrays)]
        rc, tickets = o2tpc_submit_many(self.ctx, ts)
        if rc != O2TPC_OK:
            raise O2TPCError(rc, "o2tpc_submit_many")
        for tk, tf, a, t in zip(tickets, tfs, arrays, ts):
            self._pending[tk] = (tf, a, t)
        return tickets

    def poll(self, ticket: int, timeout_ms: int = -1, keep: bool = False):
        """Waits for ``ticket``; returns the result as a dict (None on timeout).
        ``keep``: do not release (stages stay readable) - call ``release``."""
        rc, res = o2tpc_poll(self.ctx, ticket, timeout_ms)
        if rc == O2TPC_PENDING:
            return None
        if rc != O2TPC_OK:
            raise O2TPCError(rc, "o2tpc_poll")
        out = result_to_dict(res.contents)
        if keep:
            out["_res"] = res
        else:
            o2tpc_result_release(self.ctx, res)
            self._pending.pop(ticket, None)
        return out

    def wait(self, ticket: int, timeout_ms: int = -1):
        """Waits for ``ticket`` and releases it without copying the arrays;
        returns status, track / cluster counts and the stats (None on
        timeout)."""
        rc, res = o2tpc_poll(self.ctx, ticket, timeout_ms)
        if rc == O2TPC_PENDING:
            return None
        if rc != O2TPC_OK:
            raise O2TPCError(rc, "o2tpc_poll")
        r = res.contents
        n = int(r.n_tracks)
        out = dict(status=int(r.status), n_tracks=n, n_cluster_refs=int(r.offsets[n]), ctf_bytes=int(r.ctf_bytes),
                   stats={k: (list(getattr(r.stats, k)) if k == "ms_stage" else getattr(r.stats, k))
                          for k, _ in o2tpc_stats._fields_})
        o2tpc_result_release(self.ctx, res)
        self._pending.pop(ticket, None)
        return out

    def release(self, ticket: int, result: dict) -> None:
        o2tpc_result_release(self.ctx, result["_res"])
        self._pending.pop(ticket, None)

    def tuning(self) -> dict:
        rc, t = o2tpc_get_tuning(self.ctx)
        if rc != O2TPC_OK:
            raise O2TPCError(rc, "o2tpc_get_tuning")
        return {"tuned": bool(t.tuned), "nf_hits_per_block": t.nf_hits_per_block, "nf_staged": bool(t.nf_staged),
                "sort_threads_per_row": t.sort_threads_per_row, "tuned_on_clusters": t.tuned_on_clusters,
                "nf_ms": list(t.nf_ms), "sort_ms": list(t.sort_ms)}

    def stage(self, ticket: int, name: str) -> np.ndarray:
        rc, need = o2tpc_get_stage(self.ctx, ticket, name, None, 0)
        if need == 0 and rc not in (O2TPC_OK, O2TPC_EINVAL):
            raise O2TPCError(rc, f"o2tpc_get_stage({name})")
        dt = np.float32 if name in ("tl_state", "st_in", "st_out") else np.int32
        buf = np.empty(max(need, 4) // 4, dtype=dt)
        rc, need = o2tpc_get_stage(self.ctx, ticket, name, buf.ctypes.data, buf.nbytes)
        if rc != O2TPC_OK:
            raise O2TPCError(rc, f"o2tpc_get_stage({name})")
        buf = buf[: need // 4]
        if name == "sorted_yz":
            buf = buf.reshape(-1, 2)
        elif name == "row_grid":
            buf = buf.reshape(-1, 8)
        elif name in ("tl_state", "st_in", "st_out"):
            buf = buf.reshape(-1, 21)
        elif name == "tl_hits":
            buf = buf.reshape(-1, 152)
        return buf

    def track(self, tf, **kw) -> dict:
        """Submit + poll; raises if the TF's own status is an error other than
        O2TPC_EINVAL (invalid cluster content, reported in the result)."""
        r = self.poll(self.submit(tf, **kw))
        if r["status"] not in (O2TPC_OK, O2TPC_EINVAL):
            raise O2TPCError(r["status"], "tracking")
        return r

    def close(self) -> None:
        if getattr(self, "ctx", None):
            rc = o2tpc_destroy(self.ctx)
            self.ctx = None
            if rc != O2TPC_OK:
                raise O2TPCError(rc, "o2tpc_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
