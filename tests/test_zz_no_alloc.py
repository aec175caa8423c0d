"""The allocation-free binning/sort entry point (o2tpc_sort_tf_static).

It exists for callers that cannot allocate device memory while they run (a
framework owning every device buffer, a fixed memory plan, code that must
not synchronise the device through an allocation); its scratch memory is
static device storage inside the library.  Here it is checked through the
C-ABI against the regular allocating path, whose stages are bit-exact
against the oracle: the same sort order, sorted coordinates, row grid and
cell starts, on two different Time Frames in a row (the second call reuses
the static scratch left behind by the first).
"""
import numpy as np
import pytest

import oracle
from paper_2106_03636_gb300 import o2tpc, synth

pytestmark = pytest.mark.gpu

ROWS = 36 * 152


def static_sort(tf):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    if tf.fmt == synth.FMT_FIXED:
        arrays = {"packed": torch.from_numpy(np.ascontiguousarray(tf.packed)).to(dev)}
    else:
        arrays = {k: torch.from_numpy(np.ascontiguousarray(getattr(tf, k))).to(dev) for k in ("sector", "row", "y", "z")}
    n = tf.n
    so = torch.full((max(n, 1),), -7, dtype=torch.int32, device=dev)
    yz = torch.full((max(n, 1), 2), -7, dtype=torch.int32, device=dev)
    grid = torch.full((ROWS, 8), -7, dtype=torch.int32, device=dev)
    cap = n // 4 + 46 * ROWS + 2
    cs = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    t = o2tpc.make_tf(tf, o2tpc.O2TPC_LOC_DEVICE, arrays)
    torch.cuda.synchronize()
    rc = o2tpc.o2tpc_sort_tf_static(t, tf.vdrift, so.data_ptr(), yz.data_ptr(), grid.data_ptr(), cs.data_ptr(), cap,
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == o2tpc.O2TPC_OK, o2tpc.o2tpc_strerror(rc)
    g = grid.cpu().numpy()
    ncells = int(g[-1, 2] + g[-1, 3] * g[-1, 4])
    return so.cpu().numpy()[:n], yz.cpu().numpy()[:n], g, cs.cpu().numpy()[: ncells + 1]


def regular_sort(tfs):
    out = []
    with o2tpc.Tracker(flags=o2tpc.O2TPC_FLAG_KEEP_STAGES) as trk:
        for tf in tfs:
            ticket = trk.submit(tf)
            res = trk.poll(ticket, keep=True)
            assert res["status"] == 0
            out.append(tuple(trk.stage(ticket, k) for k in ("sorted_orig", "sorted_yz", "row_grid", "cell_start")))
            trk.release(ticket, res)
    return out


def test_static_sort_equals_regular_path_twice():
    tfs = [synth.single_sector(seed=31, ntracks=400),
           synth.full_tpc_1ms(seed=32, n_coll=1, ntracks=1200, fmt=synth.FMT_FIXED)]
    assert all(0 < tf.n <= o2tpc.O2TPC_STATIC_MAX_CLUSTERS for tf in tfs)
    ref = regular_sort(tfs)
    for tf, (so_r, yz_r, g_r, cs_r) in zip(tfs, ref):
        so, yz, g, cs = static_sort(tf)
        assert np.array_equal(so, so_r)
        assert np.array_equal(yz, yz_r)
        assert np.array_equal(g, g_r)
        assert np.array_equal(cs, cs_r)


def test_static_sort_equals_oracle_and_allocates_nothing():
    """The same stages straight against the oracle; a repeated call changes
    neither the device's free memory nor PyTorch's allocated bytes."""
    torch = pytest.importorskip("torch")
    tf = synth.full_tpc_1ms(seed=33, n_coll=1, ntracks=1000, fmt=synth.FMT_FIXED)
    so, yz, g, cs = static_sort(tf)  # first call: module and symbol set-up
    o = oracle.run(tf, fields=["sorted_orig", "sorted_y", "sorted_z", "row_start", "row_count", "cell_start"])
    assert np.array_equal(so, o["sorted_orig"])
    assert np.array_equal(yz[:, 0], o["sorted_y"]) and np.array_equal(yz[:, 1], o["sorted_z"])
    assert np.array_equal(g[:, 0], o["row_start"][:-1]) and np.array_equal(g[:, 1], o["row_count"])
    assert np.array_equal(cs, o["cell_start"])
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    again = static_sort(tf)  # buffers of the same sizes come back from the caching allocator
    torch.cuda.synchronize()
    free1, alloc1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    assert np.array_equal(again[0], so)
    assert free1 == free0 and alloc1 == alloc0


def test_static_sort_empty_tf():
    """n = 0: every row count zero and the cell-start total zero."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    t = o2tpc.o2tpc_tf()
    t.n = 0
    t.format = o2tpc.O2TPC_FMT_FIXED
    t.location = o2tpc.O2TPC_LOC_DEVICE
    grid = torch.full((ROWS, 8), -7, dtype=torch.int32, device=dev)
    cap = 46 * ROWS + 2
    cs = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    rc = o2tpc.o2tpc_sort_tf_static(t, 2.58, None, None, grid.data_ptr(), cs.data_ptr(), cap,
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == o2tpc.O2TPC_OK, o2tpc.o2tpc_strerror(rc)
    g = grid.cpu().numpy()
    assert np.all(g[:, 1] == 0) and np.all(g[:, 0] == 0)
    ncells = int(g[-1, 2] + g[-1, 3] * g[-1, 4])
    c = cs.cpu().numpy()
    assert c[ncells] == 0 and np.all(c[: ncells + 1] == 0)


def test_static_sort_rejects_oversize_and_host_input():
    big = o2tpc.o2tpc_tf()
    big.n = o2tpc.O2TPC_STATIC_MAX_CLUSTERS + 1
    big.format = o2tpc.O2TPC_FMT_FIXED
    big.location = o2tpc.O2TPC_LOC_DEVICE
    assert o2tpc.o2tpc_sort_tf_static(big, 2.58, None, None, None, None, 0, None) == o2tpc.O2TPC_ETOOBIG
    host = o2tpc.o2tpc_tf()
    host.n = 10
    host.format = o2tpc.O2TPC_FMT_FIXED
    host.location = o2tpc.O2TPC_LOC_HOST
    assert o2tpc.o2tpc_sort_tf_static(host, 2.58, None, None, None, None, 0, None) == o2tpc.O2TPC_EINVAL
