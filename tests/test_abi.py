"""Host-side checks of the C ABI: the library builds, loads, exports every
function declared in include/pgabb.h, and rejects bad arguments before
touching the GPU.  No compute call is made here (no GPU needed)."""
import ctypes
import subprocess

import pytest

from paper_2209_04541_b300 import build, pgabb


def test_library_exports_every_header_symbol():
    lib = pgabb.load(register_torch_allocator=False)
    names = pgabb.header_functions()
    assert len(names) >= 19
    for name in names:
        assert hasattr(lib, name), f"{name} declared in pgabb.h but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_binding_covers_every_header_function():
    names = pgabb.header_functions()
    for name in names:
        assert callable(getattr(pgabb, name, None)), f"binding lacks {name}"


def test_built_for_sm103a():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert build.up_to_date()


def test_version_and_errors_without_gpu():
    lib = pgabb.load(register_torch_allocator=False)
    assert pgabb.pgb_version().startswith("pgabb-b300")
    n = ctypes.c_uint32()
    assert lib.pgb_graph_info(None, ctypes.byref(n), None) == pgabb.PGB_E_INVAL
    assert "NULL" in pgabb.pgb_last_error()
    out = ctypes.c_void_p()
    assert lib.pgb_partition(None, 4, 0, None, ctypes.byref(out)) == pgabb.PGB_E_INVAL
    assert lib.pgb_tc_run(None, None, None, ctypes.byref(out)) == pgabb.PGB_E_INVAL
    assert lib.pgb_graph_from_edges(None, None, 5, 10, 0, None, ctypes.byref(out)) == pgabb.PGB_E_INVAL
    assert lib.pgb_graph_from_edges(None, None, 0, 10, 7, None, ctypes.byref(out)) == pgabb.PGB_E_INVAL
    assert lib.pgb_tc_result_get(None, None, None, 0) == pgabb.PGB_E_INVAL
    assert lib.pgb_blocks_offload(None, None) == pgabb.PGB_E_INVAL
    u64, u32 = ctypes.c_uint64(), ctypes.c_uint32()
    assert lib.pgb_blocks_resident_bytes(None, 1, ctypes.byref(u64)) == pgabb.PGB_E_INVAL
    assert lib.pgb_tc_result_stream(None, ctypes.byref(u64), ctypes.byref(u32), None) == pgabb.PGB_E_INVAL
    assert lib.pgb_blocks_offload_columns(None, 0, None) == pgabb.PGB_E_INVAL
    assert lib.pgb_blocks_cache_budget(None, 1, 2, ctypes.byref(u64)) == pgabb.PGB_E_INVAL
    # freeing NULL handles is a no-op
    lib.pgb_graph_free(None)
    lib.pgb_blocks_free(None)
    lib.pgb_tc_result_free(None)


def test_opts_default():
    o = pgabb.pgb_tc_opts_default()
    assert o.mode == pgabb.PGB_MODE_PERSISTENT
    assert o.variant == pgabb.PGB_VAR_AUTO
    assert o.per_vertex == 1 and o.per_triple == 0 and o.use_graph == 0
    assert o.device_budget == 0
    assert ctypes.sizeof(pgabb.TcOpts) == 64
    assert ctypes.sizeof(pgabb.BlocksStats) == 64
    with pytest.raises(AttributeError):
        pgabb.pgb_tc_opts_default(bogus=1)


def test_allocator_pairing_checked():
    lib = pgabb.load(register_torch_allocator=False)
    fa = pgabb._ALLOC_FN(lambda size, stream, ctx: None)
    ff = ctypes.cast(None, pgabb._FREE_FN)
    assert lib.pgb_set_allocator(fa, ff, None) == pgabb.PGB_E_INVAL


def test_server_opts_and_admission_estimate():
    lib = pgabb.load(register_torch_allocator=False)
    o = pgabb.pgb_server_opts_default()
    assert o.mode == pgabb.PGB_SERVE_BATCHED and o.budget_bytes == 64 << 30
    assert o.max_inflight == 1 and o.per_vertex == 1 and o.max_batch_jobs == 256 and o.p == 8
    assert ctypes.sizeof(pgabb.ServerOpts) == 64 and ctypes.sizeof(pgabb.ServerInfo) == 64
    est = pgabb.pgb_server_job_bytes
    assert 0 < est(0, 0) < est(10, 10) < est(1000, 10) < est(1000, 100000)
    # bad arguments are refused before any device work
    bad = pgabb.pgb_server_opts_default(mode=7)
    out = ctypes.c_void_p()
    assert lib.pgb_server_create(ctypes.byref(bad), ctypes.byref(out)) == pgabb.PGB_E_INVAL
    jid = ctypes.c_uint64()
    assert lib.pgb_server_submit(None, None, None, 0, 0, 0, ctypes.byref(jid)) == pgabb.PGB_E_INVAL
    st = ctypes.c_int()
    assert lib.pgb_server_poll(None, 1, ctypes.byref(st)) == pgabb.PGB_E_INVAL
    lib.pgb_server_destroy(None)


@pytest.mark.parametrize("short", ["rowptr", "col", "perm", "total", "per_vertex"])
def test_noalloc_binding_rejects_short_arrays_without_calling_the_library(short, monkeypatch):
    """Arrays shorter than n and m require are refused in the binding, so a
    wrong n or m never turns into device reads or writes past an array."""
    import numpy as np

    def no_library():
        raise AssertionError("the library was reached")

    monkeypatch.setattr(pgabb, "load", no_library)
    n, m = 6, 8
    sizes = {"rowptr": n + 1, "col": m, "perm": n, "total": 1, "per_vertex": n}
    sizes[short] -= 1
    arrs = {k: np.zeros(v, dtype=np.uint64 if k in ("total", "per_vertex") else np.uint32)
            for k, v in sizes.items()}
    with pytest.raises(ValueError, match=short):
        pgabb.pgb_tc_count_oriented_noalloc(n, m, arrs["rowptr"], arrs["col"], arrs["perm"], arrs["total"],
                                            arrs["per_vertex"])


def test_hilbert_curve_and_block_order():
    """Host-only layout helpers: the Hilbert curve is a bijection of the
    grid onto [0, side^2) whose consecutive cells are neighbours, with the
    2 x 2 curve (0,0), (0,1), (1,1), (1,0); block orders list each upper
    block once."""
    import numpy as np

    assert [pgabb.pgb_hilbert_index(2, x, y) for x, y in ((0, 0), (0, 1), (1, 1), (1, 0))] == [0, 1, 2, 3]
    for side in (4, 8, 64):
        cells = {}
        for x in range(side):
            for y in range(side):
                cells[pgabb.pgb_hilbert_index(side, x, y)] = (x, y)
        assert sorted(cells) == list(range(side * side))
        for d in range(side * side - 1):
            (x0, y0), (x1, y1) = cells[d], cells[d + 1]
            assert abs(x0 - x1) + abs(y0 - y1) == 1
    for p in (1, 5, 16, 33):
        rm = pgabb.pgb_block_order(p, pgabb.PGB_LAYOUT_ROWMAJOR)
        hb = pgabb.pgb_block_order(p, pgabb.PGB_LAYOUT_HILBERT)
        want = [(i, j) for i in range(p) for j in range(i, p)]
        assert [tuple(x) for x in rm.tolist()] == want
        assert sorted(tuple(x) for x in hb.tolist()) == want
        keys = [pgabb.pgb_hilbert_index(1 << max(p - 1, 1).bit_length(), j, i) for i, j in hb.tolist()]
        assert keys == sorted(keys)
    with pytest.raises(pgabb.PgbError):
        pgabb.pgb_hilbert_index(6, 0, 0)
