"""sbc_count_csr_noalloc: counting for callers that cannot allocate device
memory (a fixed device-memory plan, a loop that must not enter the
allocator). Its result must equal sbc_count_csr's, exactly, call after call,
although every call reuses the same fixed scratch array; it must never reach
the allocator; and a call that fails for lack of scratch must leave the next
call (on another stream) exact.

This file is collected last (tests/test_zz_*) so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import sbc_synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch

    assert torch.cuda.is_available()
    torch.cuda.init()
    import paper_2605_03603_gb300 as m

    return m


def _c_count(lib, fn, g, p, q, device, torch):
    """Call a count entry point through the C ABI (ctypes), host or device inputs."""
    if device:
        off = torch.from_numpy(g.offsets).cuda()
        col = torch.from_numpy(g.cols).cuda()
        sgn = torch.from_numpy(g.signs).cuda()
        ptrs = (off.data_ptr(), col.data_ptr(), sgn.data_ptr())
        flags = lib.SBC_OFFS_I64 | lib.SBC_DEVICE_PTRS
        keep = (off, col, sgn)
    else:
        ptrs = (g.offsets.ctypes.data, g.cols.ctypes.data, g.signs.ctypes.data)
        flags = lib.SBC_OFFS_I64
        keep = (g,)
    out = lib.U128()
    rc = fn(g.n_u, g.n_v, g.m, ptrs[0], ptrs[1], ptrs[2], flags, p, q, ctypes.byref(out), None)
    torch.cuda.synchronize()
    del keep
    assert rc == 0, lib.sbc_last_error()
    return out.value()


def test_noalloc_equals_count_csr_on_repeated_calls(lib):
    import torch

    g = sbc_synth.plain_small()
    want = {pq: _c_count(lib, lib.lib.sbc_count_csr, g, *pq, False, torch)
            for pq in [(3, 3), (2, 4), (4, 3)]}
    for call in range(2):
        for pq, w in want.items():
            got_dev = _c_count(lib, lib.lib.sbc_count_csr_noalloc, g, *pq, True, torch)
            got_host = _c_count(lib, lib.lib.sbc_count_csr_noalloc, g, *pq, False, torch)
            assert got_dev == w, (call, pq)
            assert got_host == w, (call, pq)


def test_noalloc_other_graphs_and_limits(lib):
    import torch

    for seed in range(2):
        g = sbc_synth.chung_lu_signed(300 + seed, 900, 700, 9000, 2.2, 2.2, 0.2)
        want = _c_count(lib, lib.lib.sbc_count_csr, g, 3, 3, False, torch)
        assert _c_count(lib, lib.lib.sbc_count_csr_noalloc, g, 3, 3, True, torch) == want
    # sizes above the stated maximum are refused with SBC_E_INVAL and a message
    n = lib.SBC_NOALLOC_MAX_VERTICES + 1
    off = np.zeros(n + 1, dtype=np.int64)
    out = lib.U128()
    rc = lib.lib.sbc_count_csr_noalloc(n, 4, 0, off.ctypes.data, None, None, lib.SBC_OFFS_I64,
                                       3, 3, ctypes.byref(out), None)
    assert rc == 1
    assert "at most" in lib.sbc_last_error()


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


def test_noalloc_never_calls_the_allocator(lib):
    """With an allocator hook installed that counts its calls (and returns
    NULL, so any allocation would fail the call), the no-allocation entry
    point still counts exactly and the hook is never called."""
    import torch

    g = sbc_synth.plain_small()
    want = _c_count(lib, lib.lib.sbc_count_csr, g, 3, 3, False, torch)
    calls = {"alloc": 0, "free": 0}

    def _alloc(nbytes, stream, ctx):
        calls["alloc"] += 1
        return None

    def _free(ptr, nbytes, stream, ctx):
        calls["free"] += 1

    a_fn, f_fn = ALLOC_FN(_alloc), FREE_FN(_free)
    set_alloc = lib.lib.sbc_set_allocator
    set_alloc.restype = ctypes.c_int
    set_alloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert set_alloc(ctypes.cast(a_fn, ctypes.c_void_p), ctypes.cast(f_fn, ctypes.c_void_p), None) == 0
    try:
        for _ in range(2):
            assert _c_count(lib, lib.lib.sbc_count_csr_noalloc, g, 3, 3, True, torch) == want
            assert _c_count(lib, lib.lib.sbc_count_csr_noalloc, g, 3, 3, False, torch) == want
    finally:
        assert set_alloc(None, None, None) == 0
    assert calls == {"alloc": 0, "free": 0}


def test_noalloc_out_of_scratch_then_next_call_exact(lib):
    """K_{256,256} (65,536 edges, within the size limits) needs more than the
    fixed scratch (its 2-hop bucket area alone is far larger), so the call
    returns SBC_E_NOMEM after it has launched kernels; the next call, on
    another stream, still equals sbc_count_csr."""
    import torch

    n = 256
    uu, vv = np.divmod(np.arange(n * n, dtype=np.int64), n)
    big = sbc_synth.from_edges(n, n, uu, vv, np.ones(n * n, dtype=np.int8))
    off = np.ascontiguousarray(big.offsets, dtype=np.int64)
    out = lib.U128()
    rc = lib.lib.sbc_count_csr_noalloc(big.n_u, big.n_v, big.m, off.ctypes.data,
                                       big.cols.ctypes.data, big.signs.ctypes.data,
                                       lib.SBC_OFFS_I64, 3, 3, ctypes.byref(out), None)
    assert rc == 3, lib.sbc_last_error()  # SBC_E_NOMEM
    assert "fixed scratch" in lib.sbc_last_error()
    g = sbc_synth.plain_small()
    want = _c_count(lib, lib.lib.sbc_count_csr, g, 3, 3, False, torch)
    st = torch.cuda.Stream()
    for _ in range(2):
        o2 = lib.U128()
        rc = lib.lib.sbc_count_csr_noalloc(g.n_u, g.n_v, g.m, g.offsets.ctypes.data,
                                           g.cols.ctypes.data, g.signs.ctypes.data,
                                           lib.SBC_OFFS_I64, 3, 3, ctypes.byref(o2),
                                           ctypes.c_void_p(st.cuda_stream))
        assert rc == 0, lib.sbc_last_error()
        assert o2.value() == want
