"""sbc_count_csr_noalloc: counting for callers that cannot allocate device
memory (a fixed device-memory plan, a loop that must not enter the
allocator). Its result must equal sbc_count_csr's, exactly, call after call,
although every call reuses the same fixed scratch array.

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
