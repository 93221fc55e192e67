"""Failure paths of the counting library, driven from the host (no GPU fault):
an allocator that runs dry, counts that need more than 128 bits, and 2-hop
hash tables made to overflow. Each must return its status code, leave no
device memory behind and leave the library usable."""
import ctypes
import os

import numpy as np
import pytest

import sbc_synth

pytestmark = pytest.mark.gpu

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


@pytest.fixture(scope="module")
def sbc():
    import torch

    assert torch.cuda.is_available()
    torch.cuda.init()
    import paper_2605_03603_gb300 as m

    f = m.lib.sbc_set_allocator
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return m


class TorchAllocator:
    """Device memory from torch's caching allocator through the library's
    allocator hook; the call numbered `fail_at` (1-based) returns NULL."""

    def __init__(self, fail_at=0):
        import torch

        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        self._a = ALLOC_FN(self._alloc)
        self._f = FREE_FN(self._free)

    def _alloc(self, nbytes, stream, ctx):
        self.calls += 1
        if self.fail_at and self.calls == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(max(int(nbytes), 1))
        self.live[p] = nbytes
        return p

    def _free(self, ptr, nbytes, stream, ctx):
        self.torch.cuda.synchronize()
        self.live.pop(int(ptr))
        self.torch.cuda.caching_allocator_delete(int(ptr))

    def __enter__(self):
        assert self.sbc.lib.sbc_set_allocator(ctypes.cast(self._a, ctypes.c_void_p),
                                              ctypes.cast(self._f, ctypes.c_void_p), None) == 0
        return self

    def __exit__(self, *exc):
        assert self.sbc.lib.sbc_set_allocator(None, None, None) == 0


def test_allocator_null_gives_nomem_and_frees_everything(sbc):
    """A count whose k-th device allocation fails returns SBC_E_NOMEM for every
    k, every block allocated before the failure is freed, and the next count
    is exact."""
    TorchAllocator.sbc = sbc
    g = sbc_synth.plain_small()
    with sbc.graph_from_synth(g) as h:
        want = {pq: sbc.sbc_count(h, *pq) for pq in [(3, 3), (4, 3)]}
        for side in (0, 1):  # build both orientations outside the hook
            sbc.sbc_count_ex(h, 3, 3, anchor_side=side)
        with TorchAllocator() as probe:
            assert sbc.sbc_count(h, 3, 3) == want[(3, 3)]
        n = probe.calls
        assert n > 3 and not probe.live
        for k in range(1, n + 1):
            with TorchAllocator(fail_at=k) as a:
                with pytest.raises(sbc.SbcError) as e:
                    sbc.sbc_count(h, 3, 3)
            assert e.value.status == 3, (k, str(e.value))  # SBC_E_NOMEM
            assert "allocator hook returned NULL" in str(e.value)
            assert not a.live, (k, a.live)
        for pq, w in want.items():
            assert sbc.sbc_count(h, *pq) == w


def complete_bipartite(copies, n_u, n_v):
    """`copies` disjoint all-positive K_{n_u, n_v}."""
    uu, vv = [], []
    for c in range(copies):
        u, v = np.divmod(np.arange(n_u * n_v, dtype=np.int64), n_v)
        uu.append(u + c * n_u)
        vv.append(v + c * n_v)
    u, v = np.concatenate(uu), np.concatenate(vv)
    return sbc_synth.from_edges(copies * n_u, copies * n_v, u, v, np.ones(u.shape[0], np.int8))


def test_overflow_of_one_binomial(sbc):
    """K_{2,600000}: the balanced (2,8) count is binom(600000, 8) > 2^128."""
    g = complete_bipartite(1, 2, 600_000)
    with sbc.graph_from_synth(g) as h:
        with pytest.raises(sbc.SbcError) as e:
            sbc.sbc_count(h, 2, 8)
        assert e.value.status == 8  # SBC_E_OVERFLOW
        assert sbc.sbc_count(h, 2, 2) == 600_000 * 599_999 // 2


def test_overflow_of_the_sum(sbc):
    """Two disjoint K_{2,240000}: each (2,8) term, binom(240000, 8), is about
    0.8 * 2^128 and fits; their sum does not, and must be reported, alone and
    batched."""
    from math import comb

    assert comb(240_000, 8) < 2**128 < 2 * comb(240_000, 8)
    one = complete_bipartite(1, 2, 240_000)
    two = complete_bipartite(2, 2, 240_000)
    with sbc.graph_from_synth(one) as h1, sbc.graph_from_synth(two) as h2:
        assert sbc.sbc_count(h1, 2, 8) == comb(240_000, 8)
        with pytest.raises(sbc.SbcError) as e:
            sbc.sbc_count(h2, 2, 8)
        assert e.value.status == 8
        # batched: each graph's own count is what must fit
        assert sbc.sbc_count_batch([h1, h1], 2, 8) == [comb(240_000, 8)] * 2
        with pytest.raises(sbc.SbcError) as e:
            sbc.sbc_count_batch([h1, h2], 2, 8)
        assert e.value.status == 8
        assert sbc.sbc_count(h2, 2, 3) == 2 * comb(240_000, 3)


def test_hash_table_overflow_reported(sbc, monkeypatch):
    """With the 2-hop tables capped at 32 slots (a host-side test override),
    anchors with more distinct partners overflow their table; the kernels
    report it and the count fails with SBC_E_CUDA. Without the cap the same
    graph counts exactly again."""
    g = sbc_synth.plain_small()
    with sbc.graph_from_synth(g) as h:
        want = sbc.sbc_count(h, 3, 3)
        monkeypatch.setenv("SBC_HASH_SLOTS_CAP", "32")
        for sw in (1, 512):  # CTA tier for every anchor, then the warp tier too
            with pytest.raises(sbc.SbcError) as e:
                sbc.sbc_count_ex(h, 3, 3, tune={"small_wedges": sw})
            assert e.value.status == 4  # SBC_E_CUDA
            assert "2-hop" in str(e.value)
        monkeypatch.delenv("SBC_HASH_SLOTS_CAP")
        assert sbc.sbc_count(h, 3, 3) == want
