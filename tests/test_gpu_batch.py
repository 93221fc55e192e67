"""Batched counting (sbc_count_batch, sbc_batch_*) vs per-graph counts and the
oracle, exact."""
import random

import pytest

import oracle
import sbc_synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbc():
    import torch

    assert torch.cuda.is_available()
    torch.cuda.init()
    import paper_2605_03603_gb300 as m

    return m


def mixed_graphs(n, seed):
    """Graphs of uneven sizes and shapes; some prefer anchoring on U, some on V."""
    rng = random.Random(seed)
    out = []
    for i in range(n):
        n_u, n_v = rng.randint(5, 400), rng.randint(5, 400)
        m = min(rng.randint(10, 4000), n_u * n_v // 2)
        out.append(sbc_synth.chung_lu_signed(9000 + 17 * seed + i, n_u, n_v, m,
                                             rng.uniform(1.9, 2.6), rng.uniform(1.9, 2.6),
                                             rng.uniform(0.0, 0.3)))
    out.append(sbc_synth.from_edges(7, 9, [], [], []))  # an empty graph
    return out


@pytest.mark.parametrize("p,q", [(3, 3), (2, 2), (4, 4), (3, 4), (4, 2)])
def test_batch_equals_oracle(sbc, p, q):
    gs = mixed_graphs(40, p * 10 + q)
    want = [oracle.count(g, p, q, side=0) for g in gs]
    hs = [sbc.graph_from_synth(g) for g in gs]
    try:
        sides = {sbc.sbc_graph_info(h)["wedges_anchor_u"] <= sbc.sbc_graph_info(h)["wedges_anchor_v"]
                 for h in hs}
        assert len(sides) == 2  # both anchor sides occur in the batch
        got = sbc.sbc_count_batch(hs, p, q)
        assert got == want
        assert [sbc.sbc_count(h, p, q) for h in hs] == want
    finally:
        for h in hs:
            h.close()


def test_planned_batch_replays(sbc):
    gs = mixed_graphs(30, 7) + [sbc_synth.plain_small()]
    want = [oracle.count(g, 3, 3, side=0) for g in gs]
    hs = [sbc.graph_from_synth(g) for g in gs]
    try:
        with sbc.Batch(hs, 3, 3) as b:
            for _ in range(3):
                assert b.run() == want
        with sbc.Batch(hs, 3, 4) as b:
            w34 = [oracle.count(g, 3, 4, side=0) for g in gs]
            assert b.run() == w34
            assert b.run() == w34
    finally:
        for h in hs:
            h.close()


def test_empty_batches(sbc):
    assert sbc.sbc_count_batch([], 3, 3) == []
    gs = [sbc_synth.from_edges(3, 3, [], [], []), sbc_synth.from_edges(1, 1, [0], [0], [1])]
    hs = [sbc.graph_from_synth(g) for g in gs]
    try:
        assert sbc.sbc_count_batch(hs, 2, 2) == [0, 0]
        with sbc.Batch(hs, 2, 2) as b:
            assert b.run() == [0, 0]
    finally:
        for h in hs:
            h.close()
