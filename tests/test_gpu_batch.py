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


def test_autotuner_choice_counts_exactly(sbc):
    """The autotuner returns parameters from its search space; a batch planned
    with them, and single counts with them, stay exact."""
    gs = mixed_graphs(30, 11) + [sbc_synth.plain_small()]
    want = [oracle.count(g, 3, 3, side=0) for g in gs]
    hs = [sbc.graph_from_synth(g) for g in gs]
    try:
        t = sbc.sbc_autotune(hs, 3, 3, reps=2)
        assert t["split_per_warp"] in (0, 1, 2, 4, 8, 16)
        assert t["small_wedges"] in (0, 16, 32, 48, 64)
        assert t["pos_node_cost"] in (0, 2, 4, 6, 10, 16, 64, 1 << 20)
        assert t["ms"] > 0
        with sbc.Batch(hs, 3, 3, tune=t) as b:
            assert b.run() == want
            assert b.run() == want
        assert [sbc.sbc_count_ex(h, 3, 3, tune=t)[0] for h in hs] == want
        # a single graph is a batch of one
        t1 = sbc.sbc_autotune([hs[-1]], 4, 4, reps=1)
        assert sbc.sbc_count_ex(hs[-1], 4, 4, tune=t1)[0] == oracle.count(gs[-1], 4, 4, side=0)
    finally:
        for h in hs:
            h.close()


@pytest.mark.parametrize("tune", [
    {"small_wedges": 64, "pos_node_cost": 2, "split_per_warp": 16},
    {"small_wedges": 32, "pos_node_cost": 1 << 20, "split_per_warp": 1},
    {"small_wedges": 1, "pos_node_cost": 1, "split_per_warp": 64},
])
def test_extreme_launch_parameters_exact(sbc, tune):
    g = sbc_synth.plain_small()
    with sbc.graph_from_synth(g) as h:
        for p, q in [(3, 3), (4, 4), (2, 3), (4, 3)]:
            want = oracle.count(g, p, q, side=0)
            for side in (0, 1):
                assert sbc.sbc_count_ex(h, p, q, anchor_side=side, tune=tune)[0] == want


def test_launch_parameters_out_of_range_rejected(sbc):
    g = sbc_synth.plain_small()
    with sbc.graph_from_synth(g) as h:
        for bad in [{"small_wedges": 65}, {"split_per_warp": 65}, {"pos_node_cost": -1},
                    {"small_wedges": -2}]:
            with pytest.raises(sbc.SbcError) as e:
                sbc.sbc_count_ex(h, 3, 3, tune=bad)
            assert e.value.status == 1  # SBC_E_INVAL
    with pytest.raises(sbc.SbcError):
        sbc.sbc_autotune([], 3, 3)


@pytest.mark.parametrize("index", [4829, 7100])
def test_batch_recipe_graphs_exact(sbc, index):
    """Two graphs of the 10,000-graph batch recipe (about 2.4e5 and 4.9e5
    edges) whose counts once came out a few bicliques short: alone, in a
    small batch and with every 2-hop tier threshold, against the oracle."""
    g = sbc_synth.batch_graph(4, index)
    want = oracle.count(g, 3, 3, side=0)
    with sbc.graph_from_synth(g) as h:
        assert sbc.sbc_count(h, 3, 3) == want
        for sw in (1, 16, 64):
            assert sbc.sbc_count_ex(h, 3, 3, tune={"small_wedges": sw})[0] == want
        other = sbc.graph_from_synth(sbc_synth.batch_graph(4, index + 1))
        try:
            assert sbc.sbc_count_batch([h, other], 3, 3)[0] == want
        finally:
            other.close()


def test_two_hop_tiers_agree_on_batch_recipe(sbc):
    """Per-graph counts of 300 graphs from the batch recipe's generator
    (edges up to 2e5) are the same whichever 2-hop kernel takes the anchors
    (CTA per anchor for all, or the warp kernel up to its 64-wedge cap),
    alone and batched; small ones also against the oracle."""
    gs = sbc_synth.batch_graphs(4, 300, 500, 200_000)
    hs = [sbc.graph_from_synth(g) for g in gs]
    try:
        cta = [sbc.sbc_count_ex(h, 3, 3, tune={"small_wedges": 1})[0] for h in hs]
        warp = [sbc.sbc_count_ex(h, 3, 3, tune={"small_wedges": 64})[0] for h in hs]
        assert warp == cta
        assert sbc.sbc_count_batch(hs, 3, 3) == cta
        for i in range(0, 300, 60):
            if gs[i].m <= 20_000:
                assert cta[i] == oracle.count(gs[i], 3, 3, side=0)
    finally:
        for h in hs:
            h.close()
