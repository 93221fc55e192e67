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
        assert t["small_wedges"] in (0, 32, 64, 128, 256, 512)
        assert t["pos_node_cost"] in (0, 2, 4, 6, 10, 16, 64, 1 << 20)
        assert t["tc_min_words"] in (0, -1, 3, 5, 9, 17)
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
    {"small_wedges": 512, "pos_node_cost": 2, "split_per_warp": 16},
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
        for bad in [{"small_wedges": 513}, {"split_per_warp": 65}, {"pos_node_cost": -1},
                    {"small_wedges": -2}]:
            with pytest.raises(sbc.SbcError) as e:
                sbc.sbc_count_ex(h, 3, 3, tune=bad)
            assert e.value.status == 1  # SBC_E_INVAL
    with pytest.raises(sbc.SbcError):
        sbc.sbc_autotune([], 3, 3)


def _side(sbc, h):
    info = sbc.sbc_graph_info(h)
    return 0 if info["wedges_anchor_u"] <= info["wedges_anchor_v"] else 1


@pytest.mark.parametrize("index", [4829, 7100])
def test_batch_recipe_graphs_exact(sbc, index):
    """Two graphs of the 10,000-graph batch recipe (about 2.4e5 and 4.9e5
    edges) whose counts once came out a few bicliques short on the
    warp-per-anchor 2-hop tier: per anchor against the oracle with the tier
    threshold forced to 1 (every anchor on the CTA tier), 64, 256 and 512
    wedges, with the mask self-check on; alone and in a small batch."""
    g = sbc_synth.batch_graph(4, index)
    with sbc.graph_from_synth(g) as h:
        side = _side(sbc, h)
        want, want_per = oracle.count(g, 3, 3, side=side, per_anchor=True)
        assert sbc.sbc_count(h, 3, 3) == want
        for sw in (1, 64, 256, 512):
            got, _, per = sbc.sbc_count_ex(h, 3, 3, anchor_side=side, per_anchor=True,
                                            tune={"small_wedges": sw}, check=True)
            assert got == want, sw
            assert per == want_per, sw
        other = sbc.graph_from_synth(sbc_synth.batch_graph(4, index + 1))
        try:
            assert sbc.sbc_count_batch([h, other], 3, 3)[0] == want
        finally:
            other.close()


def test_two_hop_tiers_per_anchor_on_batch_recipe(sbc):
    """300 graphs from the batch recipe's generator (edges up to 5e4): per
    anchor against the oracle with the warp tier threshold at 64, 256 and 512
    wedges (self-check on), and batched."""
    gs = sbc_synth.batch_graphs(4, 300, 500, 50_000)
    hs = [sbc.graph_from_synth(g) for g in gs]
    try:
        want = []
        for g, h in zip(gs, hs):
            side = _side(sbc, h)
            c, per = oracle.count(g, 3, 3, side=side, per_anchor=True)
            want.append(c)
            for sw in (64, 256, 512):
                got, _, gp = sbc.sbc_count_ex(h, 3, 3, anchor_side=side, per_anchor=True,
                                               tune={"small_wedges": sw}, check=True)
                assert got == c and gp == per, (g.name if hasattr(g, "name") else None, sw)
        assert sbc.sbc_count_batch(hs, 3, 3) == want
    finally:
        for h in hs:
            h.close()


def test_batch_recipe_all_graphs_plain_equals_batched(sbc):
    """All 10,000 graphs of the batch recipe (7.2e8 edges, in chunks of 1,000):
    plain per-graph counts with the warp tier at its 512-wedge default and the
    mask self-check on equal the batched counts of each chunk. This is the
    workload on which the warp tier once lost candidate-mask bits."""
    for c0 in range(0, 10_000, 1000):
        gs = sbc_synth.batch_graphs(4, 1000, start=c0)
        hs = [sbc.graph_from_synth(g) for g in gs]
        del gs
        try:
            plain = [sbc.sbc_count_ex(h, 3, 3, check=True)[0] for h in hs]
            assert sbc.sbc_count_batch(hs, 3, 3) == plain, c0
        finally:
            for h in hs:
                h.close()


def test_autotune_cache_reuses_the_tuning(sbc, tmp_path):
    """The per-GPU tuning cache: the first call searches and stores, the
    second finds the same key and returns the stored parameters without
    running; a batch planned with them counts exactly; another (p, q) is a
    different key."""
    gs = mixed_graphs(20, 21)
    want = [oracle.count(g, 3, 3, side=0) for g in gs]
    hs = [sbc.graph_from_synth(g) for g in gs]
    path = tmp_path / "tune_cache.txt"
    try:
        t1 = sbc.sbc_autotune(hs, 3, 3, reps=1, cache=path)
        assert t1["from_cache"] is False and path.exists()
        t2 = sbc.sbc_autotune(hs, 3, 3, reps=1, cache=path)
        assert t2["from_cache"] is True
        for k in ("small_wedges", "pos_node_cost", "split_per_warp", "tc_min_words"):
            assert t1[k] == t2[k]
        with sbc.Batch(hs, 3, 3, tune=t2) as b:
            assert b.run() == want
        t3 = sbc.sbc_autotune(hs, 4, 3, reps=1, cache=path)
        assert t3["from_cache"] is False
        assert len(path.read_text().splitlines()) == 2
    finally:
        for h in hs:
            h.close()
