"""The tensor-core pair step (two partners, wide candidate masks: Gram matrix
of the candidates' same-sign / different-sign masks on tcgen05) against the
oracle, the closed forms of complete bipartite graphs and the POPC path of the
tuple kernel, per anchor and exact."""
from math import comb

import numpy as np
import pytest

import oracle
import sbc_synth

pytestmark = pytest.mark.gpu

TC_OFF = {"tc_min_words": -1}


@pytest.fixture(scope="module")
def sbc():
    import torch

    assert torch.cuda.is_available()
    torch.cuda.init()
    import paper_2605_03603_gb300 as m

    return m


def dense_faction_graph(m, n, density, seed, flip=0.05):
    rng = np.random.default_rng(seed)
    u, v = np.divmod(np.arange(m * n), n)
    keep = rng.random(m * n) < density
    lab_u = rng.choice([-1, 1], m)
    lab_v = rng.choice([-1, 1], n)
    s = (lab_u[u] * lab_v[v]).astype(np.int8)
    s[rng.random(m * n) < flip] *= -1
    return sbc_synth.from_edges(m, n, u[keep], v[keep], s[keep])


def priority_order(g):
    deg = np.diff(g.offsets)
    return np.lexsort((np.arange(g.n_u), deg)).tolist()


@pytest.mark.parametrize("p,q,density,seed", [(3, 3, 0.6, 17), (3, 4, 0.5, 18), (3, 6, 0.7, 19)])
def test_tc_per_anchor_equals_popc_path_and_oracle(sbc, p, q, density, seed):
    """Every anchor's share with the tensor-core step on equals its share with
    the step off (tuple kernel only), and a sample of anchors equals the
    oracle; the step must have taken anchors."""
    g = dense_faction_graph(900, 600, density, seed)
    with sbc.graph_from_synth(g) as h:
        on, st_on, per_on = sbc.sbc_count_ex(h, p, q, anchor_side=0, per_anchor=True)
        off, st_off, per_off = sbc.sbc_count_ex(h, p, q, anchor_side=0, per_anchor=True, tune=TC_OFF)
        other, _, _ = sbc.sbc_count_ex(h, p, q, anchor_side=1)
    assert st_on["tc_anchors"] > 0 and st_on["tc_tiles"] > 0
    assert st_off["tc_anchors"] == 0
    assert on == off == other
    assert per_on == per_off
    order = priority_order(g)
    sample = order[:8] + order[100:104] + order[300:302]
    _, want = oracle.count(g, p, q, side=0, per_anchor=True, anchors=sample)
    assert [per_on[a] for a in sample] == [want[a] for a in sample]
    assert sum(want[a] for a in sample) > 0


@pytest.mark.parametrize("tc_min_words", [1, 2, 4])
def test_tc_thresholds_exact(sbc, tc_min_words):
    """Other thresholds (down to one mask word) move anchors between the two
    paths without changing any anchor's share."""
    g = dense_faction_graph(700, 240, 0.55, 31)
    with sbc.graph_from_synth(g) as h:
        base, _, per_off = sbc.sbc_count_ex(h, 3, 3, anchor_side=0, per_anchor=True, tune=TC_OFF)
        got, st, per = sbc.sbc_count_ex(h, 3, 3, anchor_side=0, per_anchor=True,
                                         tune={"tc_min_words": tc_min_words})
    assert got == base and per == per_off
    assert st["tc_anchors"] > 0


def complete_factions_one_flip(m, n, seed):
    """K_{m,n} with planted two-faction signs and one edge flipped against its
    faction: switching-equivalent to all positive but one negative edge."""
    rng = np.random.default_rng(seed)
    u, v = np.divmod(np.arange(m * n, dtype=np.int64), n)
    lab_u = rng.choice([-1, 1], m)
    lab_v = rng.choice([-1, 1], n)
    s = (lab_u[u] * lab_v[v]).astype(np.int8)
    s[(m // 2) * n + n // 3] *= -1
    return sbc_synth.from_edges(m, n, u, v, s)


@pytest.mark.parametrize("q", [3, 5, 8])
def test_tc_large_common_neighbourhoods_closed_form(sbc, q):
    """K_{160,20000}: pairs of anchors' candidates share 20,000 positions, so
    Gram entries reach 2e4 (beyond fp16-sized partial sums) and binom(x, q)
    needs 64 to 128 bits; the count is the closed form
    binom(m,3) binom(n,q) - binom(m-1,2) binom(n-1,q-1)."""
    m, n = 160, 20000
    g = complete_factions_one_flip(m, n, q)
    want = comb(m, 3) * comb(n, q) - comb(m - 1, 2) * comb(n - 1, q - 1)
    with sbc.graph_from_synth(g) as h:
        got, st, per = sbc.sbc_count_ex(h, 3, q, anchor_side=0, per_anchor=True)
        off, _, per_off = sbc.sbc_count_ex(h, 3, q, anchor_side=0, per_anchor=True, tune=TC_OFF)
    assert st["tc_anchors"] > 0
    assert got == want
    assert off == want and per == per_off


def test_tc_batched_and_replayed(sbc):
    """Graphs with tensor-core anchors in a batch: each graph's count is its
    own (the epilogue attributes tiles to graphs), on the first run and on
    replays of the captured CUDA graph."""
    gs = [dense_faction_graph(500 + 40 * i, 300, 0.6, 40 + i) for i in range(3)]
    gs.append(sbc_synth.plain_small())
    hs = [sbc.graph_from_synth(g) for g in gs]
    try:
        want = [sbc.sbc_count_ex(h, 3, 3, tune=TC_OFF)[0] for h in hs]
        assert sbc.sbc_count_batch(hs, 3, 3) == want
        with sbc.Batch(hs, 3, 3) as b:
            for _ in range(3):
                assert b.run() == want
    finally:
        for h in hs:
            h.close()
