"""The CTA-wide 2-hop kernel's bucketed strategy (§4.3's candidate step for
anchors with many wedges): wedges scattered by hash class, a second scatter
at exact class offsets when one partner fills its class, and sub-class
windows when a class has more distinct partners than one hash table holds.
Each is driven on small graphs and compared per anchor with the default
strategy and with the oracle."""
import numpy as np
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


def faction_signs(rng, n_u, n_v, u, v, flip):
    lab_u = rng.choice([-1, 1], n_u)
    lab_v = rng.choice([-1, 1], n_v)
    s = (lab_u[u] * lab_v[v]).astype(np.int8)
    s[rng.random(u.shape[0]) < flip] *= -1
    return s


def twin_anchor_graph(d=4000, covers=2, per_cover=3, others=24, deg_other=300, seed=3):
    """U vertex 0 has d neighbours. U vertex 1 has the same d and one more, so
    it ranks above vertex 0 and shares all d positions with it: one hash class
    receives a third of anchor 0's wedges. `covers` times over, the d positions
    are split among `per_cover` further U vertices, each padded with vertices
    of its own to degree d + 1 (so they rank above vertex 0 too, and every
    position has covers + 1 partners of anchor 0). The remaining U vertices
    have deg_other neighbours among the d and rank below all of these."""
    rng = np.random.default_rng(seed)
    uu = [np.zeros(d, np.int64), np.ones(d + 1, np.int64)]
    vv = [np.arange(d), np.arange(d + 1)]
    n_v, nxt = d + 1, 2
    for _ in range(covers):
        for part in np.array_split(rng.permutation(d), per_cover):
            own = d + 1 - part.shape[0]
            uu.append(np.full(d + 1, nxt, np.int64))
            vv.append(np.concatenate([np.sort(part), n_v + np.arange(own)]))
            n_v += own
            nxt += 1
    for i in range(others):
        uu.append(np.full(deg_other, nxt + i, np.int64))
        vv.append(np.sort(rng.choice(d, deg_other, replace=False)))
    u, v = np.concatenate(uu), np.concatenate(vv).astype(np.int64)
    n_u = nxt + others
    return sbc_synth.from_edges(n_u, n_v, u, v, faction_signs(rng, n_u, n_v, u, v, 0.05))


def test_skewed_class_takes_the_second_scatter(sbc):
    """A third of anchor 0's 12,000 wedges go to one partner: its class
    overflows the 1.5x capacity, the wedges are scattered again at exact class
    offsets, and every anchor's share equals the oracle's."""
    g = twin_anchor_graph()
    with sbc.graph_from_synth(g) as h:
        for p, q in [(3, 3), (3, 4), (4, 3)]:
            got, st, per = sbc.sbc_count_ex(h, p, q, anchor_side=0, per_anchor=True, check=True)
            want_total, want = oracle.count(g, p, q, side=0, per_anchor=True)
            assert st["twohop_anchors"][3] >= 1, st["twohop_anchors"]
            assert got == want_total and per == want
            assert want[0] > 0


def windows_forced(monkeypatch):
    # every anchor above 32 wedges is bucketed and every table has 32 slots:
    # classes with more distinct partners go to sub-class windows
    monkeypatch.setenv("SBC_TWOHOP_WINDOW", "32")
    monkeypatch.setenv("SBC_HASH_SLOTS_CAP", "32")


@pytest.mark.parametrize("side,p,q", [(0, 3, 3), (0, 4, 3), (0, 3, 5), (1, 3, 3), (1, 4, 3)])
def test_bucketed_and_subclass_windows_per_anchor(sbc, monkeypatch, side, p, q):
    g = sbc_synth.plain_small()
    with sbc.graph_from_synth(g) as h:
        base, _, per_base = sbc.sbc_count_ex(h, p, q, anchor_side=side, per_anchor=True)
        windows_forced(monkeypatch)
        got, st, per = sbc.sbc_count_ex(h, p, q, anchor_side=side, per_anchor=True,
                                        check=True, tune={"small_wedges": 1})
    assert st["twohop_anchors"][1] + st["twohop_anchors"][3] > 0
    assert st["twohop_split_classes"] > 0
    assert got == base == oracle.count(g, p, q, side=side)
    assert per == per_base


def test_bucketed_windows_on_dense_factions(sbc, monkeypatch):
    """Dense anchors: many wedges per partner (classes far above their
    expected size) and the tensor-core step fed from bucketed masks."""
    rng = np.random.default_rng(11)
    m, n = 700, 260
    u, v = np.divmod(np.arange(m * n, dtype=np.int64), n)
    keep = rng.random(m * n) < 0.5
    u, v = u[keep], v[keep]
    g = sbc_synth.from_edges(m, n, u, v, faction_signs(rng, m, n, u, v, 0.05))
    with sbc.graph_from_synth(g) as h:
        base, _, per_base = sbc.sbc_count_ex(h, 3, 3, anchor_side=0, per_anchor=True)
        windows_forced(monkeypatch)
        got, st, per = sbc.sbc_count_ex(h, 3, 3, anchor_side=0, per_anchor=True, check=True,
                                        tune={"small_wedges": 1})
    assert st["tc_anchors"] > 0
    assert got == base and per == per_base
    order = np.lexsort((np.arange(m), np.diff(g.offsets))).tolist()
    sample = order[:6] + order[300:303]
    _, want = oracle.count(g, 3, 3, side=0, per_anchor=True, anchors=sample)
    assert [per[a] for a in sample] == [want[a] for a in sample]
