"""Host side of the dynamic count (no GPU): the local graph H(u, v) that
sbc_edge_local_graph builds. An update of edge (u, v) must change the oracle's
balanced (p,q) count by the oracle's count of the complete (p-1, q-1)
subgraphs of H (its balanced count with every sign positive): checked for
insertions, deletions and sign changes on random and faction graphs, plus
H's layout on a hand-made case and the entry point's argument checks."""
import numpy as np
import pytest

import oracle
import sbc_synth

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def sbc():
    import paper_2605_03603_gb300 as m

    return m


def edge_dict(g):
    u, v, s = g.edges()
    return {(int(a), int(b)): int(c) for a, b, c in zip(u.tolist(), v.tolist(), s.tolist())}


def from_dict(n_u, n_v, d):
    keys = sorted(d)
    u = np.array([k[0] for k in keys], dtype=np.int64)
    v = np.array([k[1] for k in keys], dtype=np.int64)
    s = np.array([d[k] for k in keys], dtype=np.int8)
    return sbc_synth.from_edges(n_u, n_v, u, v, s)


def local_count(sbc, g, u, v, sign, p, q):
    n_l, n_r, off, col = sbc.edge_local_graph(g.n_u, g.n_v, g.offsets, g.cols, g.signs, u, v, sign)
    h = sbc_synth.SignedBipartite(n_l, n_r, off, col, np.ones(col.shape[0], dtype=np.int8))
    return oracle.count(h, p - 1, q - 1, side=0)


def random_graph(rng, m, n, density, factions):
    u, v = np.divmod(np.arange(m * n, dtype=np.int64), n)
    keep = rng.random(m * n) < density
    u, v = u[keep], v[keep]
    if factions:
        s = (rng.choice([-1, 1], m)[u] * rng.choice([-1, 1], n)[v]).astype(np.int8)
        s[rng.random(u.shape[0]) < 0.08] *= -1
    else:
        s = rng.choice([-1, 1], u.shape[0]).astype(np.int8)
    return sbc_synth.from_edges(m, n, u, v, s)


@pytest.mark.parametrize("p,q", [(3, 3), (3, 4), (4, 3), (4, 4)])
def test_updates_change_the_count_by_the_local_count(sbc, p, q):
    rng = np.random.default_rng(100 + 10 * p + q)
    for trial in range(6):
        m, n = int(rng.integers(8, 16)), int(rng.integers(8, 16))
        g = random_graph(rng, m, n, rng.uniform(0.5, 0.9), factions=trial % 2 == 0)
        e = edge_dict(g)
        base = oracle.count(g, p, q)
        # insertion of an absent pair, with either sign
        absent = [(a, b) for a in range(m) for b in range(n) if (a, b) not in e]
        if absent:
            a, b = absent[int(rng.integers(len(absent)))]
            for s in (1, -1):
                after = oracle.count(from_dict(m, n, {**e, (a, b): s}), p, q)
                assert after - base == local_count(sbc, g, a, b, s, p, q), (trial, a, b, s)
        # deletion and sign change of present edges
        present = list(e)
        for k in rng.choice(len(present), size=min(3, len(present)), replace=False):
            a, b = present[int(k)]
            s = e[(a, b)]
            rest = {x: y for x, y in e.items() if x != (a, b)}
            assert base - oracle.count(from_dict(m, n, rest), p, q) == local_count(sbc, g, a, b, s, p, q)
            flipped = oracle.count(from_dict(m, n, {**e, (a, b): -s}), p, q)
            assert flipped - base == (local_count(sbc, g, a, b, -s, p, q) -
                                      local_count(sbc, g, a, b, s, p, q))


def test_updates_at_a_high_degree_vertex(sbc):
    """u adjacent to most of V and its partners of low degree: the local graph
    is assembled by lookups into Gamma(u) rather than merges."""
    rng = np.random.default_rng(77)
    m, n = 30, 220
    d = {}
    for b in range(n):
        if rng.random() < 0.9:
            d[(0, b)] = int(rng.choice([-1, 1]))
    for a in range(1, m):
        for b in rng.choice(n, size=int(rng.integers(3, 12)), replace=False).tolist():
            d[(a, b)] = int(rng.choice([-1, 1]))
    for b in range(0, n, 7):  # a few columns shared by many rows
        for a in range(1, m, 2):
            d[(a, b)] = d.get((a, b), 1)
    g = from_dict(m, n, d)
    for p, q in [(3, 3), (3, 4), (4, 3)]:
        base = oracle.count(g, p, q)
        present = [k for k in d if k[0] == 0]
        for a, b in present[:6]:
            s = d[(a, b)]
            rest = {x: y for x, y in d.items() if x != (a, b)}
            assert base - oracle.count(from_dict(m, n, rest), p, q) == local_count(sbc, g, a, b, s, p, q)
        absent = [b for b in range(n) if (0, b) not in d]
        for b in absent[:4]:
            for s in (1, -1):
                after = oracle.count(from_dict(m, n, {**d, (0, b): s}), p, q)
                assert after - base == local_count(sbc, g, 0, b, s, p, q)


def test_local_graph_layout(sbc):
    """u = 0 with neighbours {0, 1, 2}; v = 1 with neighbours {0, 1, 3};
    rows are Gamma(v) - {u} = (1, 3), columns Gamma(u) - {v} = (0, 2)."""
    edges = {(0, 0): 1, (0, 1): -1, (0, 2): 1,
             (1, 0): -1, (1, 1): 1, (1, 2): 1,   # w = 1: sign products decide
             (3, 1): 1, (3, 2): -1,              # w = 3: only column 2 is shared
             (2, 0): 1}                          # not adjacent to v: no row
    g = from_dict(4, 3, edges)
    n_l, n_r, off, col = sbc.edge_local_graph(g.n_u, g.n_v, g.offsets, g.cols, g.signs, 0, 1, -1)
    assert (n_l, n_r) == (2, 2)
    # (w, x) kept when s(u,v) s(u,x) s(w,v) s(w,x) = +1:
    # w = 1: x = 0: (-1)(1)(1)(-1) = 1 keep; x = 2: (-1)(1)(1)(1) = -1 drop
    # w = 3: x = 2: (-1)(1)(1)(-1) = 1 keep
    assert off.tolist() == [0, 1, 2] and col.tolist() == [0, 1]


def test_local_graph_rejects_bad_arguments(sbc):
    g = sbc_synth.plain_small()
    args = (g.n_u, g.n_v, g.offsets, g.cols, g.signs)
    with pytest.raises(sbc.SbcError) as e:
        sbc.edge_local_graph(*args, g.n_u, 0, 1)
    assert e.value.status == 1
    with pytest.raises(sbc.SbcError) as e:
        sbc.edge_local_graph(*args, 0, 0, 2)
    assert e.value.status == 1
    bad = g.signs.copy()
    bad[0] = 0
    with pytest.raises(sbc.SbcError) as e:
        sbc.edge_local_graph(g.n_u, g.n_v, g.offsets, g.cols, bad, 0, 0, 1)
    assert e.value.status == 2
