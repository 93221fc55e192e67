"""Dynamic counts on the GPU (sbc_dyn_*): after every insertion, deletion or
sign change the maintained count equals the oracle's count of the current
graph, and invalid updates leave the handle unchanged."""
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


def edge_dict(g):
    u, v, s = g.edges()
    return {(int(a), int(b)): int(c) for a, b, c in zip(u.tolist(), v.tolist(), s.tolist())}


def from_dict(n_u, n_v, d):
    keys = sorted(d)
    u = np.array([k[0] for k in keys], dtype=np.int64)
    v = np.array([k[1] for k in keys], dtype=np.int64)
    s = np.array([d[k] for k in keys], dtype=np.int8)
    return sbc_synth.from_edges(n_u, n_v, u, v, s)


def faction_graph(rng, m, n, density):
    u, v = np.divmod(np.arange(m * n, dtype=np.int64), n)
    keep = rng.random(m * n) < density
    u, v = u[keep], v[keep]
    s = (rng.choice([-1, 1], m)[u] * rng.choice([-1, 1], n)[v]).astype(np.int8)
    s[rng.random(u.shape[0]) < 0.08] *= -1
    return sbc_synth.from_edges(m, n, u, v, s)


@pytest.mark.parametrize("p,q", [(3, 3), (4, 3), (3, 5)])
def test_random_updates_equal_recounts(sbc, p, q):
    rng = np.random.default_rng(500 + 10 * p + q)
    m, n = 40, 36
    g = faction_graph(rng, m, n, 0.45)
    e = edge_dict(g)
    with sbc.Dynamic.from_synth(g, p, q) as d:
        assert d.count() == oracle.count(g, p, q)
        for step in range(30):
            kind = int(rng.integers(3))
            if kind == 0:
                while True:
                    a, b = int(rng.integers(m)), int(rng.integers(n))
                    if (a, b) not in e:
                        break
                s = int(rng.choice([-1, 1]))
                got = d.insert(a, b, s)
                e[(a, b)] = s
            else:
                keys = list(e)
                a, b = keys[int(rng.integers(len(keys)))]
                if kind == 1:
                    got = d.delete(a, b)
                    del e[(a, b)]
                else:
                    got = d.set_sign(a, b, -e[(a, b)])
                    e[(a, b)] = -e[(a, b)]
            assert got == oracle.count(from_dict(m, n, e), p, q), (step, kind, a, b)
        assert d.count() == got and d.edges() == len(e)


def test_updates_at_hub_edges_of_the_benchmark_graph(sbc):
    """Edges at the highest-degree vertices of the 20k-edge graph: large local
    graphs (hundreds of rows and columns)."""
    g = sbc_synth.plain_small()
    e = edge_dict(g)
    deg_u = np.diff(g.offsets)
    deg_v = np.bincount(g.cols, minlength=g.n_v)
    hubs_u = np.argsort(-deg_u)[:3].tolist()
    hubs_v = np.argsort(-deg_v)[:3].tolist()
    with sbc.Dynamic.from_synth(g, 3, 3) as d:
        for a in hubs_u:
            for b in hubs_v:
                if (a, b) in e:
                    got = d.set_sign(a, b, -e[(a, b)])
                    e[(a, b)] = -e[(a, b)]
                else:
                    got = d.insert(a, b, 1)
                    e[(a, b)] = 1
                assert got == oracle.count(from_dict(g.n_u, g.n_v, e), 3, 3), (a, b)
        a, b = hubs_u[0], hubs_v[0]
        got = d.delete(a, b)
        del e[(a, b)]
        assert got == oracle.count(from_dict(g.n_u, g.n_v, e), 3, 3)


def test_invalid_updates_leave_the_count(sbc):
    rng = np.random.default_rng(9)
    g = faction_graph(rng, 12, 10, 0.5)
    e = edge_dict(g)
    a, b = next(iter(e))
    absent = next((x, y) for x in range(12) for y in range(10) if (x, y) not in e)
    with pytest.raises(sbc.SbcError) as err:
        sbc.Dynamic.from_synth(g, 2, 3)
    assert err.value.status == 1
    with sbc.Dynamic.from_synth(g, 3, 3) as d:
        c0, m0 = d.count(), d.edges()
        for call in (lambda: d.insert(a, b, 1), lambda: d.delete(*absent),
                     lambda: d.set_sign(*absent, 1), lambda: d.insert(*absent, 0),
                     lambda: d.insert(12, 0, 1)):
            with pytest.raises(sbc.SbcError) as err:
                call()
            assert err.value.status == 1
        assert (d.count(), d.edges()) == (c0, m0) == (oracle.count(g, 3, 3), len(e))
