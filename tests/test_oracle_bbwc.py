"""The wedge-centric counter (BBWC, Algorithm 1, Section 4.2) as a second CPU
counter, independent of the oracle (its own C library, no shared code): it
must equal the definition by brute force on tiny graphs, the closed forms of
complete bipartite graphs, and the oracle on graphs too large for brute
force; and every planted mistake of the oracle must disagree with it
somewhere, so that it cross-checks the oracle on its own."""
from math import comb

import numpy as np
import pytest

import oracle
import sbc_synth
from test_oracle import faction_graph, special_rows_graph


def random_tiny(rng, factions):
    m, n = int(rng.integers(2, 12)), int(rng.integers(2, 12))
    u, v = np.divmod(np.arange(m * n, dtype=np.int64), n)
    keep = rng.random(m * n) < rng.uniform(0.3, 0.95)
    u, v = u[keep], v[keep]
    if factions:
        s = (rng.choice([-1, 1], m)[u] * rng.choice([-1, 1], n)[v]).astype(np.int8)
        s[rng.random(u.shape[0]) < 0.1] *= -1
    else:
        s = rng.choice([-1, 1], u.shape[0]).astype(np.int8)
    return sbc_synth.from_edges(m, n, u, v, s)


def test_bbwc_equals_the_definition_on_tiny_graphs():
    rng = np.random.default_rng(2024)
    checked = 0
    for trial in range(60):
        g = random_tiny(rng, factions=trial % 2 == 1)
        for p in (2, 3, 4):
            for q in (2, 3, 4):
                want = oracle.brute_count_c(g, p, q)
                for side in (0, 1):
                    assert oracle.bbwc_count(g, p, q, side=side) == want, (trial, p, q, side)
                    checked += 1
    assert checked == 60 * 9 * 2


def complete(m, n, sign):
    u, v = np.divmod(np.arange(m * n, dtype=np.int64), n)
    s = np.array([sign(a, b) for a, b in zip(u.tolist(), v.tolist())], dtype=np.int8)
    return sbc_synth.from_edges(m, n, u, v, s)


@pytest.mark.parametrize("p,q", [(2, 2), (3, 3), (3, 5), (5, 2), (4, 4)])
def test_bbwc_closed_forms(p, q):
    m, n = 7, 9
    lab_u = [1, -1, 1, 1, -1, -1, 1]
    lab_v = [-1, 1, 1, -1, 1, -1, 1, 1, -1]
    # all positive, and planted factions (switching-equivalent to all positive)
    for sign in (lambda a, b: 1, lambda a, b: lab_u[a] * lab_v[b]):
        g = complete(m, n, sign)
        for side in (0, 1):
            assert oracle.bbwc_count(g, p, q, side=side) == comb(m, p) * comb(n, q)
    # one negative edge: every biclique holding both its ends is unbalanced
    g = complete(m, n, lambda a, b: -1 if (a, b) == (3, 4) else 1)
    want = comb(m, p) * comb(n, q) - comb(m - 1, p - 1) * comb(n - 1, q - 1)
    for side in (0, 1):
        assert oracle.bbwc_count(g, p, q, side=side) == want


def test_bbwc_equals_the_oracle_on_larger_graphs():
    """Graphs beyond brute force: the 20k-edge benchmark graph (anchors on V,
    where the wedges stay few) and small graphs of the batch recipe."""
    g = sbc_synth.plain_small()
    for p, q in [(3, 3), (4, 3)]:
        assert oracle.bbwc_count(g, p, q, side=1) == oracle.count(g, p, q)
    checked = 0
    for i in range(60):
        b = sbc_synth.batch_graph(4, i, 500, 20000)
        if max(np.diff(b.offsets).max(), np.bincount(b.cols, minlength=b.n_v).max()) > 80:
            continue
        for side in (0, 1):
            assert oracle.bbwc_count(b, 3, 3, side=side) == oracle.count(b, 3, 3), (i, side)
        for p, q in [(4, 3), (3, 4)]:
            assert oracle.bbwc_count(b, p, q, side=0) == oracle.count(b, p, q), (i, p, q)
        checked += 1
    assert checked >= 15


def _mutant_disagrees(lib) -> bool:
    """Whether the oracle library `lib` differs from BBWC on some case of a
    fixed set of graphs and sizes."""
    rng = np.random.default_rng(7)
    cases = [(random_tiny(rng, factions=k % 2 == 1), p, q)
             for k in range(12) for p, q in [(2, 3), (3, 3), (3, 2), (4, 3)]]
    cases.append((faction_graph(3, 10, 10, 0.92, 0.06), 5, 5))
    pats = {7: {0, 1, 2, 3, 4, 5}, 8: {0, 1, 2, 6, 7}, 9: {0, 3, 6, 8, 9}}
    special = special_rows_graph(10, 11, pats)
    cases += [(special, 6, 3), (special, 8, 2)]
    for g, p, q in cases:
        for side in (0, 1):
            if oracle.count(g, p, q, side=side, lib=lib) != oracle.bbwc_count(g, p, q, side=side):
                return True
    return False


def test_oracle_agrees_with_bbwc_on_the_cross_check_set():
    assert not _mutant_disagrees(None)


@pytest.mark.parametrize("mutant", range(1, 8))
def test_bbwc_catches_each_planted_oracle_mistake(mutant, tmp_path):
    assert _mutant_disagrees(oracle.mutant(mutant, str(tmp_path)))
