"""Pins for the CPU oracle (no GPU).

The oracle (`oracle.count`, a depth-first count over common neighbourhoods in
C) and the brute forces (`oracle.brute_count` in Python and
`oracle.brute_count_c` in C, the definition of Section 3) are checked against
facts that do not come from either: the butterflies of Figure 2, the worked
example of Figure 3, a hand-derived count on Figure 1(b), closed forms on
complete bipartite graphs up to (p,q) = (8,8), the (2,q) pair formula, exact
binomials and invariances.
Each pin is chosen so that a plausible slip (ties in the vertex priority, a
wrong sign relation, a dropped binomial term, a transposed side) fails it.
"""
import itertools
import random
from math import comb

import numpy as np
import pytest

import oracle
import sbc_synth
from golden_io import butterflies, expectations, graph


def complete(m, n, sign_fn=lambda u, v: 1):
    u, v = np.divmod(np.arange(m * n), n)
    s = np.array([sign_fn(a, b) for a, b in zip(u.tolist(), v.tolist())], dtype=np.int8)
    return sbc_synth.from_edges(m, n, u, v, s)


def transpose(g):
    u, v, s = g.edges()
    return sbc_synth.from_edges(g.n_v, g.n_u, v, u, s)


# --- Figure 2: butterfly parity --------------------------------------------

@pytest.mark.parametrize("panel", butterflies(), ids=lambda b: b[0])
def test_fig2_butterfly_parity(panel):
    _, s11, s12, s21, s22, balanced = panel
    assert oracle.butterfly_balanced(s11, s12, s21, s22) == balanced
    g = sbc_synth.from_edges(2, 2, [0, 0, 1, 1], [0, 1, 0, 1], [s11, s12, s21, s22])
    assert oracle.brute_count(g, 2, 2) == int(balanced)
    for side in (0, 1):
        assert oracle.count(g, 2, 2, side=side) == int(balanced)


# --- Figure 3: worked example ------------------------------------------------

def test_fig3_example_counts():
    g = graph("fig3_example.txt", 4, 4)
    # printed: balanced (3,3) = 0 (no triple has 3 common neighbours) for any
    # signs; check the all-positive and random signings
    rng = random.Random(3)
    for trial in range(20):
        signs = [1] * g.m if trial == 0 else [rng.choice((1, -1)) for _ in range(g.m)]
        h = graph("fig3_example.txt", 4, 4, signs)
        for side in (0, 1):
            assert oracle.count(h, 3, 3, side=side) == 0
        assert oracle.brute_count(h, 3, 3) == 0
    # the printed triple intersections have size 2, so with all edges positive
    # each of the three triples with u1 contributes binom(2,2) = 1, and
    # {u2,u3,u4} shares only v1: (3,2) = 3
    assert oracle.count(g, 3, 2, side=0) == 3
    # printed candidate set: u2, u3, u4 each share 3 neighbours with u1, so
    # with all edges positive the (2,3) count is 3 (one per pair (u1, ui));
    # other pairs share at most 2 neighbours
    assert oracle.count(g, 2, 3, side=0) == 3
    assert oracle.count(g, 2, 3, side=1) == 3


def test_fig3_per_anchor():
    g = graph("fig3_example.txt", 4, 4)
    # anchors are the lowest-priority vertex of their tuple; the (3,2) count of
    # 3 all comes from tuples containing u1 (degree 4) and two of u2..u4
    # (degree 3). The lowest-priority vertex of {u1,u2,u3} is u2 (degree 3,
    # id 1 < id 2), etc.; per-anchor values must add up to the total.
    total, per = oracle.count(g, 3, 2, side=0, per_anchor=True)
    assert total == 3 and sum(per) == 3
    # {u1,u2,u3} -> {v1,v2} and {u1,u2,u4} -> {v1,v3} are anchored at u2,
    # {u1,u3,u4} -> {v1,v4} at u3; u1 (degree 4) and u4 (highest id among
    # the degree-3 vertices) anchor none
    assert per == [0, 2, 1, 0]


# --- Figure 1(b): hand-derived count ----------------------------------------

def test_fig1b_hand_derived():
    g = graph("fig1b_k44.txt", 4, 4)
    for p, q, c in expectations("fig1b_k44.txt"):
        assert oracle.brute_count(g, p, q) == c
        assert oracle.count(g, p, q, side=0) == c
        assert oracle.count(g, p, q, side=1) == c


# --- closed forms on complete bipartite graphs ------------------------------

@pytest.mark.parametrize("m,n", [(3, 3), (4, 5), (6, 4), (7, 7)])
def test_complete_all_positive(m, n):
    g = complete(m, n)
    for p in range(2, min(m, 5) + 1):
        for q in range(2, min(n, 5) + 1):
            want = comb(m, p) * comb(n, q)
            assert oracle.count(g, p, q, side=0) == want
            assert oracle.count(g, p, q, side=1) == want
            if m * n <= 30:
                assert oracle.brute_count(g, p, q) == want


@pytest.mark.parametrize("m,n,seed", [(5, 4, 1), (6, 6, 2), (8, 5, 3)])
def test_complete_two_factions(m, n, seed):
    # planted factions without flips are switching-equivalent to all positive
    rng = random.Random(seed)
    lu = [rng.choice((1, -1)) for _ in range(m)]
    lv = [rng.choice((1, -1)) for _ in range(n)]
    g = complete(m, n, lambda u, v: lu[u] * lv[v])
    for p, q in [(2, 2), (3, 3), (2, 4), (4, 3)]:
        want = comb(m, p) * comb(n, q)
        assert oracle.count(g, p, q, side=0) == want
        assert oracle.count(g, p, q, side=1) == want
        assert oracle.brute_count(g, p, q) == want


@pytest.mark.parametrize("m,n,us,vs", [(4, 4, 0, 0), (5, 6, 2, 3), (6, 5, 5, 4)])
def test_complete_one_negative_edge(m, n, us, vs):
    # every biclique holding both u* and v* has a butterfly (u*, u', v*, v')
    # with exactly one negative edge; all others are balanced
    g = complete(m, n, lambda u, v: -1 if (u, v) == (us, vs) else 1)
    for p, q in [(2, 2), (3, 3), (2, 3), (3, 2), (4, 4)]:
        want = comb(m, p) * comb(n, q) - comb(m - 1, p - 1) * comb(n - 1, q - 1)
        assert oracle.count(g, p, q, side=0) == want
        assert oracle.count(g, p, q, side=1) == want
        assert oracle.brute_count(g, p, q) == want


# Signed closed forms up to (8,8). On K_{m,n} with all edges positive except
# chosen special rows x whose edges to a column set B_x are negative, a
# column set R is balanced with row set L when every butterfly has an even
# number of negative edges, i.e. when the rows' sign vectors on R agree up
# to one global flip. Group L's rows: T = its special rows. If L also holds
# an ordinary row (all +1 on R), every special row must be constant on R:
# R lies in one cell of V under membership in the B_x, x in T. If L = T, the
# membership vectors of R's columns must agree up to complement. Summing
# over T (binom(m - #specials, p - |T|) choices of the ordinary rows) gives
# the count.

def special_rows_graph(m, n, patterns):
    """K_{m,n}, rows listed in `patterns` (row -> set of columns) negative
    on their set."""
    return complete(m, n, lambda u, v: -1 if v in patterns.get(u, ()) else 1)


def special_rows_count(m, n, patterns, p, q):
    spec = sorted(patterns)
    total = 0
    for t in range(len(spec) + 1):
        for T in itertools.combinations(spec, t):
            if p - t < 0:
                continue
            cells = {}
            for v in range(n):
                key = tuple(v in patterns[x] for x in T)
                if p == t and key and key[0]:  # no ordinary row: up to complement
                    key = tuple(not b for b in key)
                cells[key] = cells.get(key, 0) + 1
            total += comb(m - len(spec), p - t) * sum(comb(c, q) for c in cells.values())
    return total


@pytest.mark.parametrize("p,q", [(5, 7), (8, 8), (6, 5), (7, 3), (4, 8), (2, 8)])
def test_signed_closed_forms_large_pq(p, q):
    m, n = 10, 11
    # one negative edge
    us, vs = m - 1, 4
    g1 = complete(m, n, lambda u, v: -1 if (u, v) == (us, vs) else 1)
    want1 = comb(m, p) * comb(n, q) - comb(m - 1, p - 1) * comb(n - 1, q - 1)
    # planted factions, no flips (switching-equivalent to all positive)
    rng = random.Random(p * 10 + q)
    lu = [rng.choice((1, -1)) for _ in range(m)]
    lv = [rng.choice((1, -1)) for _ in range(n)]
    g2 = complete(m, n, lambda u, v: lu[u] * lv[v])
    want2 = comb(m, p) * comb(n, q)
    # three special rows with the highest ids (the last members of every set
    # that holds them), patterns cutting V into up to 8 cells
    pats = {m - 3: {0, 1, 2, 3, 4, 5}, m - 2: {0, 1, 2, 6, 7}, m - 1: {0, 3, 6, 8, 9}}
    g3 = special_rows_graph(m, n, pats)
    want3 = special_rows_count(m, n, pats, p, q)
    for g, want in ((g1, want1), (g2, want2), (g3, want3)):
        for side in (0, 1):
            assert oracle.count(g, p, q, side=side) == want, (side, want)


def test_special_rows_formula_against_brute_force():
    """The special-rows formula itself, against the butterfly-by-butterfly
    definition on graphs small enough for it."""
    pats = {4: {0, 1, 2}, 5: {0, 3}, 6: {1, 3, 5}}
    g = special_rows_graph(7, 7, pats)
    for p, q in [(2, 2), (3, 3), (4, 2), (5, 3), (6, 2), (7, 2), (3, 5)]:
        assert oracle.brute_count_c(g, p, q) == special_rows_count(7, 7, pats, p, q)


# --- (2,q): balanced bicliques through a vertex pair --------------------------

def pair_formula(g, q):
    """p = 2: the two rows agree (same sign) on a set A and disagree on a set B
    of common neighbours; a column set is balanced iff it lies in A or in B."""
    nb = [dict(zip(g.cols[g.offsets[u]:g.offsets[u + 1]].tolist(),
                   g.signs[g.offsets[u]:g.offsets[u + 1]].tolist())) for u in range(g.n_u)]
    total = 0
    for a, b in itertools.combinations(range(g.n_u), 2):
        common = set(nb[a]) & set(nb[b])
        same = sum(1 for v in common if nb[a][v] == nb[b][v])
        total += comb(same, q) + comb(len(common) - same, q)
    return total


@pytest.mark.parametrize("seed", range(6))
def test_pair_formula(seed):
    g = sbc_synth.tiny_random(100 + seed, 12, 10, 0.6, 0.3)
    for q in (2, 3, 4):
        want = pair_formula(g, q)
        assert oracle.count(g, 2, q, side=0) == want
        assert oracle.count(g, 2, q, side=1) == want


# --- brute force on random tiny graphs ---------------------------------------

@pytest.mark.parametrize("seed", range(10))
def test_brute_force_c_equals_python(seed):
    rng = random.Random(1000 + seed)
    g = sbc_synth.tiny_random(500 + seed, rng.randint(2, 6), rng.randint(2, 6),
                              rng.uniform(0.5, 1.0), rng.uniform(0.0, 0.5))
    for p in range(2, 5):
        for q in range(2, 5):
            assert oracle.brute_count_c(g, p, q) == oracle.brute_count(g, p, q), (p, q)


def faction_graph(seed, n_u, n_v, density, flip):
    """Dense graph with planted two-faction signs and a few flipped edges, so
    that large balanced bicliques exist and the flips split their classes."""
    rng = random.Random(seed)
    lu = [rng.choice((1, -1)) for _ in range(n_u)]
    lv = [rng.choice((1, -1)) for _ in range(n_v)]
    uu, vv, ss = [], [], []
    for u in range(n_u):
        for v in range(n_v):
            if rng.random() < density:
                uu.append(u)
                vv.append(v)
                ss.append(lu[u] * lv[v] * (-1 if rng.random() < flip else 1))
    return sbc_synth.from_edges(n_u, n_v, uu, vv, ss)


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_large_pq_on_10x10(seed):
    """(p,q) up to (5,5) and (6,4) on 10 x 10 graphs, against the definition."""
    g = faction_graph(seed, 10, 10, 0.92, 0.06)
    for p, q in [(5, 5), (4, 5), (5, 3), (6, 4), (3, 6)]:
        want = oracle.brute_count_c(g, p, q)
        assert oracle.count(g, p, q, side=0) == want, (p, q)
        assert oracle.count(g, p, q, side=1) == want, (p, q)

@pytest.mark.parametrize("seed", range(40))
def test_brute_force_random_tiny(seed):
    rng = random.Random(seed)
    n_u, n_v = rng.randint(2, 7), rng.randint(2, 7)
    g = sbc_synth.tiny_random(seed, n_u, n_v, rng.uniform(0.5, 1.0), rng.uniform(0.0, 0.5))
    for p in range(2, 5):
        for q in range(2, 5):
            want = oracle.brute_count(g, p, q)
            assert oracle.count(g, p, q, side=0) == want, (p, q)
            assert oracle.count(g, p, q, side=1) == want, (p, q)


def test_degree_ties_count_once():
    # a regular graph: every vertex has the same degree, so the priority is
    # decided by ids alone; a tie rule that admits rho(w) >= rho(u) would count
    # tuples more than once
    g = complete(5, 5)
    assert oracle.count(g, 3, 3, side=0) == comb(5, 3) ** 2
    cyc_u, cyc_v = [], []
    for i in range(6):
        for d in range(3):
            cyc_u.append(i)
            cyc_v.append((i + d) % 6)
    g2 = sbc_synth.from_edges(6, 6, cyc_u, cyc_v, [1] * len(cyc_u))
    for p, q in [(2, 2), (2, 3), (3, 2), (3, 3)]:
        assert oracle.count(g2, p, q, side=0) == oracle.brute_count(g2, p, q)


# --- invariances --------------------------------------------------------------

def switched(g, side, x):
    u, v, s = g.edges()
    s = s.copy()
    s[(u if side == 0 else v) == x] *= -1
    return sbc_synth.from_edges(g.n_u, g.n_v, u, v, s)


@pytest.mark.parametrize("seed", range(3))
def test_invariances_small_chung_lu(seed):
    g = sbc_synth.chung_lu_signed(50 + seed, 60, 40, 600, 2.1, 2.1, 0.2)
    for p, q in [(3, 3), (2, 3), (3, 4)]:
        c = oracle.count(g, p, q, side=0)
        assert oracle.count(g, p, q, side=1) == c
        assert oracle.count(transpose(g), q, p, side=1) == c  # side swap
        assert oracle.count(switched(g, 0, 3), p, q) == c  # switching at u
        assert oracle.count(switched(g, 1, 5), p, q) == c  # switching at v
        neg = sbc_synth.from_edges(g.n_u, g.n_v, *g.edges()[:2], -g.edges()[2])
        assert oracle.count(neg, p, q) == c  # global negation
        pu = np.random.default_rng(seed).permutation(g.n_u)
        pv = np.random.default_rng(seed + 9).permutation(g.n_v)
        u, v, s = g.edges()
        relab = sbc_synth.from_edges(g.n_u, g.n_v, pu[u], pv[v], s)
        assert oracle.count(relab, p, q) == c  # relabelling


@pytest.mark.parametrize("seed", range(3))
def test_all_positive_equals_unsigned(seed):
    g = sbc_synth.tiny_random(200 + seed, 9, 9, 0.7, 0.0)
    for p, q in [(2, 2), (3, 3), (3, 2), (4, 3)]:
        assert oracle.count(g, p, q) == oracle.unsigned_count(g, p, q)


def test_empty_and_degenerate():
    g = sbc_synth.from_edges(5, 5, [], [], [])
    assert oracle.count(g, 3, 3) == 0
    g1 = sbc_synth.from_edges(1, 1, [0], [0], [1])
    assert oracle.count(g1, 2, 2) == 0
    star = sbc_synth.from_edges(1, 6, [0] * 6, list(range(6)), [1] * 6)
    assert oracle.count(star, 2, 2) == 0


# --- exact binomials -----------------------------------------------------------

def test_binomials_exact():
    for n in list(range(0, 40)) + [1000, 65535, 2**20 + 7, 2**31 - 1, 10**9]:
        for k in range(0, 9):
            want = comb(n, k)
            if want.bit_length() <= 128:
                assert oracle.binom(n, k) == want
            else:
                with pytest.raises(OverflowError):
                    oracle.binom(n, k)
    # beyond 64 bits, and right at the 128-bit edge
    assert oracle.binom(2**40, 3) == comb(2**40, 3)
    lo, hi = 8, 2**40  # largest n with binom(n, 8) < 2^128, by bisection
    while lo < hi:
        mid = (lo + hi + 1) // 2
        lo, hi = (mid, hi) if comb(mid, 8).bit_length() <= 128 else (lo, mid - 1)
    n = lo
    assert oracle.binom(n, 8) == comb(n, 8)
    with pytest.raises(OverflowError):
        oracle.binom(n + 1, 8)


def test_tuples_metric_matches_candidate_sets():
    # the enumerated (p-1)-subsets equal sum over anchors of binom(|C|, p-1);
    # on K_{m,n} every higher-priority vertex is a candidate
    m, n = 7, 5
    g = complete(m, n)
    _, tup = oracle.count(g, 3, 3, side=0, with_tuples=True)
    assert tup == sum(comb(m - 1 - i, 2) for i in range(m))


# --- the oracle's test options: anchor subsets and the subset cap ----------------

def _algorithm2_candidates(g, p, q):
    """|C(u)| of Algorithm 2 for every U-vertex u, straight from the
    definition: partners w with higher priority (degree, then id) sharing at
    least q neighbours with u (dense numpy, small graphs only)."""
    deg = np.diff(g.offsets)
    order = np.lexsort((np.arange(g.n_u), deg))
    rank = np.empty(g.n_u, np.int64)
    rank[order] = np.arange(g.n_u)
    a = np.zeros((g.n_u, g.n_v), np.int32)
    u, v, _ = g.edges()
    a[u, v] = 1
    common = a @ a.T
    higher = rank[None, :] > rank[:, None]
    return ((common >= q) & higher).sum(axis=1)


def test_anchor_subsets_partition_the_count():
    g = sbc_synth.plain_small()
    total, per = oracle.count(g, 3, 3, side=0, per_anchor=True)
    rng = np.random.default_rng(5)
    part = rng.integers(0, 3, g.n_u)
    sums = 0
    for k in range(3):
        sub = np.nonzero(part == k)[0]
        t, pk = oracle.count(g, 3, 3, side=0, per_anchor=True, anchors=sub)
        assert all(pk[a] == per[a] for a in sub)
        assert all(pk[a] == 0 for a in np.nonzero(part != k)[0])
        sums += t
    assert sums == total


def test_subset_cap_skips_exactly_the_large_anchors():
    g = sbc_synth.plain_small()
    p, q, cap = 3, 3, 40
    total, per = oracle.count(g, p, q, side=0, per_anchor=True)
    skipped = set()
    _, capped = oracle.count(g, p, q, side=0, per_anchor=True, max_subsets=cap,
                             skipped=skipped)
    ncand = _algorithm2_candidates(g, p, q)
    want = {int(a) for a in range(g.n_u) if comb(int(ncand[a]), p - 1) > cap}
    assert skipped == want and skipped
    assert all(capped[a] == per[a] for a in range(g.n_u) if a not in skipped)
    assert all(capped[a] == 0 for a in skipped)


# --- the pins catch planted mistakes -------------------------------------------

def _pins_pass(lib):
    """Run a cross-section of the pins above against one oracle library."""
    g = graph("fig1b_k44.txt", 4, 4)
    for p, q, c in expectations("fig1b_k44.txt"):
        for side in (0, 1):
            if oracle.count(g, p, q, side=side, lib=lib) != c:
                return False
    for m, n, us, vs in [(5, 6, 2, 3)]:
        h = complete(m, n, lambda u, v: -1 if (u, v) == (us, vs) else 1)
        for p, q in [(2, 2), (3, 3), (3, 2)]:
            want = comb(m, p) * comb(n, q) - comb(m - 1, p - 1) * comb(n - 1, q - 1)
            for side in (0, 1):
                if oracle.count(h, p, q, side=side, lib=lib) != want:
                    return False
    for seed in range(8):
        t = sbc_synth.tiny_random(seed, 6, 6, 0.8, 0.3)
        for p, q in [(2, 3), (3, 3), (3, 2)]:
            want = oracle.brute_count(t, p, q)
            for side in (0, 1):
                if oracle.count(t, p, q, side=side, lib=lib) != want:
                    return False
    pats = {7: {0, 1, 2, 3, 4, 5}, 8: {0, 1, 2, 6, 7}, 9: {0, 3, 6, 8, 9}}
    h = special_rows_graph(10, 11, pats)
    for p, q in [(6, 3), (8, 2)]:
        if oracle.count(h, p, q, side=0, lib=lib) != special_rows_count(10, 11, pats, p, q):
            return False
    t = faction_graph(3, 10, 10, 0.92, 0.06)
    if oracle.count(t, 5, 5, side=0, lib=lib) != oracle.brute_count_c(t, 5, 5):
        return False
    return True


def test_pins_pass_on_oracle():
    assert _pins_pass(None)


@pytest.mark.parametrize("mutant", range(1, 8))
def test_pins_catch_planted_mistakes(mutant, tmp_path):
    lib = oracle.mutant(mutant, str(tmp_path))
    assert not _pins_pass(lib)


def test_prepared_lists_count_the_same():
    """The prepared form (lists built once, counted many times, as the
    benchmark's CPU legs use it) gives the plain call's results."""
    g = sbc_synth.plain_small()
    rng = np.random.default_rng(3)
    for side in (0, 1):
        n_s = g.n_u if side == 0 else g.n_v
        sample = np.nonzero(rng.random(n_s) < 0.3)[0]
        with oracle.Prepared(g, side) as prep:
            for p, q in [(3, 3), (4, 3), (3, 4)]:
                want = oracle.count(g, p, q, side=side, per_anchor=True, with_tuples=True)
                assert prep.count(p, q, per_anchor=True, with_tuples=True) == want
                assert (prep.count(p, q, anchors=sample, with_tuples=True) ==
                        oracle.count(g, p, q, side=side, anchors=sample, with_tuples=True))
