"""CUDA path vs the CPU oracle, bit-exact (integer counts).

Inputs are seeded synthetic graphs from sbc_synth; expected values come only
from the oracle (Algorithm 2 in plain C) or from closed forms.
"""
import random
from math import comb

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


def gpu_count(sbc, g, p, q, side=-1, **kw):
    with sbc.graph_from_synth(g, **kw) as h:
        c, st, _ = sbc.sbc_count_ex(h, p, q, anchor_side=side)
        return c


def complete(m, n, sign_fn=lambda u, v: 1):
    u, v = np.divmod(np.arange(m * n), n)
    s = np.array([sign_fn(a, b) for a, b in zip(u.tolist(), v.tolist())], dtype=np.int8)
    return sbc_synth.from_edges(m, n, u, v, s)


# ---------------------------------------------------------------- tiny graphs

@pytest.mark.parametrize("seed", range(12))
def test_tiny_random_all_pq(sbc, seed):
    rng = random.Random(seed)
    g = sbc_synth.tiny_random(seed, rng.randint(2, 9), rng.randint(2, 9),
                              rng.uniform(0.4, 1.0), rng.uniform(0.0, 0.5))
    with sbc.graph_from_synth(g) as h:
        for p in range(2, 6):
            for q in range(2, 6):
                want = oracle.count(g, p, q, side=0)
                for side in (0, 1):
                    got, _, _ = sbc.sbc_count_ex(h, p, q, anchor_side=side)
                    assert got == want, (p, q, side)


def test_fig1b_and_complete_closed_forms(sbc):
    from golden_io import expectations, graph

    g = graph("fig1b_k44.txt", 4, 4)
    for p, q, c in expectations("fig1b_k44.txt"):
        assert gpu_count(sbc, g, p, q, 0) == c
        assert gpu_count(sbc, g, p, q, 1) == c
    for m, n in [(5, 7), (9, 6)]:
        k = complete(m, n)
        for p, q in [(2, 2), (3, 3), (4, 2), (3, 5)]:
            assert gpu_count(sbc, k, p, q) == comb(m, p) * comb(n, q)
        one = complete(m, n, lambda u, v: -1 if (u, v) == (1, 2) else 1)
        for p, q in [(2, 2), (3, 3), (2, 4)]:
            want = comb(m, p) * comb(n, q) - comb(m - 1, p - 1) * comb(n - 1, q - 1)
            assert gpu_count(sbc, one, p, q) == want


# ---------------------------------------------------------------- small workload

@pytest.fixture(scope="module")
def small():
    return sbc_synth.plain_small()


@pytest.mark.parametrize("side", [0, 1])
def test_small_33_total_per_anchor_and_tuples(sbc, small, side):
    want, per, tuples = oracle.count(small, 3, 3, side=side, per_anchor=True, with_tuples=True)
    with sbc.graph_from_synth(small) as h:
        got, st, pa = sbc.sbc_count_ex(h, 3, 3, anchor_side=side, per_anchor=True,
                                       paper_tuples=True)
    assert got == want
    assert pa == per
    assert st["anchor_tuples"] == tuples
    assert st["anchor_side"] == side


@pytest.mark.parametrize("p,q", [(2, 2), (2, 3), (3, 2), (4, 4), (3, 4), (4, 3), (2, 5), (5, 5)])
def test_small_other_pq(sbc, small, p, q):
    want = oracle.count(small, p, q, side=0)
    with sbc.graph_from_synth(small) as h:
        for side in (-1, 0, 1):
            got, st, _ = sbc.sbc_count_ex(h, p, q, anchor_side=side)
            assert got == want, (p, q, side)


@pytest.mark.parametrize("seed", range(4))
def test_random_chung_lu(sbc, seed):
    rng = random.Random(seed)
    n_u, n_v = rng.randint(300, 3000), rng.randint(300, 3000)
    m = rng.randint(3000, 30000)
    g = sbc_synth.chung_lu_signed(1000 + seed, n_u, n_v, m, rng.uniform(1.9, 2.5),
                                  rng.uniform(1.9, 2.5), rng.uniform(0.0, 0.3))
    for p, q in [(3, 3), (2, 4), (4, 3)]:
        want, tup = oracle.count(g, p, q, side=0, with_tuples=True)
        with sbc.graph_from_synth(g) as h:
            got, st, _ = sbc.sbc_count_ex(h, p, q, anchor_side=0, paper_tuples=True)
            assert got == want
            assert st["anchor_tuples"] == tup
            got2, _, _ = sbc.sbc_count_ex(h, p, q, anchor_side=1)
            assert got2 == want


# ---------------------------------------------------------------- input forms

def test_input_forms_agree(sbc, small):
    import torch

    want = oracle.count(small, 3, 3)
    assert gpu_count(sbc, small, 3, 3) == want
    assert gpu_count(sbc, small, 3, 3, device=True) == want
    assert gpu_count(sbc, small, 3, 3, sign_bits=True) == want
    assert gpu_count(sbc, small, 3, 3, device=True, sign_bits=True) == want
    # int32 offsets, shuffled rows
    rng = np.random.default_rng(5)
    cols = small.cols.copy()
    signs = small.signs.copy()
    for u in range(small.n_u):
        a, b = small.offsets[u], small.offsets[u + 1]
        perm = rng.permutation(b - a) + a
        cols[a:b] = small.cols[perm]
        signs[a:b] = small.signs[perm]
    with sbc.sbc_graph_create(small.n_u, small.n_v, small.offsets.astype(np.int32), cols,
                              signs) as h:
        assert sbc.sbc_count(h, 3, 3) == want
    assert sbc.sbc_count_csr(small.n_u, small.n_v, small.offsets, small.cols, small.signs,
                             3, 3) == want
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with sbc.graph_from_synth(small, stream=s) as h:
            assert sbc.sbc_count(h, 3, 3, stream=s) == want


# ---------------------------------------------------------------- edge cases

def test_empty_and_degenerate(sbc):
    e = sbc_synth.from_edges(10, 7, [], [], [])
    assert gpu_count(sbc, e, 3, 3) == 0
    z = sbc_synth.from_edges(0, 5, [], [], [])
    assert gpu_count(sbc, z, 2, 2) == 0
    one = sbc_synth.from_edges(1, 1, [0], [0], [-1])
    assert gpu_count(sbc, one, 2, 2) == 0
    star = sbc_synth.from_edges(1, 50, [0] * 50, list(range(50)), [1] * 50)
    assert gpu_count(sbc, star, 2, 2) == 0
    assert gpu_count(sbc, complete(2, 2), 2, 2) == 1


def test_bad_inputs_rejected(sbc):
    off = np.array([0, 2, 3], dtype=np.int64)
    ok_cols = np.array([0, 1, 1], dtype=np.int32)
    ok_signs = np.array([1, -1, 1], dtype=np.int8)
    with pytest.raises(sbc.SbcError) as e:
        sbc.sbc_graph_create(2, 2, off, np.array([0, 0, 1], dtype=np.int32), ok_signs)
    assert e.value.status == 2  # duplicate edge
    with pytest.raises(sbc.SbcError) as e:
        sbc.sbc_graph_create(2, 2, off, np.array([0, 5, 1], dtype=np.int32), ok_signs)
    assert e.value.status == 2  # column out of range
    with pytest.raises(sbc.SbcError) as e:
        sbc.sbc_graph_create(2, 2, off, ok_cols, np.array([1, 0, 1], dtype=np.int8))
    assert e.value.status == 2  # sign 0
    with pytest.raises(sbc.SbcError) as e:
        sbc.sbc_graph_create(2, 2, np.array([0, 3, 2], dtype=np.int64), ok_cols, ok_signs)
    assert e.value.status == 2  # decreasing offsets
    with sbc.sbc_graph_create(2, 2, off, ok_cols, ok_signs) as h:
        for p, q in [(1, 3), (3, 1), (9, 2), (2, 9)]:
            with pytest.raises(sbc.SbcError) as e:
                sbc.sbc_count(h, p, q)
            assert e.value.status == 1


# ---------------------------------------------------------------- kernel paths

def test_wide_anchors(sbc):
    # anchors with more than 256 useful neighbours take the streamed path
    rng = np.random.default_rng(7)
    m, n = 24, 700
    u, v = np.divmod(np.arange(m * n), n)
    keep = rng.random(m * n) < 0.85
    lab_u = rng.choice([-1, 1], m)
    lab_v = rng.choice([-1, 1], n)
    s = (lab_u[u] * lab_v[v]).astype(np.int8)
    flip = rng.random(m * n) < 0.02
    s[flip] *= -1
    g = sbc_synth.from_edges(m, n, u[keep], v[keep], s[keep])
    for p, q in [(2, 3), (3, 3), (4, 3), (3, 4)]:
        want = oracle.count(g, p, q, side=0)
        assert gpu_count(sbc, g, p, q, 0) == want, (p, q)


def test_hash_windows(sbc):
    # an anchor whose 2-hop set is far above one table window
    rng = np.random.default_rng(11)
    hubs = 12
    n_u, n_v = 6000, 40
    us, vs = [], []
    for h in range(hubs):
        members = rng.choice(np.arange(1, n_u), size=2500, replace=False)
        us.extend(members.tolist())
        vs.extend([h] * len(members))
        if h < 3:  # vertex 0: low degree (low priority), neighbours are hubs
            us.append(0)
            vs.append(h)
    for v in range(hubs, n_v):
        members = rng.choice(n_u, size=50, replace=False)
        us.extend(members.tolist())
        vs.extend([v] * 50)
    key = np.unique(np.array(us) * n_v + np.array(vs))
    u, v = np.divmod(key, n_v)
    s = np.where(rng.random(len(u)) < 0.3, -1, 1)
    g = sbc_synth.from_edges(n_u, n_v, u, v, s)
    for p, q in [(2, 2), (2, 3), (3, 3)]:
        want = oracle.count(g, p, q, side=0)
        with sbc.graph_from_synth(g) as h:
            got, st, _ = sbc.sbc_count_ex(h, p, q, anchor_side=0)
        assert got == want, (p, q)


def test_large_binomials_u128(sbc):
    # K_{3, 5000}: binom(5000, 8) needs more than 64 bits
    m, n = 3, 5000
    g = complete(m, n)
    for p, q in [(2, 8), (3, 8), (3, 7)]:
        want = comb(m, p) * comb(n, q)
        with sbc.graph_from_synth(g) as h:
            got, st, _ = sbc.sbc_count_ex(h, p, q, anchor_side=0)
        assert got == want


# ---------------------------------------------------------------- invariances

def test_switching_and_negation_invariance(sbc, small):
    u, v, s = small.edges()
    want = gpu_count(sbc, small, 3, 3)
    s2 = s.copy()
    s2[u == 17] *= -1
    s2[v == 3] *= -1
    g2 = sbc_synth.from_edges(small.n_u, small.n_v, u, v, s2)
    assert gpu_count(sbc, g2, 3, 3) == want
    g3 = sbc_synth.from_edges(small.n_u, small.n_v, u, v, -s)
    assert gpu_count(sbc, g3, 3, 3) == want
    gt = sbc_synth.from_edges(small.n_v, small.n_u, v, u, s)
    assert gpu_count(sbc, gt, 4, 3) == gpu_count(sbc, small, 3, 4)


def test_sharding_partitions_anchors(sbc, small):
    want = oracle.count(small, 3, 3)
    with sbc.graph_from_synth(small) as h:
        parts = [sbc.sbc_count_ex(h, 3, 3, shard=i, shard_count=3)[0] for i in range(3)]
    assert sum(parts) == want


def test_resumable_count_after_an_interruption(sbc, small, tmp_path):
    """sbc_count_resumable: a count interrupted after two of five shards and
    resumed from its state file gives the oracle's total."""
    want = oracle.count(small, 3, 3)
    path = str(tmp_path / "count.json")
    calls = {"n": 0}

    def flaky(*a, **k):
        calls["n"] += 1
        if calls["n"] == 3:
            raise RuntimeError("interrupted")
        return sbc.sbc_count_ex(*a, **k)

    with sbc.graph_from_synth(small) as h:
        with pytest.raises(RuntimeError):
            sbc.sbc_count_resumable(h, 3, 3, 5, path, count_fn=flaky)
        assert sbc.sbc_count_resumable(h, 3, 3, 5, path) == want


# ---------------------------------------------------------------- both sides

@pytest.mark.parametrize("method", ["candidate", "position"])
@pytest.mark.parametrize("seed", range(3))
def test_enumeration_sides_agree(sbc, method, seed):
    """Candidate-subset and position-subset enumeration give the oracle's
    count (totals and per anchor) on random graphs and all (p,q) in [2,5]^2."""
    rng = random.Random(seed)
    g = sbc_synth.chung_lu_signed(500 + seed, rng.randint(200, 900), rng.randint(200, 900),
                                  rng.randint(2000, 9000), 2.0, 2.2, 0.15)
    with sbc.graph_from_synth(g) as h:
        for p in range(2, 6):
            for q in range(2, 6):
                want, per = oracle.count(g, p, q, side=0, per_anchor=True)
                got, st, pa = sbc.sbc_count_ex(h, p, q, anchor_side=0, method=method,
                                               per_anchor=True)
                assert got == want, (p, q, method)
                assert pa == per, (p, q, method)


@pytest.mark.parametrize("method", ["auto", "candidate", "position"])
def test_small_workload_all_methods(sbc, small, method):
    with sbc.graph_from_synth(small) as h:
        for p, q in [(3, 3), (4, 4), (3, 4), (4, 3)]:
            want = oracle.count(small, p, q, side=0)
            for side in (0, 1):
                got, _, _ = sbc.sbc_count_ex(h, p, q, anchor_side=side, method=method)
                assert got == want, (p, q, side, method)


@pytest.mark.parametrize("budget_kb", [1, 64])
def test_anchor_groups_under_pool_budget(sbc, small, monkeypatch, budget_kb):
    """A pool budget far below the candidate masks' total splits the anchors
    into many groups run one after another; counts, per-anchor values and the
    plan's counters do not change (the tuple-phase counters depend on where
    work items are split, which follows each group's cost total)."""
    with sbc.graph_from_synth(small) as h:
        ref = {pq: sbc.sbc_count_ex(h, *pq, anchor_side=0, per_anchor=True)
               for pq in [(3, 3), (4, 4), (3, 4)]}
        monkeypatch.setenv("SBC_POOL_BUDGET_KB", str(budget_kb))
        for (p, q), (c0, st0, pa0) in ref.items():
            got, st, pa = sbc.sbc_count_ex(h, p, q, anchor_side=0, per_anchor=True)
            assert got == c0 == oracle.count(small, p, q, side=0)
            assert pa == pa0
            for key in ("candidates", "wedges"):
                assert st[key] == st0[key], key
            # more launches than the single-group plan
            assert st["kernels"] > st0["kernels"]


def test_batch_replay_with_anchor_groups(sbc, small, monkeypatch):
    """A batch whose plan needs several anchor groups is not captured and
    re-plans on each run; totals stay exact."""
    gs = [small, sbc_synth.plain_small()]
    want = [oracle.count(g, 3, 3, side=0) for g in gs]
    monkeypatch.setenv("SBC_POOL_BUDGET_KB", "4")
    hs = [sbc.graph_from_synth(g) for g in gs]
    try:
        with sbc.Batch(hs, 3, 3) as b:
            assert b.run() == want
            assert b.run() == want
        assert sbc.sbc_count_batch(hs, 3, 3) == want
    finally:
        for h in hs:
            h.close()


def dense_faction_graph(m, n, density, seed, flip=0.05):
    rng = np.random.default_rng(seed)
    u, v = np.divmod(np.arange(m * n), n)
    keep = rng.random(m * n) < density
    lab_u = rng.choice([-1, 1], m)
    lab_v = rng.choice([-1, 1], n)
    s = (lab_u[u] * lab_v[v]).astype(np.int8)
    s[rng.random(m * n) < flip] *= -1
    return sbc_synth.from_edges(m, n, u[keep], v[keep], s[keep])


def sparse_with_block(m, n, rho_block, rho_other, bu, bv, seed, flip=0.05):
    """Sparse random edges (density rho_block on bu planted U-vertices,
    rho_other on the rest) plus a complete bu x bv block with faction signs.
    The planted vertices have the lowest degrees, so they come first in the
    priority order with every other vertex as a partner; among themselves
    they share the block, so three-partner tuples survive."""
    rng = np.random.default_rng(seed)
    bu_ids = rng.choice(m, bu, replace=False)
    rho = np.full(m, rho_other)
    rho[bu_ids] = rho_block
    mask = rng.random((m, n)) < rho[:, None]
    mask[np.ix_(bu_ids, rng.choice(n, bv, replace=False))] = True
    u, v = np.nonzero(mask)
    lab_u = rng.choice([-1, 1], m)
    lab_v = rng.choice([-1, 1], n)
    s = (lab_u[u] * lab_v[v]).astype(np.int8)
    s[rng.random(len(u)) < flip] *= -1
    return sbc_synth.from_edges(m, n, u, v, s), bu_ids


def lowest_priority(g, k, among=None):
    """The k U-vertices first in the priority order (degree, then id), or the
    first k of `among`: they have the most higher-priority partners."""
    deg = np.diff(g.offsets)
    order = np.lexsort((np.arange(g.n_u), deg)).tolist()
    if among is not None:
        keep = set(int(x) for x in among)
        order = [x for x in order if x in keep]
    return order[:k]


@pytest.mark.parametrize("case", ["pairs", "pairs_q4", "triples_slot", "triples_scratch"])
def test_global_mask_paths(sbc, case):
    """Anchors whose candidate masks exceed the tuple kernel's shared memory
    (two partners: blocked path; three partners: shared per-warp slot and
    global scratch), per anchor against the oracle; the whole count against
    the other anchor side."""
    if case.startswith("pairs"):
        g = dense_faction_graph(1200, 700, 0.6, seed=17)
        anchors = lowest_priority(g, 6)
        p, q = (3, 3) if case == "pairs" else (3, 4)
    else:
        rho_b, rho_o = (0.03, 0.05) if case == "triples_slot" else (0.04, 0.06)
        g, block = sparse_with_block(420, 25000, rho_b, rho_o, 30, 250, seed=23)
        anchors = lowest_priority(g, 6, among=block)
        p, q = 4, 3
    with sbc.graph_from_synth(g) as h:
        total, st, per = sbc.sbc_count_ex(h, p, q, anchor_side=0, per_anchor=True)
        other, _, _ = sbc.sbc_count_ex(h, p, q, anchor_side=1)
    assert total == other
    _, want = oracle.count(g, p, q, side=0, per_anchor=True, anchors=anchors)
    assert [per[a] for a in anchors] == [want[a] for a in anchors]
    assert sum(want[a] for a in anchors) > 0
