"""Parity at the benchmark's full size (200,000 x 100,000, 2,000,000 edges),
in the launch configuration bench.py times (device-resident input, automatic
anchor side and method), and on the 60,000,000-edge workload.

The oracle cannot count the whole graph within a test for (4,4), so:
* per-anchor contributions of a seeded sample of anchors (uniform, nonzero,
  and the heaviest, uncapped) are compared with the oracle computed for those
  anchors only;
* totals are compared through properties that hold at any size: the (3,3)
  count is the same whether the anchors are U or V vertices (side swap), and
  the per-anchor values add up to the total; the full (3,3) total is also
  compared with the oracle's.
"""
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


@pytest.fixture(scope="module")
def medium(sbc):
    import torch

    g = sbc_synth.plain_medium()
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    sgn = torch.from_numpy(g.signs).cuda()
    h = sbc.sbc_graph_create(g.n_u, g.n_v, off, col, sgn)
    yield g, h
    h.close()


def sample_anchors(per, rng, n_uniform=120, n_nonzero=120, n_top=12):
    per = np.asarray([float(x) for x in per])
    nz = np.nonzero(per)[0]
    top = nz[np.argsort(-per[nz])][:n_top]
    pick = set(rng.choice(len(per), size=n_uniform, replace=False).tolist())
    pick |= set(rng.choice(nz, size=min(n_nonzero, len(nz)), replace=False).tolist())
    pick |= set(top.tolist())
    return sorted(pick), top


@pytest.mark.parametrize("p,q,cap", [(3, 3, 0), (4, 4, 0)])
def test_fullsize_sampled_anchors(sbc, medium, p, q, cap):
    g, h = medium
    total, st, per = sbc.sbc_count_ex(h, p, q, anchor_side=0, per_anchor=True)
    assert sum(per) == total
    rng = np.random.default_rng(100 * p + q)
    anchors, top = sample_anchors(per, rng)
    skipped = set()
    _, want = oracle.count(g, p, q, side=0, per_anchor=True, anchors=anchors,
                           max_subsets=cap, skipped=skipped)
    compared = [a for a in anchors if a not in skipped]
    assert len(compared) >= 200 and set(top) <= set(compared)  # the 12 heaviest included
    mism = [(a, per[a], want[a]) for a in compared if per[a] != want[a]]
    assert not mism, mism[:5]
    # the heaviest compared anchors carry a real share of the count
    assert sum(per[a] for a in compared) > 0


def test_fullsize_totals_side_swap(sbc, medium):
    """(3,3) anchored on U and on V agree. The (4,4) swap is left to the small
    graphs: anchored on V this graph has about 100x the candidate-side work
    (V-anchors with up to 10^4 candidates and too many for the position side),
    which the cost model never picks."""
    g, h = medium
    a, _, _ = sbc.sbc_count_ex(h, 3, 3, anchor_side=0)
    b, _, _ = sbc.sbc_count_ex(h, 3, 3, anchor_side=1)
    auto = sbc.sbc_count(h, 3, 3)
    assert a == b == auto


def test_fullsize_33_total_equals_oracle_reference(sbc, medium):
    """The full (3,3) total against the complete oracle count (all anchors).
    About a minute of host time on 16 cores."""
    g, h = medium
    want = oracle.count(g, 3, 3, side=0)
    assert sbc.sbc_count(h, 3, 3) == want


# ------------------------------------------------------------------ 60M edges

@pytest.fixture(scope="module")
def large(sbc):
    """5,000,000 x 1,000,000, 60,000,000 edges, signs packed one bit per
    edge, int64 row offsets (the largest workload)."""
    g = sbc_synth.plain_large()
    h = sbc.graph_from_synth(g, device=True, sign_bits=True)
    yield g, h
    h.close()


def _large_sampled(sbc, g, h, p, q, seed, n_top=8):
    """Per-anchor values of the automatic count for a seeded sample of anchors
    (uniform, nonzero, the heaviest) against the oracle on the same side,
    uncapped; per-anchor values add up to the total. Returns (total, side)."""
    total, st, per = sbc.sbc_count_ex(h, p, q, per_anchor=True)
    side = st["anchor_side"]
    assert sum(per) == total
    rng = np.random.default_rng(seed)
    anchors, top = sample_anchors(per, rng, n_uniform=100, n_nonzero=150, n_top=n_top)
    _, want = oracle.count(g, p, q, side=side, per_anchor=True, anchors=anchors)
    mism = [(a, per[a], want[a]) for a in anchors if per[a] != want[a]]
    assert not mism, mism[:5]
    assert len(anchors) >= 150 and sum(per[a] for a in anchors) > 0
    return total, side


def test_large_33_sampled_anchors(sbc, large):
    """(3,3) on the preferred anchor side (V), uncapped oracle sample; the
    plain count (no per-anchor output) gives the same total."""
    g, h = large
    total, side = _large_sampled(sbc, g, h, 3, 3, 333)
    assert side == 1
    assert total == sbc.sbc_count(h, 3, 3)


def test_large_43_sampled_anchors(sbc, large):
    """(4,3): four vertices from U, three from V; anchored on V, where the
    tuples have three vertices (two partners: the tensor-core form)."""
    g, h = large
    _, side = _large_sampled(sbc, g, h, 4, 3, 433)
    assert side == 1


def test_large_34_sampled_anchors(sbc, large):
    """(3,4): three vertices from U, four from V. The automatic side is U
    (tuples of three there, of four on V); per-anchor values against the
    oracle."""
    g, h = large
    _, side = _large_sampled(sbc, g, h, 3, 4, 344)
    assert side == 0
