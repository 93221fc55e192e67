"""Checkpoint / resume of long counts (sbc_count_resumable), host logic with a
stand-in for the per-shard count: partial sums recorded after every shard,
an interrupted count resumed without recounting recorded shards, the side
fixed by the first shard, and a state file of another count refused."""
import json
import types

import pytest


@pytest.fixture(scope="module")
def sbc():
    import paper_2605_03603_gb300 as m

    return m


class FakeShards:
    """Per-shard counts above 2^64; raises once at shard `fail_at`."""

    def __init__(self, fail_at=None):
        self.fail_at = fail_at
        self.calls = []

    def value(self, i):
        return (i + 1) * (2**70 + 12345)

    def __call__(self, g, p, q, anchor_side, shard, shard_count, stream):
        self.calls.append((shard, anchor_side))
        if shard == self.fail_at:
            self.fail_at = None
            raise RuntimeError("interrupted")
        return self.value(shard), {"anchor_side": 1}, None


G = types.SimpleNamespace(n_u=10, n_v=20, nnz=30)


def test_interrupted_count_resumes(sbc, tmp_path):
    path = str(tmp_path / "state.json")
    f = FakeShards(fail_at=4)
    with pytest.raises(RuntimeError):
        sbc.sbc_count_resumable(G, 3, 3, 7, path, count_fn=f)
    st = json.load(open(path))
    assert st["done"] == [0, 1, 2, 3] and int(st["partial"]) == sum(f.value(i) for i in range(4))
    assert st["side"] == 1
    f.calls.clear()
    total = sbc.sbc_count_resumable(G, 3, 3, 7, path, count_fn=f)
    assert total == sum(f.value(i) for i in range(7))
    # only the missing shards were counted, on the side the first shard chose
    assert f.calls == [(i, 1) for i in range(4, 7)]
    f.calls.clear()
    assert sbc.sbc_count_resumable(G, 3, 3, 7, path, count_fn=f) == total and not f.calls


def test_state_of_another_count_is_refused(sbc, tmp_path):
    path = str(tmp_path / "state.json")
    sbc.sbc_count_resumable(G, 3, 3, 4, path, count_fn=FakeShards())
    for args in [(G, 3, 4, 4), (G, 3, 3, 5), (types.SimpleNamespace(n_u=10, n_v=20, nnz=31), 3, 3, 4)]:
        with pytest.raises(ValueError):
            sbc.sbc_count_resumable(*args, path, count_fn=FakeShards())
    with pytest.raises(ValueError):
        sbc.sbc_count_resumable(G, 3, 3, 4, path, anchor_side=0, count_fn=FakeShards())
