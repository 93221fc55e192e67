"""The N > 1 host path on CPU: two gloo ranks count disjoint anchor shards with
the oracle and combine the exact u128 partials with
paper_2605_03603_gb300.dist; the sum equals the whole-graph count. Also checks
limb carries and the 128-bit overflow report across ranks."""
import json
import os
import socket

import pytest

import oracle
import sbc_synth

WORLD = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    import torch.distributed as dist

    from paper_2605_03603_gb300 import dist as sd

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=WORLD)
    res = {}
    try:
        g = sbc_synth.plain_small()
        parts = []
        for p, q, side in [(3, 3, 0), (2, 2, 1), (3, 4, 0), (4, 3, 1)]:
            n_s = g.n_u if side == 0 else g.n_v
            mine = [a for a in range(n_s) if a % WORLD == rank]
            parts.append(oracle.count(g, p, q, side=side, threads=2, anchors=mine))
        res["counts"] = [str(v) for v in sd.allreduce_counts(parts)]
        # carries across limbs and across the 64-bit boundary
        big = [(1 << 96) - 1, (1 << 64) - 1, (1 << 127) - 5] if rank == 0 else [1, 1, 4]
        res["big"] = [str(v) for v in sd.allreduce_counts(big)]
        try:
            sd.allreduce_counts([1 << 127])
            res["overflow"] = False
        except OverflowError:
            res["overflow"] = True
        res["max"] = sd.max_over_ranks(10.0 + rank)
        res["empty"] = sd.allreduce_counts([])
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_sharded_counts_sum_exactly(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.spawn(_rank_main, args=(port, str(tmp_path)), nprocs=WORLD, join=True)
    g = sbc_synth.plain_small()
    want = [oracle.count(g, p, q, side=side) for p, q, side in
            [(3, 3, 0), (2, 2, 1), (3, 4, 0), (4, 3, 1)]]
    assert want[0] > 0
    for r in range(WORLD):
        with open(tmp_path / f"rank{r}.json") as f:
            res = json.load(f)
        assert [int(v) for v in res["counts"]] == want
        assert [int(v) for v in res["big"]] == [1 << 96, 1 << 64, (1 << 127) - 1]
        assert res["overflow"] is True
        assert res["max"] == 11.0
        assert res["empty"] == []


def test_limbs_roundtrip():
    from paper_2605_03603_gb300 import dist as sd

    for x in [0, 1, (1 << 32) - 1, 1 << 32, (1 << 128) - 1, 0x0123456789ABCDEF_FEDCBA9876543210]:
        assert sd.from_limbs(sd.to_limbs(x)) == x
    with pytest.raises(OverflowError):
        sd.to_limbs(1 << 128)
    with pytest.raises(OverflowError):
        sd.to_limbs(-1)
