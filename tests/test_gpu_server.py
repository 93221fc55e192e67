"""Serving (sbc_server_*): every answer equals the count of the same request
made alone, whatever mix of requests it was fused or overlapped with."""
import random
import threading

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
def resident(sbc):
    rng = random.Random(5)
    gs = []
    for i in range(24):
        n_u, n_v = rng.randint(20, 600), rng.randint(20, 600)
        m = min(rng.randint(100, 6000), n_u * n_v // 2)
        gs.append(sbc_synth.chung_lu_signed(7000 + i, n_u, n_v, m, rng.uniform(1.9, 2.5),
                                            rng.uniform(1.9, 2.5), rng.uniform(0.0, 0.3)))
    gs.append(sbc_synth.plain_small())
    gs.append(sbc_synth.chung_lu_signed(7100, 20000, 15000, 120000, 2.2, 2.2, 0.2))
    hs = [sbc.graph_from_synth(g) for g in gs]
    yield gs, hs
    for h in hs:
        h.close()


PQS = [(3, 3), (3, 4), (4, 4)]


def test_server_mix_equals_alone(sbc, resident):
    gs, hs = resident
    alone = {(i, p, q): sbc.sbc_count(h, p, q) for i, h in enumerate(hs) for p, q in PQS}
    # the alone counts themselves match the oracle on the small graphs
    for i in range(0, 24, 6):
        for p, q in PQS:
            assert alone[(i, p, q)] == oracle.count(gs[i], p, q, side=0)
    with sbc.Server(lanes=3, max_batch=16, small_edges=30000) as srv:
        gids = [srv.add_graph(h) for h in hs]
        rng = random.Random(11)
        work = [(rng.randrange(len(gids)), *rng.choice(PQS)) for _ in range(240)]
        tickets = [None] * len(work)

        def submitter(k):
            for idx in range(k, len(work), 3):
                g, p, q = work[idx]
                tickets[idx] = srv.submit(gids[g], p, q)

        ths = [threading.Thread(target=submitter, args=(k,)) for k in range(3)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        for idx, (g, p, q) in enumerate(work):
            got, lat = srv.wait(tickets[idx])
            assert got == alone[(g, p, q)], (g, p, q)
            assert lat >= 0
        st = srv.stats()
        assert st["completed"] == len(work) and st["failed"] == 0
        assert st["jobs"] <= len(work)
        assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]


def test_server_tiny_budget_serialises(sbc, resident):
    gs, hs = resident
    with sbc.Server(mem_budget_bytes=1, lanes=4, max_batch=8) as srv:
        gids = [srv.add_graph(h) for h in hs[:8]]
        ts = [(g, srv.submit(gids[g], 3, 3)) for g in range(8) for _ in range(2)]
        for g, t in ts:
            got, _ = srv.wait(t)
            assert got == sbc.sbc_count(hs[g], 3, 3)
        assert srv.stats()["peak_admitted_bytes"] > 0


def test_server_errors_and_timeouts(sbc, resident):
    gs, hs = resident
    with sbc.Server(lanes=1) as srv:
        gid = srv.add_graph(hs[-2])
        with pytest.raises(sbc.SbcError) as e:
            srv.submit(gid + 100, 3, 3)
        assert e.value.status == 1
        with pytest.raises(sbc.SbcError) as e:
            srv.submit(gid, 1, 3)
        assert e.value.status == 1
        t = srv.submit(gid, 3, 3)
        try:
            got, _ = srv.wait(t, timeout_us=0)
        except sbc.SbcError as err:
            assert err.status == 5  # SBC_E_TIMEOUT: still pending, wait again
            got, _ = srv.wait(t)
        assert got == sbc.sbc_count(hs[-2], 3, 3)
        with pytest.raises(sbc.SbcError) as e:
            srv.wait(t)  # ticket already released
        assert e.value.status == 1
