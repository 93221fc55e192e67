#!/usr/bin/env python
"""Benchmark: balanced (p,q)-biclique counting on one GB300 (or N replicas).

Workload (default): one seeded signed Chung-Lu graph, |U| = 5,000,000,
|V| = 1,000,000, 60,000,000 edges (exponent 2.4 on U, 1.9 on V with V hubs
capped at 50,000 expected degree, 4 planted factions with flip probability
0.2), counted for (p,q) = (3,3). Inputs (the 60M-edge CSR, ~1.1 GB on the
device) are larger than L2; L2 is also flushed between steps (512 MiB write).

A step is the whole hot path on device-resident CSR input: graph build
(validation, degrees, vertex priority, oriented adjacency) + the exact (3,3)
count. The metric is anchor tuples per second: the number of (k-1)-subsets of
candidates Algorithm 2 enumerates (sum over anchors of binom(|C(u)|, k-1),
counted once, outside the timed region) over the step time; the line also
gives seconds to the exact (3,3) count (seconds_to_exact_33).

The line also carries:
* roofline: the step's dominant kernel against its bound (the tuple kernel
  in population counts per second against the POPC rate measured on this GPU
  in the same run; the tensor-core pair kernel in fp8 TFLOP/s against the
  measured bf16 peak times 2; the 2-hop kernels in bytes per second against
  the measured HBM copy peak), and roofline_kernels with all three;
* e2e: the same metric through the public API from pinned host buffers
  (upload + build + count + the 16-byte result read);
* cpu_baseline: the oracle (plain C, all host cores) on a bounded random
  sample of anchors of the same count, with its estimate for the whole count;
* medium: the 2M-edge graph, (3,3) + (4,4) per step;
* batch: the 10,000-graph batch recipe (graphs/s of the per-graph path, one
  batched count, CUDA-graph replay, replay with autotuned launch parameters);
* serve: Poisson requests on resident graphs (p50/p99, throughput) against
  a one-request-at-a-time server (one lane, no fusing) on the same arrivals.

--impl reference runs the oracle on the same workload and count, one bounded
random anchor sample per step (graph lists built once, outside the timing),
and reports the same metric.

Multi-GPU (torchrun): anchors are sharded by rank (anchor rank mod N) over a
replicated graph; each rank counts its shard; partial counts are summed
exactly on the host (paper_2605_03603_gb300.dist). Total work is fixed, so
scaling is strong.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "anchor tuples/sec and seconds to exact balanced (3,3) count; batched graphs/sec, p99"
WORKLOAD = "plain-5M-1M-60M"
PQ = [(3, 3)]
# DRAM bytes (read + write) of a kernel's launches in one step of a workload
# (the same unit as the kernel's `achieved`), from one ncu capture of the
# current kernels; None where not captured. k_twohop: its two CTA-tier
# launches of the (3,3) count.
TRAFFIC = {("k_twohop", "plain-5M-1M-60M"): 279_530_419_712}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


WORKLOADS = {"plain-200k-100k-2M": "plain_medium", "plain-50k-25k-500k": "plain_quarter",
             "plain-2k-1.5k-20k": "plain_small", "plain-5M-1M-60M": "plain_large",
             "dense-3000x400": "dense_factions", "dense-3000x800": "dense_factions_wide"}


def load_workload(name=None):
    import sbc_synth

    return getattr(sbc_synth, WORKLOADS[name or WORKLOAD])()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def anchor_side(g) -> int:
    """The side the library's cost model anchors on: fewer 2-paths to visit,
    sum over the other side of binom(degree, 2) (ties: U)."""
    du = np.diff(g.offsets).astype(np.float64)
    dv = np.bincount(g.cols, minlength=g.n_v).astype(np.float64)
    wu = float((dv * (dv - 1) / 2).sum())  # anchoring on U visits wedges through V
    wv = float((du * (du - 1) / 2).sum())
    return 0 if wu <= wv else 1


# ------------------------------------------------------------------ CPU oracle

def oracle_sample(prep, g, side, p, q, frac, seed, threads=0):
    """The oracle on a seeded random sample of anchors (lists already built).
    Returns (tuples, seconds, anchors, threads)."""
    import oracle

    rng = np.random.default_rng(seed)
    n_s = g.n_u if side == 0 else g.n_v
    anchors = np.nonzero(rng.random(n_s) < frac)[0]
    t0 = time.perf_counter()
    _, tuples = prep.count(p, q, threads=threads, with_tuples=True, anchors=anchors)
    dt = time.perf_counter() - t0
    return tuples, dt, len(anchors), oracle.max_threads() if threads == 0 else threads


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    g = load_workload()
    side = anchor_side(g)
    p, q = PQ[0]
    frac = args.ref_frac
    tot_t, tot_tuples, cores, anchors = 0.0, 0, 0, 0
    with oracle.Prepared(g, side) as prep:
        for i in range(args.warmup):
            oracle_sample(prep, g, side, p, q, frac / 4, 100 + i)
        for i in range(args.steps):
            tup, dt, na, cores = oracle_sample(prep, g, side, p, q, frac, 1000 + i)
            tot_t += dt
            tot_tuples += tup
            anchors += na
    value = tot_tuples / tot_t
    side_name = "U" if side == 0 else "V"
    sample = (f"({p},{q}) on a seeded random {frac:.3%} sample of {side_name} anchors per step "
              f"({anchors // max(args.steps, 1)} anchors), oracle in C with OpenMP, graph "
              f"lists built once before the timed steps")
    est_s = (tot_t / args.steps) / frac  # the sampled anchors' time scaled to all anchors
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "anchor tuples/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * tot_t / max(args.steps, 1), "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "pq": f"({p},{q})", "sample": sample},
        "seconds_to_exact_33_estimate": est_s,
        "cpu_baseline": {"value": value, "unit": "anchor tuples/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "anchor tuples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ extra legs

def medium_leg(sbc, torch, args):
    """The 2M-edge graph: graph build + (3,3) + (4,4) per step (3 timed steps)."""
    g = load_workload("plain-200k-100k-2M")
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    sgn = torch.from_numpy(g.signs).cuda()
    pqs = [(3, 3), (4, 4)]
    tuples, counts = {}, {}
    with sbc.sbc_graph_create(g.n_u, g.n_v, off, col, sgn) as h:
        for p, q in pqs:
            c, st, _ = sbc.sbc_count_ex(h, p, q, paper_tuples=True)
            counts[(p, q)], tuples[(p, q)] = c, st["anchor_tuples"]

    def step():
        with sbc.sbc_graph_create(g.n_u, g.n_v, off, col, sgn) as h:
            out = []
            for p, q in pqs:
                c, st, _ = sbc.sbc_count_ex(h, p, q)
                assert c == counts[(p, q)]
                out.append(st)
            return out

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sts = [step() for _ in range(3)]
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0) / 3
    ms33 = float(np.mean([s[0]["ms_total"] for s in sts]))
    return {"workload": "plain-200k-100k-2M", "pq": "(3,3)+(4,4)", "ms_per_step": ms,
            "anchor_tuples_per_s": sum(tuples.values()) / (ms / 1e3),
            "ms_33": ms33, "anchor_tuples_per_s_33": tuples[(3, 3)] / (ms33 / 1e3),
            "counts": {str(k): v for k, v in counts.items()},
            "phase_ms": {f"({p},{q})": {k: sts[-1][i][k] for k in
                                         ("ms_twohop", "ms_tuples", "ms_tc", "ms_prepare")}
                         for i, (p, q) in enumerate(pqs)}}


def dynamic_leg(sbc, torch, args):
    """Exact counts under single-edge updates (sbc_dyn_*) on the 2M-edge
    graph, (3,3): latency of random insertions, each undone by deleting the
    edge (the count must return to the start), of sign changes of present
    edges (each undone), and of updates (insertion or sign change) of the
    pairs of the eight highest-degree vertices of each side."""
    g = load_workload("plain-200k-100k-2M")
    rng = np.random.default_rng(17)
    u_all, v_all, s_all = g.edges()
    keys = np.sort(u_all.astype(np.int64) * g.n_v + v_all.astype(np.int64))

    def absent(u, v):
        k = u * g.n_v + v
        i = int(np.searchsorted(keys, k))
        return i == keys.shape[0] or int(keys[i]) != k

    t0 = time.perf_counter()
    d = sbc.Dynamic.from_synth(g, 3, 3)
    create_s = time.perf_counter() - t0
    try:
        base = d.count()
        ins, dele, flip, hub = [], [], [], []
        n = args.dyn_updates
        while len(ins) < n:
            u, v = int(rng.integers(g.n_u)), int(rng.integers(g.n_v))
            if not absent(u, v):
                continue
            t = time.perf_counter()
            d.insert(u, v, int(rng.choice([-1, 1])))
            ins.append(time.perf_counter() - t)
            t = time.perf_counter()
            c = d.delete(u, v)
            dele.append(time.perf_counter() - t)
            if c != base:
                raise AssertionError(f"count {c} after undoing an insertion, expected {base}")
        for e in rng.choice(u_all.shape[0], size=max(1, n // 4), replace=False).tolist():
            u, v, s = int(u_all[e]), int(v_all[e]), int(s_all[e])
            t = time.perf_counter()
            d.set_sign(u, v, -s)
            flip.append(time.perf_counter() - t)
            if d.set_sign(u, v, s) != base:
                raise AssertionError("count changed after undoing a sign change")
        hubs_u = np.argsort(-np.diff(g.offsets))[:8].tolist()
        hubs_v = np.argsort(-np.bincount(g.cols, minlength=g.n_v))[:8].tolist()
        sign_of = dict(zip((u_all * g.n_v + v_all).tolist(), s_all.tolist())) if hubs_u else {}
        t_hub = time.perf_counter()
        for u in hubs_u:
            for v in hubs_v:
                if time.perf_counter() - t_hub > 20.0:  # bounded wall time for the leg
                    break
                t = time.perf_counter()
                if absent(u, v):
                    d.insert(u, v, 1)
                    hub.append(time.perf_counter() - t)
                    undone = d.delete(u, v)
                else:
                    s = int(sign_of[u * g.n_v + v])
                    d.set_sign(u, v, -s)
                    hub.append(time.perf_counter() - t)
                    undone = d.set_sign(u, v, s)
                if undone != base:
                    raise AssertionError("count changed after undoing a hub update")
    finally:
        d.close()
    ms = lambda x: {"median_ms": 1e3 * float(np.median(x)), "p99_ms": 1e3 * float(np.percentile(x, 99)),
                    "max_ms": 1e3 * float(np.max(x)), "n": len(x)} if x else None
    return {"workload": "plain-200k-100k-2M", "pq": "(3,3)", "create_s": create_s, "count": base,
            "insert": ms(ins), "delete": ms(dele), "set_sign": ms(flip), "hub_updates": ms(hub),
            "exact": "every update undone returned the count to its start"}


def batch_leg(sbc, torch, args):
    """Graphs/s for B independent graphs of the 10,000-graph batch recipe:
    plain one-count-per-graph path, one batched count (sbc_count_batch), a
    planned batch replayed from a CUDA graph, and the same replay with the
    autotuner's launch parameters (tuning time reported)."""
    import sbc_synth

    t0 = time.perf_counter()
    gs = sbc_synth.batch_graphs(4, args.batch_graphs)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    hs = [sbc.graph_from_synth(g) for g in gs]
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    edges = sum(g.m for g in gs)
    del gs
    p, q = 3, 3

    def timed(fn, reps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            res = fn()
        torch.cuda.synchronize()
        return res, (time.perf_counter() - t) / reps

    plain, t_plain = timed(lambda: [sbc.sbc_count(h, p, q) for h in hs], 1)
    batched, t_batch = timed(lambda: sbc.sbc_count_batch(hs, p, q), 2)
    with sbc.Batch(hs, p, q) as b:
        b.run()
        replay, t_replay = timed(b.run, 3)
    # the autotuner times a sample of the batch (at most 1,000 graphs)
    n_tune = min(len(hs), 1000)
    t0 = time.perf_counter()
    tune = sbc.sbc_autotune(hs[:n_tune], p, q, reps=2)
    t_tune = time.perf_counter() - t0
    with sbc.Batch(hs, p, q, tune=tune) as b:
        b.run()
        tuned, t_tuned = timed(b.run, 3)
    for name, other in (("batched", batched), ("replay", replay), ("tuned", tuned)):
        bad = [i for i in range(len(plain)) if plain[i] != other[i]]
        if bad:
            raise AssertionError(f"{name} differs from the per-graph counts on {len(bad)} graphs "
                                 f"(first: {bad[:5]})")
    for h in hs:
        h.close()
    n = len(hs)
    return {"graphs": n, "edges": int(edges), "pq": "(3,3)", "generate_s": t_gen,
            "create_s": t_create, "plain_graphs_per_s": n / t_plain,
            "batched_graphs_per_s": n / t_batch, "replay_graphs_per_s": n / t_replay,
            "tuned_replay_graphs_per_s": n / t_tuned, "autotune_s": t_tune,
            "autotune_graphs": n_tune, "tune": tune,
            "batched_vs_plain": t_plain / t_batch, "replay_vs_plain": t_plain / t_replay,
            "tuned_replay_vs_plain": t_plain / t_tuned, "total_count": sum(plain),
            "equal_to_plain": True}


def _serve_run(sbc, srv, gids, reqs, arr, want):
    """Submit `reqs` at arrival times `arr` (seconds from now) from a client
    thread; wait for all; check each count; return the server's stats."""
    srv.reset_stats()
    tickets = [None] * len(reqs)
    t_base = time.perf_counter()

    def client():
        for i, ((g, pq), a) in enumerate(zip(reqs, arr)):
            dt = t_base + a - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets[i] = srv.submit(gids[g], *pq)

    th = threading.Thread(target=client)
    th.start()
    th.join()
    for i, (g, pq) in enumerate(reqs):
        c, _ = srv.wait(tickets[i])
        assert c == want[(g, pq)]  # the same count alone and in the mix
    return srv.stats()


def serve_leg(sbc, torch, args):
    """Poisson-arriving requests (graph, p, q) on resident graphs: p50/p99
    latency and throughput of the server (continuous batching over lanes,
    fused small-graph requests) against a server that serves one request at a
    time with the plain path (one lane, no fusing), on the same arrivals."""
    import sbc_synth

    t0 = time.perf_counter()
    gs = sbc_synth.batch_graphs(5, args.serve_graphs, 1e3, args.serve_max_edges)
    t_gen = time.perf_counter() - t0
    hs = [sbc.graph_from_synth(g) for g in gs]
    edges = int(sum(g.m for g in gs))
    del gs
    pqs = [(3, 3), (3, 4), (4, 4)]
    rng = np.random.default_rng(5)
    want = {}
    t0 = time.perf_counter()
    for i, h in enumerate(hs):
        for pq in pqs:
            want[(i, pq)] = sbc.sbc_count(h, *pq)
    t_all = time.perf_counter() - t0  # every (graph, p, q) once, one at a time
    out = []
    budget = int(args.serve_budget_gb * 2**30)
    with sbc.Server(mem_budget_bytes=budget) as srv, \
            sbc.Server(mem_budget_bytes=budget, lanes=1, max_batch=1) as one:
        gids = [srv.add_graph(h) for h in hs]
        gids1 = [one.add_graph(h) for h in hs]
        for rate in args.serve_rates:
            n = int(min(args.serve_requests, max(200, rate * args.serve_seconds)))
            reqs = [(int(rng.integers(len(hs))), pqs[int(rng.integers(3))]) for _ in range(n)]
            arr = np.cumsum(rng.exponential(1.0 / rate, size=n))
            st = _serve_run(sbc, srv, gids, reqs, arr, want)
            # the one-at-a-time server saturates early; it serves a prefix of
            # the same arrivals (its queue only grows, so the prefix's
            # latencies understate the full run's)
            n1 = min(n, args.serve_baseline_requests)
            st1 = _serve_run(sbc, one, gids1, reqs[:n1], arr[:n1], want)
            out.append({"rate_per_s": rate, "requests": n, "p50_ms": st["p50_ms"],
                        "p99_ms": st["p99_ms"], "throughput_rps": st["throughput_rps"],
                        "jobs": st["jobs"], "fused_requests": st["fused_requests"],
                        "peak_admitted_gb": st["peak_admitted_bytes"] / 2**30,
                        "one_at_a_time": {"requests": n1, "p50_ms": st1["p50_ms"],
                                          "p99_ms": st1["p99_ms"],
                                          "throughput_rps": st1["throughput_rps"]}})
    for h in hs:
        h.close()
    return {"graphs": len(hs), "edges": edges, "max_edges": args.serve_max_edges,
            "generate_s": t_gen, "all_pairs_once_s": t_all,
            "pq": "(3,3)|(3,4)|(4,4) uniform", "budget_gb": args.serve_budget_gb,
            "rates": out}


def pq_sweep_leg(sbc, torch, args):
    """Seconds per exact count for p in {3,4,5}, q in {3..7} (the paper's
    (p,q) experiments) on the 20k-edge graph and for p in {3,4} on the
    2M-edge graph: automatic anchor side, graph resident, median of three
    counts."""
    out = {}
    for name in ("plain-2k-1.5k-20k", "plain-200k-100k-2M"):
        g = load_workload(name)
        rows = []
        with sbc.graph_from_synth(g, device=True) as h:
            for p in ((3, 4, 5) if name == "plain-2k-1.5k-20k" else (3, 4)):
                for q in range(3, 8):
                    times, st = [], None
                    for _ in range(3):
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        c, st, _ = sbc.sbc_count_ex(h, p, q)
                        times.append(time.perf_counter() - t0)
                    rows.append({"pq": f"({p},{q})", "count": c, "s": float(np.median(times)),
                                 "side": "UV"[st["anchor_side"]],
                                 "tc_anchors": st["tc_anchors"]})
        out[name] = rows
    return out


def _leg(fn, *a):
    """Run an extra leg; a failure is reported in the leg's object (the main
    line is still printed) and on stderr."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001 - reported, not swallowed
        import traceback

        traceback.print_exc()
        return {"error": f"{type(e).__name__}: {e}"}


# ------------------------------------------------------------------ GPU arm

def run_ours(args):
    import torch

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        gloo = dist.new_group(backend="gloo")
    else:
        torch.cuda.set_device(0)
    import paper_2605_03603_gb300 as sbc

    dev = torch.cuda.current_device()
    g = load_workload()
    import sbc_synth

    input_digest = sbc_synth.digest(g)  # compare with tests/golden/input_digests.txt
    stream = torch.cuda.Stream()
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    sgn = torch.from_numpy(g.signs).cuda()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    shard = dict(shard=rank, shard_count=ws) if ws > 1 else {}

    # Algorithm 2's anchor tuples and the exact counts (untimed, once)
    counts, tuples = {}, {}
    with torch.cuda.stream(stream):
        with sbc.sbc_graph_create(g.n_u, g.n_v, off, col, sgn, stream=stream) as h:
            for p, q in PQ:
                c, st, _ = sbc.sbc_count_ex(h, p, q, paper_tuples=True, stream=stream, **shard)
                counts[(p, q)] = c
                tuples[(p, q)] = st["anchor_tuples"]

    def step():
        with sbc.sbc_graph_create(g.n_u, g.n_v, off, col, sgn, stream=stream) as h:
            out = []
            for p, q in PQ:
                c, st, _ = sbc.sbc_count_ex(h, p, q, stream=stream, **shard)
                assert c == counts[(p, q)]
                out.append(st)
            return out

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()

    sampler = ClockSampler(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    ev33 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(args.steps)]
    per_step_stats = []
    launches0 = sbc.sbc_launch_count()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    # the integer-ALU rates of this GPU at the clocks of this run
    alu = sbc.sbc_measure_alu_rates(stream=stream)
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.zero_()  # L2 flush, outside the timed events
            ev[i][0].record(stream)
            ev33[i][0].record(stream)
            with sbc.sbc_graph_create(g.n_u, g.n_v, off, col, sgn, stream=stream) as h:
                sts = []
                for j, (p, q) in enumerate(PQ):
                    c, st, _ = sbc.sbc_count_ex(h, p, q, stream=stream, **shard)
                    if j == 0:
                        ev33[i][1].record(stream)
                    sts.append(st)
            ev[i][1].record(stream)
            per_step_stats.append(sts)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    launches = sbc.sbc_launch_count() - launches0 - 8  # the 8 ALU-rate launches
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms33 = [a.elapsed_time(b) for a, b in ev33]
    ms = float(np.sum(step_ms))
    if ws > 1:
        from paper_2605_03603_gb300 import dist as sd

        ms = sd.max_over_ranks(ms, group=gloo)
        ms33_tot = sd.max_over_ranks(float(np.sum(ms33)), group=gloo)
        keys = list(counts)
        totals = {str(k): v for k, v in
                  zip(keys, sd.allreduce_counts([counts[k] for k in keys], group=gloo))}
        tuples = dict(zip(keys, sd.allreduce_counts([tuples[k] for k in keys], group=gloo)))
        tuples_total = sum(tuples.values())
    else:
        ms33_tot = float(np.sum(ms33))
        totals = {str(k): v for k, v in counts.items()}
        tuples_total = sum(tuples.values())
    ms_per_step = ms / args.steps
    value = tuples_total / (ms_per_step / 1000.0)

    # rooflines of the step's kernels; "roofline" is the one with most time
    peaks, peak_kind = measured_peaks()
    nl = len(PQ)
    mean = lambda key: float(np.mean([sum(s[key] for s in sts) for sts in per_step_stats]))
    t_tup, t_hop, t_tc = mean("ms_tuples"), mean("ms_twohop"), mean("ms_tc")
    s_first = per_step_stats[0]
    popc = sum(s["popc_words"] for s in s_first)
    popc_peak = alu["popc_per_s"] / 1e12
    tup_ach = popc / (t_tup / 1000.0) / 1e12 if t_tup > 0 else 0.0
    roofs = {
        "k_tuples": {"kernel": "k_tuples (tuple enumeration, AND/POPC type counts)",
                     "bound": "alu", "achieved": tup_ach, "peak": popc_peak, "unit": "Tpopc/s",
                     "frac": tup_ach / popc_peak, "ms": t_tup, "launches": nl,
                     "traffic": TRAFFIC.get(("k_tuples", WORKLOAD)),
                     "peak_basis": f"POPC rate measured in this run by sbc_measure_alu_rates "
                                   f"({alu['popc_per_s'] / 1e12:.2f} T/s; LOP3 "
                                   f"{alu['lop3_per_s'] / 1e12:.2f} T/s)"},
    }
    kb = sum(s.get("tc_kblocks", 0) for s in s_first)
    if kb and t_tc > 0:
        flops = 2.0 * kb * 128 * 256 * 128
        tc_ach = flops / (t_tc / 1000.0) / 1e12
        bf16 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0))
        tc_peak = 2.0 * bf16  # fp8 dense = 2 x bf16 dense (nominal 4.5 / 2.25 PF)
        roofs["k_tcpairs"] = {
            "kernel": "k_zexpand + k_tcpairs (tensor-core pair counts, tcgen05 kind::f8f6f4)",
            "bound": "tensor", "achieved": tc_ach, "peak": tc_peak, "unit": "TFLOP/s",
            "frac": tc_ach / tc_peak, "ms": t_tc, "traffic": TRAFFIC.get(("k_tcpairs", WORKLOAD)),
            "flops_per_step": flops, "tiles": sum(s.get("tc_tiles", 0) for s in s_first),
            "peak_basis": "2 x measured sustained bf16 TFLOP/s (fp8 is twice bf16 nominally)"}
    # 2-hop: one 4-byte B entry per visited wedge + A_ent, A_pos and the bit
    # index of every anchor-side edge (12 B per edge)
    hop_bytes = sum(4 * s["wedges"] + 12 * g.m for s in s_first)
    hop_gbs = hop_bytes / (t_hop / 1000.0) / 1e9
    roofs["k_twohop"] = {"kernel": "k_twohop_large + k_twohop_small (2-hop candidates)",
                         "bound": "hbm", "achieved": hop_gbs, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": hop_gbs / peaks["hbm_gbs"], "ms": t_hop,
                         "traffic": TRAFFIC.get(("k_twohop", WORKLOAD)),
                         "bytes_per_step": int(hop_bytes),
                         "entries_read_per_wedge": (sum(s["twohop_reads"] for s in s_first)
                                                    / max(1, sum(s["wedges"] for s in s_first)))}
    dominant = max(roofs, key=lambda k: roofs[k]["ms"])
    roof = dict(roofs[dominant])
    roof["share_of_step"] = roof["ms"] / float(np.mean(step_ms))

    # end to end through the public API with pinned host buffers
    h_off = torch.from_numpy(g.offsets).pin_memory()
    h_col = torch.from_numpy(g.cols).pin_memory()
    h_sgn = torch.from_numpy(g.signs).pin_memory()
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, args.e2e_steps))
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(e2e_steps)]
    with torch.cuda.stream(stream):
        for i in range(e2e_steps):
            flush.zero_()
            e2e_ev[i][0].record(stream)
            with sbc.sbc_graph_create(g.n_u, g.n_v, h_off, h_col, h_sgn, stream=stream) as h:
                for p, q in PQ:
                    c, _, _ = sbc.sbc_count_ex(h, p, q, stream=stream, **shard)
                    assert c == counts[(p, q)]
            e2e_ev[i][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = float(np.mean([a.elapsed_time(b) for a, b in e2e_ev])) if e2e_ev else float("nan")
    if ws > 1:
        e2e_ms = sd.max_over_ranks(e2e_ms, group=gloo)
    h2d = g.offsets.nbytes + g.cols.nbytes + g.signs.nbytes
    e2e = {"value": tuples_total / (e2e_ms / 1000.0), "unit": "anchor tuples/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 16 * len(PQ),
           "ms_per_step": e2e_ms, "steps": e2e_steps}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle

        side = anchor_side(g)
        p, q = PQ[0]
        with oracle.Prepared(g, side) as prep:
            tup, dt, na, cores = oracle_sample(prep, g, side, p, q, args.cpu_frac, 7)
            # the same oracle on one thread, on a tenth of the sample
            tup1, dt1, na1, _ = oracle_sample(prep, g, side, p, q, args.cpu_frac / 10, 8, threads=1)
        cpu = {"value": tup / dt, "unit": "anchor tuples/s", "cores": cores, "kind": "oracle",
               "sample": f"({p},{q}) on a seeded random {args.cpu_frac:.3%} sample of "
                         f"{'U' if side == 0 else 'V'} anchors ({na} anchors, {tup} tuples, "
                         f"{dt:.1f} s; graph lists built once beforehand)",
               "seconds_to_exact_33_estimate": dt / args.cpu_frac,
               "one_thread": {"value": tup1 / dt1 if dt1 > 0 else None, "cores": 1,
                              "sample": f"{args.cpu_frac / 10:.4%} of the anchors "
                                        f"({na1} anchors, {tup1} tuples, {dt1:.1f} s)"}}

    medium = batch = serve = sweep = dyn = None
    if rank == 0 and ws == 1 and args.pq_sweep:
        sweep = _leg(pq_sweep_leg, sbc, torch, args)
    if rank == 0 and ws == 1 and not args.no_medium:
        medium = _leg(medium_leg, sbc, torch, args)
    if rank == 0 and ws == 1 and args.dyn_updates > 0:
        dyn = _leg(dynamic_leg, sbc, torch, args)
    if rank == 0 and ws == 1 and args.batch_graphs > 0:
        batch = _leg(batch_leg, sbc, torch, args)
    if rank == 0 and ws == 1 and args.serve_requests > 0:
        serve = _leg(serve_leg, sbc, torch, args)

    if rank == 0:
        s0 = per_step_stats[0]
        line = {
            "metric": METRIC, "value": value, "unit": "anchor tuples/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "u32/u64 integer masks, fp8 0/1 tensor-core operands (exact u128 counts)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "pq": "+".join(f"({p},{q})" for p, q in PQ),
                       "n_u": g.n_u, "n_v": g.n_v, "edges": g.m,
                       "input_sha256": input_digest,
                       "l2": "inputs (1.1 GB on the device) larger than L2, and flushed "
                             "between steps (512 MiB write)",
                       "parallelism": f"anchor shards x{ws}" if ws > 1 else "1 GPU"},
            "seconds_to_exact_33": ms33_tot / args.steps / 1000.0,
            "counts": totals, "anchor_tuples": {str(k): v for k, v in tuples.items()},
            "phase_ms": {"tuples": t_tup, "tensor_core_pairs": t_tc, "twohop": t_hop,
                         "other": float(np.mean(step_ms)) - t_tup - t_tc - t_hop},
            "tuples_tested": [s["tuples_tested"] for s in s0],
            "tuples_typed": [s["tuples_typed"] for s in s0],
            "tc_anchors": [s.get("tc_anchors", 0) for s in s0],
            "roofline": roof, "roofline_kernels": roofs, "peak_source": peak_kind,
            "alu_rates": alu, "clocks": clocks, "gpu_launches": int(launches), "e2e": e2e,
            "cpu_baseline": cpu, "medium": medium, "batch": batch, "serve": serve,
            "pq_sweep": sweep, "dynamic": dyn,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_profile_target(args):
    """Plain counts of the workload (no timing contract): the command the
    ncu summaries under profiles/ were taken with. Prints each count's
    statistics."""
    import torch

    import paper_2605_03603_gb300 as sbc

    torch.cuda.set_device(0)
    g = load_workload()
    side = {"auto": -1, "U": 0, "V": 1}[args.side]
    with sbc.graph_from_synth(g, device=True) as h:
        for _ in range(args.steps):
            for p, q in PQ:
                c, st, _ = sbc.sbc_count_ex(h, p, q, anchor_side=side)
                print(json.dumps({"workload": WORKLOAD, "pq": f"({p},{q})", "count": c,
                                  **{k: st[k] for k in ("anchor_side", "ms_total", "ms_twohop",
                                                        "ms_tuples", "ms_tc", "wedges",
                                                        "popc_words", "tc_tiles",
                                                        "tc_kblocks")}}), flush=True)
    return 0


def main():
    global PQ, WORKLOAD
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-medium", action="store_true", help="skip the 2M-edge leg")
    ap.add_argument("--pq-sweep", action="store_true",
                    help="also time p in {3,4,5} x q in {3..7} on the 20k- and 2M-edge graphs")
    ap.add_argument("--dyn-updates", type=int, default=200,
                    help="random edge insertions of the dynamic-count leg (0: skip the leg)")
    ap.add_argument("--batch-graphs", type=int, default=10000,
                    help="graphs of the batch leg (0 skips it; the full recipe is 10000)")
    ap.add_argument("--serve-graphs", type=int, default=500)
    ap.add_argument("--serve-max-edges", type=float, default=1e6,
                    help="largest graph of the serving leg (the recipe's 1e7-edge graphs take "
                         "minutes to hours per (4,4) request)")
    ap.add_argument("--serve-requests", type=int, default=50000,
                    help="most requests per rate (0 skips the serving leg)")
    ap.add_argument("--serve-seconds", type=float, default=1.0,
                    help="arrival span per rate: requests = min(serve-requests, rate x this)")
    ap.add_argument("--serve-rates", type=float, nargs="+",
                    default=[50.0, 100.0, 150.0, 300.0, 1000.0, 5000.0, 20000.0])
    ap.add_argument("--serve-budget-gb", type=float, default=80.0)
    ap.add_argument("--serve-baseline-requests", type=int, default=2000,
                    help="requests (a prefix of each rate's arrivals) served one at a time")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS),
                    help="graph to count (default: the 5M x 1M x 60M workload)")
    ap.add_argument("--pq", action="append", default=None,
                    help="p,q pair to count (repeatable); default 3,3")
    ap.add_argument("--cpu-frac", type=float, default=0.0005,
                    help="anchor sample fraction for the oracle CPU baseline")
    ap.add_argument("--ref-frac", type=float, default=0.0001,
                    help="anchor sample fraction per step for --impl reference")
    ap.add_argument("--profile-target", action="store_true",
                    help="only run --steps plain counts of the workload (for ncu)")
    ap.add_argument("--side", choices=["auto", "U", "V"], default="auto",
                    help="anchor side of --profile-target counts")
    args = ap.parse_args()
    WORKLOAD = args.workload
    if args.pq:
        PQ = [tuple(int(x) for x in pq.split(",")) for pq in args.pq]
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_target:
        return run_profile_target(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
