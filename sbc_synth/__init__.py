"""Seeded synthetic signed bipartite graphs (input generation only).

This module is shared by the CPU oracle, the tests and the benchmark. It draws
graphs; it computes nothing of the counting method (no degrees orderings, no
wedges, no intersections, no binomials).

Graph model (Section 5 of the paper evaluates on real signed bipartite graphs
of power-law shape, Table 1; those datasets are not available, so seeded
synthetic graphs of the same shape stand in for them):

* Chung-Lu bipartite (sampled in C, synth.c): side sizes n_u, n_v, m distinct
  edges. Expected weights w_i proportional to (i+1)^(-1/(gamma-1)) on each
  side, scaled to sum m and clipped at a cap (the excess is redistributed by
  rescaling the unclipped weights). Each edge draws its U end proportional to
  w_U and its V end proportional to w_V; duplicates are rejected (first draw
  wins) until exactly m distinct edges exist.
* Vertex ids are then randomly permuted on both sides so that id order is not
  degree order.
* Signs (Section 3: every edge is + or -): planted factions, the sign of (u,v)
  is a faction affinity, flipped with probability `flip`.

Randomness: every draw is counter-based, SplitMix64 (Steele, Lea, Flood 2014;
the public-domain mixer by S. Vigna) over (seed, stream, index), so the graph
depends only on the arguments, never on library versions.
"""
from __future__ import annotations

import concurrent.futures
import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libsbc_synth.so")
_clib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C sampler (gcc -O2) into sbc_synth/_build/ (once per
    process; safe to call from several threads)."""
    with _lock:
        os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + f".tmp{os.getpid()}.{threading.get_ident()}"
            subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _c():
    global _clib
    if _clib is None:
        lib = ctypes.CDLL(build())  # build() serialises the compile
        vp, i64, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        lib.synth_chung_lu.restype = ctypes.c_int
        lib.synth_chung_lu.argtypes = [ctypes.c_uint64, i64, i64, i64, f64, f64, f64, f64, vp, vp]
        lib.synth_csr.restype = ctypes.c_int
        lib.synth_csr.argtypes = [i64, i64, vp, vp, vp, vp, vp, vp]
        _clib = lib
    return _clib

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to uint64 states."""
    with np.errstate(over="ignore"):
        z = (x + _GOLDEN).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _stream_key(seed: int, stream: int) -> np.uint64:
    s = splitmix64(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)]))[0]
    with np.errstate(over="ignore"):
        s = splitmix64(np.array([s ^ np.uint64(stream & 0xFFFFFFFFFFFFFFFF)]))[0]
    return np.uint64(s)


def random_u64(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n counter-based 64-bit draws: splitmix64(key(seed, stream) + golden*i)."""
    key = _stream_key(seed, stream)
    idx = np.arange(start, start + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return splitmix64(key + idx * _GOLDEN)


def uniform01(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n doubles in [0, 1) with 53 random bits each."""
    return (random_u64(seed, stream, n, start) >> np.uint64(11)).astype(np.float64) * (
        1.0 / 9007199254740992.0
    )


@dataclasses.dataclass
class SignedBipartite:
    """Signed bipartite graph as CSR over U (rows) with V column ids.

    offsets: int64[n_u+1]; cols: int32[m], sorted within each row;
    signs: int8[m] in {+1, -1}.
    """

    n_u: int
    n_v: int
    offsets: np.ndarray
    cols: np.ndarray
    signs: np.ndarray
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.cols.shape[0])

    def edges(self):
        """(u, v, sign) arrays in CSR order."""
        rows = np.repeat(np.arange(self.n_u, dtype=np.int64), np.diff(self.offsets))
        return rows, self.cols.astype(np.int64), self.signs

    def packed_sign_bits(self) -> np.ndarray:
        """Signs as 1 bit per edge (bit set = negative), little-endian bytes."""
        return np.packbits((self.signs < 0).astype(np.uint8), bitorder="little")


def from_edges(n_u: int, n_v: int, u, v, s, name: str = "") -> SignedBipartite:
    """Build a CSR (rows ascending in u, each row sorted by v) from edge
    arrays; no duplicate check."""
    u = np.ascontiguousarray(u, dtype=np.int64)
    v = np.ascontiguousarray(v, dtype=np.int64)
    s = np.ascontiguousarray(s, dtype=np.int8)
    m = u.shape[0]
    offsets = np.zeros(n_u + 1, dtype=np.int64)
    cols = np.zeros(m, dtype=np.int32)
    sgn = np.zeros(m, dtype=np.int8)
    if _c().synth_csr(n_u, m, u.ctypes.data, v.ctypes.data, s.ctypes.data, offsets.ctypes.data,
                      cols.ctypes.data, sgn.ctypes.data):
        raise MemoryError("CSR build failed")
    return SignedBipartite(n_u, n_v, offsets, cols, sgn, name)


def chung_lu_edges(seed, n_u, n_v, m, gamma_u, gamma_v, cap_u=None, cap_v=None):
    """m distinct (u, v) pairs of a bipartite Chung-Lu graph, ids permuted.

    Expected degrees (i+1)^(-1/(gamma-1)) per side, scaled to m and capped
    (default half the other side; excess spread by rescaling); endpoints drawn
    proportionally (U from stream 1, V from stream 2); duplicates rejected,
    first draw wins, until m distinct pairs; ids relabelled by random
    permutations (streams 3 and 4). Runs in C (synth.c)."""
    if m > n_u * n_v:
        raise ValueError("more edges than vertex pairs")
    cap_u = 0.5 * n_v if cap_u is None else cap_u
    cap_v = 0.5 * n_u if cap_v is None else cap_v
    u = np.empty(m, dtype=np.int64)
    v = np.empty(m, dtype=np.int64)
    rc = _c().synth_chung_lu(seed & 0xFFFFFFFFFFFFFFFF, n_u, n_v, m, float(gamma_u), float(gamma_v),
                             float(cap_u), float(cap_v), u.ctypes.data, v.ctypes.data)
    if rc == -2:
        raise RuntimeError("could not draw enough distinct edges")
    if rc != 0:
        raise MemoryError("sampler allocation failed")
    return u, v


def faction_signs(seed, u, v, n_u, n_v, flip, p_plus=0.5):
    """Two planted factions: label +1 with probability p_plus, sign = l_u*l_v,
    flipped with probability `flip`."""
    lu = np.where(uniform01(seed, 5, n_u) < p_plus, 1, -1).astype(np.int8)
    lv = np.where(uniform01(seed, 6, n_v) < p_plus, 1, -1).astype(np.int8)
    s = lu[u] * lv[v]
    f = uniform01(seed, 7, u.shape[0]) < flip
    return np.where(f, -s, s).astype(np.int8)


def affinity_signs(seed, u, v, n_u, n_v, flip, factions=4):
    """`factions` planted factions; a seeded random +-1 affinity matrix M gives
    sign(u,v) = M[f(u), f(v)], flipped with probability `flip`."""
    fu = (random_u64(seed, 8, n_u) % np.uint64(factions)).astype(np.int64)
    fv = (random_u64(seed, 9, n_v) % np.uint64(factions)).astype(np.int64)
    mat = np.where(uniform01(seed, 10, factions * factions) < 0.5, 1, -1).astype(np.int8)
    mat = mat.reshape(factions, factions)
    s = mat[fu[u], fv[v]]
    f = uniform01(seed, 7, u.shape[0]) < flip
    return np.where(f, -s, s).astype(np.int8)


# Probability of label +1 that gives about 75% positive edges at flip 0.15:
# P(same) * 0.85 + (1 - P(same)) * 0.15 = 0.75 with P(same) = pi^2 + (1-pi)^2.
_PI_75 = 0.5 * (1.0 + math.sqrt(1.0 - 2.0 * (1.0 - (0.75 - 0.15) / 0.70)))


def chung_lu_signed(seed, n_u, n_v, m, gamma_u, gamma_v, flip, p_plus=0.5,
                    cap_u=None, cap_v=None, name=""):
    u, v = chung_lu_edges(seed, n_u, n_v, m, gamma_u, gamma_v, cap_u, cap_v)
    s = faction_signs(seed, u, v, n_u, n_v, flip, p_plus)
    return from_edges(n_u, n_v, u, v, s, name)


def plain_small(seed: int = 1) -> SignedBipartite:
    """2,000 x 1,500, 20,000 edges, exponent 2.1 both sides, uniform factions,
    flip 0.1 (the small plain-path workload)."""
    return chung_lu_signed(seed, 2000, 1500, 20000, 2.1, 2.1, 0.1,
                           name="plain-2k-1.5k-20k")


def plain_medium(seed: int = 2) -> SignedBipartite:
    """200,000 x 100,000, 2,000,000 edges, exponents 2.0 (U) / 2.3 (V),
    two factions with about 75% positive edges, flip 0.15."""
    return chung_lu_signed(seed, 200_000, 100_000, 2_000_000, 2.0, 2.3, 0.15,
                           p_plus=_PI_75, name="plain-200k-100k-2M")


def plain_quarter(seed: int = 2) -> SignedBipartite:
    """The medium workload's shape at a quarter of its size: 50,000 x 25,000,
    500,000 edges (profiling case)."""
    return chung_lu_signed(seed, 50_000, 25_000, 500_000, 2.0, 2.3, 0.15,
                           p_plus=_PI_75, name="plain-50k-25k-500k")


def dense_factions(m: int = 3000, n: int = 400, density: float = 0.45, seed: int = 5,
                   flip: float = 0.05) -> SignedBipartite:
    """Dense random bipartite graph (each pair an edge with probability
    `density`) with planted two-faction signs, a fraction `flip` flipped:
    anchors with thousands of candidates over a few hundred positions (the
    tensor-core pair step's profiling case at the defaults)."""
    r = uniform01(seed, 21, m * n)
    f = uniform01(seed, 22, m * n)
    lab = uniform01(seed, 23, m + n)
    lu = np.where(lab[:m] < 0.5, -1, 1)
    lv = np.where(lab[m:] < 0.5, -1, 1)
    uu, vv = np.divmod(np.arange(m * n, dtype=np.int64), n)
    keep = r < density
    s = (lu[uu] * lv[vv] * np.where(f < flip, -1, 1)).astype(np.int8)
    return from_edges(m, n, uu[keep], vv[keep], s[keep], f"dense-{m}x{n}")


def plain_large(seed: int = 3) -> SignedBipartite:
    """5,000,000 x 1,000,000, 60,000,000 edges, exponents 2.4 (U) / 1.9 (V),
    V hubs capped at 50,000 expected degree; 4 planted factions, flip 0.2."""
    n_u, n_v, m = 5_000_000, 1_000_000, 60_000_000
    u, v = chung_lu_edges(seed, n_u, n_v, m, 2.4, 1.9, cap_u=0.5 * n_v, cap_v=50_000)
    s = affinity_signs(seed, u, v, n_u, n_v, 0.2)
    return from_edges(n_u, n_v, u, v, s, "plain-5M-1M-60M")


def _loguniform(r: float, lo: float, hi: float) -> float:
    return math.exp(math.log(lo) + r * (math.log(hi) - math.log(lo)))


def batch_graph_params(seed: int, i: int, m_lo: float, m_hi: float):
    """Shape parameters of graph i of a batch: edges log-uniform in [m_lo, m_hi],
    |U|:|V| log-uniform in [1/4, 4], |U|+|V| = ceil(m/6) (at least enough
    vertex pairs), exponent uniform in [1.9, 2.5], flip uniform in [0, 0.3]."""
    r = uniform01(seed, 1000 + i, 4)
    m = int(round(_loguniform(float(r[0]), m_lo, m_hi)))
    ratio = _loguniform(float(r[1]), 0.25, 4.0)
    nv_tot = max(int(math.ceil(m / 6.0)), 8)
    n_u = max(2, int(round(nv_tot * ratio / (1.0 + ratio))))
    n_v = max(2, nv_tot - n_u)
    while n_u * n_v < 2 * m:
        n_u += 1
        n_v += 1
    gamma = 1.9 + 0.6 * float(r[2])
    flip = 0.3 * float(r[3])
    return m, n_u, n_v, gamma, flip


def batch_graph(seed: int, i: int, m_lo: float = 500, m_hi: float = 500_000) -> SignedBipartite:
    """Graph i of a batch of independent signed Chung-Lu graphs."""
    m, n_u, n_v, gamma, flip = batch_graph_params(seed, i, m_lo, m_hi)
    sub = int(splitmix64(np.array([np.uint64(seed * 1_000_003 + i)]))[0] >> np.uint64(1))
    return chung_lu_signed(sub, n_u, n_v, m, gamma, gamma, flip,
                           name=f"batch-{seed}-{i}")


def tiny_random(seed: int, n_u: int, n_v: int, density: float, neg: float) -> SignedBipartite:
    """Dense tiny graph for brute-force checks: each pair is an edge with
    probability `density`, negative with probability `neg`."""
    r = uniform01(seed, 11, n_u * n_v)
    s = uniform01(seed, 12, n_u * n_v)
    uu, vv = np.divmod(np.arange(n_u * n_v, dtype=np.int64), n_v)
    keep = r < density
    sign = np.where(s < neg, -1, 1).astype(np.int8)
    return from_edges(n_u, n_v, uu[keep], vv[keep], sign[keep], f"tiny-{seed}")


def batch_graphs(seed: int, count: int, m_lo: float = 500, m_hi: float = 500_000,
                 threads: int = 0, start: int = 0):
    """Graphs start..start+count-1 of a batch, generated on host threads (the
    C sampler releases the interpreter lock)."""
    threads = threads or min(32, os.cpu_count() or 1)
    with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda i: batch_graph(seed, i, m_lo, m_hi), range(start, start + count)))


def dense_factions_wide() -> SignedBipartite:
    """dense_factions over 800 positions: anchors of about 360 useful
    positions (three 128-position blocks), the typical tensor-core tile of
    the 60M-edge graph's (3,3) count."""
    return dense_factions(n=800, seed=6)


def digest(g: SignedBipartite) -> str:
    """SHA-256 of a graph's content: n_u, n_v (int64), offsets (int64), cols
    (int32), signs (int8), little-endian, in that order. Equal digests mean
    the generator produced the same graph (on any machine)."""
    import hashlib

    h = hashlib.sha256()
    h.update(np.array([g.n_u, g.n_v], dtype="<i8").tobytes())
    h.update(np.ascontiguousarray(g.offsets, dtype="<i8").tobytes())
    h.update(np.ascontiguousarray(g.cols, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.signs, dtype="i1").tobytes())
    return h.hexdigest()
