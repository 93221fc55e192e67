"""CPU oracle for balanced (p,q)-biclique counting.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use it; the product path never imports it. It shares no code with
the CUDA path.

Independent counters:

* `count` -- plain C (`sbc_oracle.c`): every p-subset L of U with a common
  neighbourhood of at least q vertices, reached by a depth-first extension
  over common neighbourhoods, adds sum over classes of binom(|class|, q),
  the classes being the common neighbours grouped by their sign vector
  relative to L's first member (the characterisation of a balanced biclique
  by Lemma 1 and its converse, Section 4.2).
* `brute_count_c` -- the definition itself (Section 3, Definitions 1-4 and
  the problem statement) in plain C: every p-subset L of U and q-subset R of
  V, kept when L x R is complete and every butterfly in it has an even number
  of negative edges. Graphs of at most 64 vertices per side.
* `brute_count` -- the same definition in pure Python, for the tiniest cases.
* `bbwc_count` -- the wedge-centric method (BBWC, Algorithm 1, Section 4.2)
  in plain C (`sbc_bbwc.c`, its own library sharing no code with
  `sbc_oracle.c`): signed p-wedges of each anchor bucketed by type and
  anchor set, binom(wedges, q) per bucket. A second cross-check of `count`
  on graphs too large for brute force.

Convention (the problem statement takes p vertices from one partition and q
from the other): p vertices come from U (the CSR rows) and q from V.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
from math import comb

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsbc_oracle.so")
_BBWC_SRC = os.path.join(_HERE, "sbc_bbwc.c")
_BBWC_PATH = os.path.join(_BUILD, "libsbc_bbwc.so")
_lib = None
_bbwc = None


def _compile(src: str, lib: str, force: bool) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, src]
        )
        os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Compile the C oracle and the wedge-centric cross-check (gcc -O2
    -fopenmp) into oracle/_build/; returns the oracle's library path."""
    _compile(_BBWC_SRC, _BBWC_PATH, force)
    return _compile(_SRC, _LIB_PATH, force)


def _declare(lib):
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.sbc_oracle_count.restype = ctypes.c_int
    lib.sbc_oracle_count.argtypes = [
        ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p, ctypes.c_void_p,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
    ]
    lib.sbc_oracle_prepare.restype = ctypes.c_void_p
    lib.sbc_oracle_prepare.argtypes = [
        ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.c_int, ctypes.POINTER(ctypes.c_int),
    ]
    lib.sbc_oracle_count_prepared.restype = ctypes.c_int
    lib.sbc_oracle_count_prepared.argtypes = [
        ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p, ctypes.c_void_p,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
    ]
    lib.sbc_oracle_release.restype = None
    lib.sbc_oracle_release.argtypes = [ctypes.c_void_p]
    lib.sbc_oracle_brute.restype = ctypes.c_int
    lib.sbc_oracle_brute.argtypes = [
        ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.c_int, ctypes.c_int, u64p,
    ]
    lib.sbc_oracle_binom.restype = ctypes.c_int
    lib.sbc_oracle_binom.argtypes = [ctypes.c_int64, ctypes.c_int, u64p]
    lib.sbc_oracle_max_threads.restype = ctypes.c_int
    return lib


def mutant(n: int, outdir: str):
    """A copy of the oracle with planted mistake `n` (see ORACLE_MUTANT in
    sbc_oracle.c), for tests that show the pins catch it."""
    path = os.path.join(outdir, f"libsbc_oracle_mutant{n}.so")
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-shared", "-fPIC",
                           f"-DORACLE_MUTANT={n}", "-o", path, _SRC])
    return _declare(ctypes.CDLL(path))


def _load():
    global _lib
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _load_bbwc():
    global _bbwc
    if _bbwc is None:
        build()
        lib = ctypes.CDLL(_BBWC_PATH)
        lib.sbc_bbwc_count.restype = ctypes.c_int
        lib.sbc_bbwc_count.argtypes = [
            ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.POINTER(ctypes.c_uint64)]
        _bbwc = lib
    return _bbwc


def bbwc_count(g, p: int, q: int, side: int | None = None, threads: int = 0) -> int:
    """Balanced (p,q)-bicliques of `g` (p from U, q from V) by the
    wedge-centric method of Algorithm 1 (Section 4.2), on anchor side `side`
    (0 = U, 1 = V; default the smaller partition). Independent of `count`."""
    if side is None:
        side = default_side(g.n_u, g.n_v)
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    col = np.ascontiguousarray(g.cols, dtype=np.int32)
    sgn = np.ascontiguousarray(g.signs, dtype=np.int8)
    out = (ctypes.c_uint64 * 2)()
    rc = _load_bbwc().sbc_bbwc_count(g.n_u, g.n_v, off.ctypes.data, col.ctypes.data,
                                     sgn.ctypes.data, p, q, side, threads, out)
    if rc == 1:
        raise OverflowError("balanced biclique count exceeds 128 bits")
    if rc != 0:
        raise RuntimeError(f"wedge-centric count failed with code {rc}")
    return _u128(out[0], out[1])


def max_threads() -> int:
    return int(_load().sbc_oracle_max_threads())


def default_side(n_u: int, n_v: int) -> int:
    """Default side the sets L are drawn from: the smaller partition (ties: U),
    as Algorithm 2 does. 0 = U, 1 = V. The count is the same either way."""
    return 0 if n_u <= n_v else 1


def _u128(lo, hi) -> int:
    return int(lo) | (int(hi) << 64)


class Prepared:
    """The graph's lists built once for one anchor side, for repeated counts
    (for example, timed anchor samples of a large graph). Use as a context
    manager or call close()."""

    def __init__(self, g, side: int, lib=None):
        self.lib = _load() if lib is None else lib
        self.g = g
        self.side = side
        rc = ctypes.c_int(0)
        self._keep = (np.ascontiguousarray(g.offsets, dtype=np.int64),
                      np.ascontiguousarray(g.cols, dtype=np.int32),
                      np.ascontiguousarray(g.signs, dtype=np.int8))
        off, col, sgn = self._keep
        self.h = self.lib.sbc_oracle_prepare(g.n_u, g.n_v, off.ctypes.data, col.ctypes.data,
                                             sgn.ctypes.data, side, ctypes.byref(rc))
        if not self.h:
            raise RuntimeError(f"oracle prepare failed with code {rc.value}")

    def count(self, p: int, q: int, threads: int = 0, per_anchor: bool = False,
              with_tuples: bool = False, anchors=None, max_subsets: int = 0, skipped=None):
        """Same results as `count` (module function) on this side."""
        return _count_call(self.lib, self.g, self.side, p, q, threads, per_anchor, with_tuples,
                           anchors, max_subsets, skipped, prepared=self.h)

    def close(self):
        if self.h:
            self.lib.sbc_oracle_release(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def count(g, p: int, q: int, side: int | None = None, threads: int = 0,
          per_anchor: bool = False, with_tuples: bool = False, lib=None, anchors=None,
          max_subsets: int = 0, skipped=None):
    """Balanced (p,q)-bicliques of `g` (p from U, q from V).

    side: the partition S the sets L are drawn from (0 = U with set size p,
    1 = V with set size q); default the smaller partition. threads: OpenMP
    threads (0 = all). Returns the count (int); with per_anchor, also a list
    of each anchor's share (the bicliques whose S-member of lowest priority
    rho, Definition 4, it is; indexed by vertex id of S); with with_tuples,
    also sum over anchors u of binom(|C(u)|, |L|-1), C(u) the vertices of
    higher priority sharing at least the other side's size of neighbours
    with u (the number of subsets Algorithm 2 enumerates). anchors: optional
    iterable of S-vertex ids; only those anchors are processed. max_subsets
    (tests only): anchors with more such subsets are left out; their ids are
    added to the set `skipped` if given.
    """
    lib = _load() if lib is None else lib
    if side is None:
        side = default_side(g.n_u, g.n_v)
    return _count_call(lib, g, side, p, q, threads, per_anchor, with_tuples, anchors,
                       max_subsets, skipped)


def _count_call(lib, g, side, p, q, threads, per_anchor, with_tuples, anchors, max_subsets,
                skipped, prepared=None):
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    col = np.ascontiguousarray(g.cols, dtype=np.int32)
    sgn = np.ascontiguousarray(g.signs, dtype=np.int8)
    out = (ctypes.c_uint64 * 2)()
    tup = (ctypes.c_uint64 * 2)()
    n_s = g.n_u if side == 0 else g.n_v
    anc = np.zeros(2 * max(n_s, 1), dtype=np.uint64) if per_anchor else None
    skip = np.zeros(max(n_s, 1), dtype=np.uint8) if max_subsets else None
    mask = None
    if anchors is not None:
        mask = np.zeros(max(n_s, 1), dtype=np.uint8)
        mask[np.asarray(list(anchors), dtype=np.int64)] = 1
    anc_p = anc.ctypes.data if anc is not None else None
    mask_p = mask.ctypes.data if mask is not None else None
    skip_p = skip.ctypes.data if skip is not None else None
    if prepared is not None:
        rc = lib.sbc_oracle_count_prepared(prepared, p, q, threads, out, anc_p,
                                           ctypes.addressof(tup), mask_p, max_subsets, skip_p)
    else:
        rc = lib.sbc_oracle_count(g.n_u, g.n_v, off.ctypes.data, col.ctypes.data,
                                  sgn.ctypes.data, p, q, side, threads, out, anc_p,
                                  ctypes.addressof(tup), mask_p, max_subsets, skip_p)
    if skip is not None and skipped is not None:
        skipped.update(np.nonzero(skip)[0].tolist())
    if rc == 1:
        raise OverflowError("balanced biclique count term exceeds 128 bits")
    if rc != 0:
        raise RuntimeError(f"oracle failed with code {rc}")
    total = _u128(out[0], out[1])
    res = [total]
    if per_anchor:
        res.append([_u128(anc[2 * i], anc[2 * i + 1]) for i in range(n_s)])
    if with_tuples:
        res.append(_u128(tup[0], tup[1]))
    return res[0] if len(res) == 1 else tuple(res)


def brute_count_c(g, p: int, q: int, lib=None) -> int:
    """The definition by brute force in C (at most 64 vertices per side)."""
    lib = _load() if lib is None else lib
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    col = np.ascontiguousarray(g.cols, dtype=np.int32)
    sgn = np.ascontiguousarray(g.signs, dtype=np.int8)
    out = (ctypes.c_uint64 * 2)()
    rc = lib.sbc_oracle_brute(g.n_u, g.n_v, off.ctypes.data, col.ctypes.data, sgn.ctypes.data,
                              p, q, out)
    if rc != 0:
        raise RuntimeError(f"brute force failed with code {rc}")
    return _u128(out[0], out[1])


def binom(n: int, k: int) -> int:
    """The oracle's exact binomial (for pinning it against closed forms)."""
    out = (ctypes.c_uint64 * 2)()
    if _load().sbc_oracle_binom(n, k, out):
        raise OverflowError("binomial exceeds 128 bits")
    return _u128(out[0], out[1])


def butterfly_balanced(s11: int, s12: int, s21: int, s22: int) -> bool:
    """A butterfly is balanced when it has an even number of negative edges."""
    return sum(1 for s in (s11, s12, s21, s22) if s < 0) % 2 == 0


def brute_count(g, p: int, q: int) -> int:
    """Count by the definition: complete L x R with no unbalanced butterfly."""
    sign = {}
    rows, cols, sg = g.edges()
    for u, v, s in zip(rows.tolist(), cols.tolist(), sg.tolist()):
        sign[(u, v)] = s
    total = 0
    for L in itertools.combinations(range(g.n_u), p):
        common = None
        for u in L:
            nb = set(cols[g.offsets[u]:g.offsets[u + 1]].tolist())
            common = nb if common is None else common & nb
        if common is None or len(common) < q:
            continue
        for R in itertools.combinations(sorted(common), q):
            ok = True
            for (u1, u2) in itertools.combinations(L, 2):
                for (v1, v2) in itertools.combinations(R, 2):
                    if not butterfly_balanced(sign[(u1, v1)], sign[(u1, v2)],
                                              sign[(u2, v1)], sign[(u2, v2)]):
                        ok = False
                        break
                if not ok:
                    break
            if ok:
                total += 1
    return total


def unsigned_count(g, p: int, q: int) -> int:
    """(p,q)-bicliques ignoring signs: sum over p-subsets L of U of
    binom(|common neighbourhood of L|, q) (tiny graphs only)."""
    total = 0
    nbs = [set(g.cols[g.offsets[u]:g.offsets[u + 1]].tolist()) for u in range(g.n_u)]
    for L in itertools.combinations(range(g.n_u), p):
        common = set.intersection(*(nbs[u] for u in L))
        total += comb(len(common), q)
    return total
