"""Readers for the small text fixtures under tests/golden/."""
import os

import numpy as np

import sbc_synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line.split()


def expectations(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("# expect "):
                p, q, c = line[len("# expect "):].split()
                out.append((int(p), int(q), int(c)))
    return out


def butterflies():
    """[(panel, s11, s12, s21, s22, balanced)] of Figure 2."""
    return [(r[0], int(r[1]), int(r[2]), int(r[3]), int(r[4]), bool(int(r[5])))
            for r in _rows("fig2_butterflies.txt")]


def graph(name, n_u, n_v, signs=None):
    rows = list(_rows(name))
    u = np.array([int(r[0]) for r in rows])
    v = np.array([int(r[1]) for r in rows])
    if signs is None:
        s = np.array([int(r[2]) if len(r) > 2 else 1 for r in rows])
    else:
        s = np.asarray(signs)
    return sbc_synth.from_edges(n_u, n_v, u, v, s, name)
