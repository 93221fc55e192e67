"""The synthetic workloads are reproducible: every named workload hashes to
the digest recorded in tests/golden/input_digests.txt (written from the
generator by tests/golden/write_input_digests.py)."""
import os

import pytest

import sbc_synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "input_digests.txt")


def recorded():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, edges, digest = line.split()
            out[name] = (int(edges), digest)
    return out


@pytest.mark.parametrize("name", sorted(recorded()))
def test_workload_digest(name):
    edges, digest = recorded()[name]
    g = getattr(sbc_synth, name)()
    assert g.m == edges
    assert sbc_synth.digest(g) == digest


def test_digest_sees_one_flipped_sign():
    g = sbc_synth.plain_small()
    d0 = sbc_synth.digest(g)
    g.signs[123] = -g.signs[123]
    assert sbc_synth.digest(g) != d0
