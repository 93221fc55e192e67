"""Writes input_digests.txt: the SHA-256 (sbc_synth.digest) of every named
synthetic workload, from the generator alone. Run from the repository root:
python tests/golden/write_input_digests.py"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import sbc_synth  # noqa: E402

WORKLOADS = ["plain_small", "plain_quarter", "plain_medium", "dense_factions",
             "dense_factions_wide", "plain_large"]


def main():
    lines = ["# SHA-256 of each synthetic workload (sbc_synth.digest over n_u, n_v,",
             "# offsets, cols, signs), written by write_input_digests.py from the",
             "# generator alone. Columns: generator function, edges, digest."]
    for name in WORKLOADS:
        g = getattr(sbc_synth, name)()
        lines.append(f"{name} {g.m} {sbc_synth.digest(g)}")
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "input_digests.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
