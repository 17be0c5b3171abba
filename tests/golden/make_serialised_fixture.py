"""Writes serialised_l8_rotation.txt: a small function built by the oracle,
in the serialised form that include/mphf.h lays out (16 header words, the
Golomb-Rice words, the Elias-Fano words), with its keys and their values.

Only the oracle computes anything here; the keys come from the seeded
generator module.  Run from the repository root:

    python tests/golden/make_serialised_fixture.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

from oracle import oracle as O  # noqa: E402
from paper_2212_09562_b300 import workloads as W  # noqa: E402
from helpers import oracle_blob  # noqa: E402

N, LEAF, BUCKET, KEY_BYTES, BIJ, TREE, SEED = 240, 8, 100, 8, O.ROTATION, O.TREE_RECSPLIT, 2212


def main():
    O.build()
    keys = W.random_keys(N, KEY_BYTES, SEED)
    o = O.build_mphf(keys, LEAF, BUCKET, BIJ, tree=TREE)
    blob = oracle_blob(o, LEAF, BUCKET, KEY_BYTES, BIJ, TREE)
    words = np.frombuffer(blob, np.uint64)
    values = o.query(keys)
    out = os.path.join(HERE, "serialised_l8_rotation.txt")
    with open(out, "w") as f:
        f.write("# A function over 240 keys (l = 8, b = 100, rotation fitting, RecSplit tree),\n")
        f.write("# built by the oracle (Section 2.2 construction, Section 4 leaves) and written\n")
        f.write("# in the serialised form of include/mphf.h.  Written by\n")
        f.write("# tests/golden/make_serialised_fixture.py from the oracle alone.\n")
        f.write(f"# params n={N} leaf={LEAF} bucket={BUCKET} key_bytes={KEY_BYTES} "
                f"bijection={BIJ} tree={TREE} seed={SEED}\n")
        f.write(f"words {len(words)}\n")
        for w in words:
            f.write(f"{int(w):016x}\n")
        f.write(f"keys {N}\n")
        for k, v in zip(keys, values):
            f.write(f"{int(k):016x} {int(v)}\n")
    print(out)


if __name__ == "__main__":
    main()
