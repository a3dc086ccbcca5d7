"""Writes tests/golden/p750_pbs_1000.txt from the oracle alone.

1000 bootstraps at P750 (n=750, N=2048, Bg=2^10 l=2, ks 2^2 x 7, p=64): keys
from seed 4, messages uniform in Z_64 (seed 4), encryption seed 4, the
identity-plus-threshold table (one test polynomial).  Each line holds the
index and the first 16 hex digits of the SHA-256 of the output ciphertext
(uint32 little-endian words).  The GPU test compares both integer
blind-rotation paths against these lines, ciphertext by ciphertext.

Usage: python tests/golden/make_p750_pbs_hashes.py   (about 30 CPU-core-hours / cores)
"""
import hashlib
import os
import sys

import numpy as np

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))

from oracle import oracle as O  # noqa: E402
from paper_2309_09025_gb300 import synth  # noqa: E402

COUNT = 1000
SEED = 4


def main():
    P = dict(synth.P750)
    p = 1 << P["log2_p"]
    keys = O.keygen(P, SEED)
    m = synth.uniform_messages(SEED, COUNT, p)
    ct = O.encrypt(P, keys, m, SEED)
    lut = synth.identity_plus_threshold_lut(p)[None]
    out = O.pbs(P, keys, ct, lut, nthreads=os.cpu_count())[0]
    path = os.path.join(os.path.dirname(__file__), "p750_pbs_1000.txt")
    with open(path, "w") as f:
        f.write("# oracle bootstraps at P750 (keys, messages and encryption seed 4; identity-plus-threshold\n")
        f.write("# table): index, first 16 hex digits of SHA-256 of the output LWE (uint32 LE words)\n")
        for i in range(COUNT):
            h = hashlib.sha256(np.ascontiguousarray(out[i], dtype="<u4").tobytes()).hexdigest()[:16]
            f.write("%d %s\n" % (i, h))
    print("wrote", path)


if __name__ == "__main__":
    main()
