"""Writes tests/golden/p630_lif_pbs_1000.txt from the oracle alone.

1000 multi-value bootstraps at P630 (n=630, N=1024, Bg=2^7 l=3, ks 2^2 x 7,
p=64), the configuration the conv-SNN benchmark runs: keys from seed 2, the
LIF table pair of 4.2 (FHE-Fire and FHE-Reset as one blind rotation with two
outputs; threshold 8, leak = right shift by 1, spike 1) and input messages
uniform over all of Z_2p = {0..127} (seed 6, encryption seed 6), so both the
positive half and the negacyclic half of the test polynomial are hit.  Each
line holds the index and, per output table, the first 16 hex digits of the
SHA-256 of the output ciphertext (uint32 little-endian words).  The GPU tests
compare both integer blind-rotation paths against these lines, ciphertext by
ciphertext.

Usage: python tests/golden/make_p630_lif_pbs_hashes.py   (about 6 CPU-core-hours / cores)
"""
import hashlib
import os
import sys

import numpy as np

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))

from oracle import oracle as O  # noqa: E402
from paper_2309_09025_gb300 import synth  # noqa: E402

COUNT = 1000
KEY_SEED = 2
MSG_SEED = 6


def main():
    P = dict(synth.P630)
    p = 1 << P["log2_p"]
    keys = O.keygen(P, KEY_SEED)
    m = synth.uniform_messages(MSG_SEED, COUNT, 2 * p)
    ct = O.encrypt(P, keys, m, MSG_SEED)
    lif = synth.LIF_DEFAULT
    luts = O.lif_luts(P, lif["v_th"], lif["leak_shift"], lif["spike_scale"])
    out = O.pbs(P, keys, ct, luts, nthreads=os.cpu_count())
    path = os.path.join(os.path.dirname(__file__), "p630_lif_pbs_1000.txt")
    with open(path, "w") as f:
        f.write("# oracle multi-value bootstraps at P630 (keys seed 2; messages uniform in Z_128 and\n")
        f.write("# encryption seed 6; LIF Fire/Reset pair, V_th 8, leak >>1): index, then per table the\n")
        f.write("# first 16 hex digits of SHA-256 of the output LWE (uint32 LE words)\n")
        for i in range(COUNT):
            hs = [hashlib.sha256(np.ascontiguousarray(out[j, i], dtype="<u4").tobytes()).hexdigest()[:16]
                  for j in range(out.shape[0])]
            f.write("%d %s\n" % (i, " ".join(hs)))
    print("wrote", path)


if __name__ == "__main__":
    main()
