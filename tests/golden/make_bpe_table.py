"""Write the 4096-merge BPE table used by the BPE workload.

The table is trained by the CPU oracle's trainer (reading C9) on the seeded
10,000,000-byte order-3 Markov corpus at 45% GC (seed 45).  Only ``synth``
(input bytes) and ``oracle`` are called.  Run from the repository root:

    python tests/golden/make_bpe_table.py
"""
import hashlib
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "bpe_merges_markov45_seed45_4096.txt")


def main():
    corpus = synth.bpe_training_corpus(seed=45, n=10_000_000)
    digest = hashlib.sha256(bytes(corpus)).hexdigest()
    t0 = time.time()
    merges = oracle.bpe_train(oracle.codes_of(bytes(corpus)), 4096)
    dt = time.time() - t0
    with open(OUT, "w") as f:
        f.write("# BPE merge table: rank r -> token id 4+r, base ids A0 C1 G2 T3.\n")
        f.write("# Trained by the CPU oracle (oracle_bpe_train, reading C9) on\n")
        f.write("# synth.bpe_training_corpus(seed=45, n=10_000_000): order-3 Markov, 45% GC.\n")
        f.write("# corpus sha256 %s ; %d merges ; written by make_bpe_table.py\n"
                % (digest, len(merges)))
        for l, r in merges.tolist():
            f.write("%d %d\n" % (l, r))
    print("wrote %s: %d merges in %.1f s" % (OUT, len(merges), dt))


if __name__ == "__main__":
    main()
