"""Write the stored Oracle B answers of the Dyck-4 Zipf workload.

For each n given on the command line this draws the Dyck-4 workload's graph
(``workloads.dyck_zipf(n)``: Zipf(2.1) out-degrees truncated for mean 3,
uniform targets, labels uniform over o1..o4, c1..c4), runs Oracle B (the
worklist CFL-reachability solver of ``oracle/``) on it, and records in
``dyck4_zipf_oracle_b.json``:

* ``graph_sha256``: SHA-256 of the edge list (src, label, dst as
  little-endian uint32 arrays, in that order), so a test can tell that it
  regenerated the same graph;
* ``pairs``: the number of pairs of Sum_S (Theorem 1's answer for S);
* ``answer_sha256``: SHA-256 of the answer's bit rows (n rows of ceil(n/64)
  little-endian uint64 words, bit y of row x = word y/64, bit y%64);
* ``block_sha1``: SHA-1 of every 256-row slice of those bit rows, so a
  mismatch names the rows that differ.

Only the oracle and the input generator are called.  Usage:
``python tests/golden/make_dyck_golden.py 8192 16384`` (Oracle B takes about
1 min at n = 8192, 8 min at 16384 and an hour at 32768 on one core).
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2103_14688_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "dyck4_zipf_oracle_b.json")
BLOCK = 256


def graph_sha256(g) -> str:
    h = hashlib.sha256()
    for a in (g.src, g.lbl, g.dst):
        h.update(np.ascontiguousarray(np.asarray(a, dtype="<u4")).tobytes())
    return h.hexdigest()


def answer_digests(words: np.ndarray):
    """words: uint64 [n, ceil(n/64)] -> (sha256 of all rows, sha1 per 256 rows)."""
    w = np.ascontiguousarray(words.astype("<u8"))
    blocks = [hashlib.sha1(w[i:i + BLOCK].tobytes()).hexdigest() for i in range(0, w.shape[0], BLOCK)]
    return hashlib.sha256(w.tobytes()).hexdigest(), blocks


def main(ns):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {
        "what": "Oracle B answers (Sum_S) of the Dyck-4 Zipf workload, stored as hashes",
        "script": "tests/golden/make_dyck_golden.py", "block_rows": BLOCK, "cases": {}}
    for n in ns:
        g, r = W.dyck_zipf(n)
        t0 = time.perf_counter()
        words = oracle.worklist_words(g, r)[0]
        dt = time.perf_counter() - t0
        full, blocks = answer_digests(words)
        pairs = int(sum(int(x).bit_count() for x in words.ravel()))
        # re-read before writing: several sizes may run side by side
        data = json.load(open(OUT)) if os.path.exists(OUT) else data
        data["cases"][str(n)] = {"n": n, "m": g.m, "graph_sha256": graph_sha256(g), "pairs": pairs,
                                 "answer_sha256": full, "block_sha1": blocks, "oracle_seconds": round(dt, 1)}
        tmp = OUT + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1)
        os.replace(tmp, OUT)
        print(n, g.m, pairs, f"{dt:.1f}s", flush=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [8192, 16384])
