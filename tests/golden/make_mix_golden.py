"""Write the stored Oracle B answers of the batched and served workloads.

* ``batched``: the 512 queries of ``workloads.batched_queries()`` (n uniform
  in [256, 8192], Erdos-Renyi graphs of mean out-degree 4 over 2-6 labels,
  generated RSMs of 3-24 states);
* ``served``: every RSM of the served pool (``workloads.serving_workload``:
  256 generated RSMs of 3-32 states) on its resident graph (n = 32768,
  Zipf(2.1) out-degrees, 8 labels).

For each query Oracle B (the worklist CFL-reachability solver of
``oracle/``) computes Sum_N of every box N; the file ``mix_oracle_b.json``
records per query:

* ``graph_sha256`` (batched only: the served graph's is stored once):
  SHA-256 of the edge list (src, label, dst as little-endian uint32 arrays);
* ``rsm_sha256``: SHA-256 of the RSM's arrays (n_states, n_boxes,
  start_box, box_start, state_box, state_final, transitions), so a test can
  tell that it regenerated the same query;
* ``pairs``: the number of pairs of every box's answer;
* ``answer_sha256``: SHA-256 of the answer's bit rows, box after box (n rows
  of ceil(n/64) little-endian uint64 words each, bit y of row x = word y/64,
  bit y%64).

Oracle B's time grows steeply with the density of the answer: a few batched
queries whose grammars make most pairs reachable take it hours.  Every query
runs in a process of its own; one still running after ``--max-seconds`` is
stopped and listed under ``too_slow_batched`` / ``too_slow_served`` (index,
n, states, the limit), and the tests check those answers otherwise (a
fixpoint of one more iteration at sampled rows).  A run resumes from the
queries an earlier run already stored.

Only the oracle and the input generator are called.  Usage:
``python tests/golden/make_mix_golden.py [--workers W] [--max-seconds S]``.
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import queue
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

OUT = os.path.join(HERE, "mix_oracle_b.json")


def graph_sha256(g) -> str:
    h = hashlib.sha256()
    for a in (g.src, g.lbl, g.dst):
        h.update(np.ascontiguousarray(np.asarray(a, dtype="<u4")).tobytes())
    return h.hexdigest()


def rsm_sha256(r) -> str:
    h = hashlib.sha256()
    h.update(np.asarray([r.n_states, r.n_boxes, r.start_box], dtype="<u4").tobytes())
    for a in (r.box_start, r.state_box, r.state_final, r.tr_from, r.tr_kind, r.tr_sym, r.tr_to):
        h.update(np.ascontiguousarray(np.asarray(a, dtype="<u4")).tobytes())
    return h.hexdigest()


def answer_digest(words: np.ndarray):
    """words: uint64 [B, n, ceil(n/64)] -> (sha256 of all boxes' rows, pairs per box)."""
    w = np.ascontiguousarray(words.astype("<u8"))
    pairs = [int(np.unpackbits(w[b].view(np.uint8)).sum()) for b in range(w.shape[0])]
    return hashlib.sha256(w.tobytes()).hexdigest(), pairs


def _worker(kind, i, g, r, out_q):
    import oracle
    t0 = time.perf_counter()
    full, pairs = answer_digest(oracle.worklist_words(g, r))
    rec = {"rsm_sha256": rsm_sha256(r), "pairs": pairs, "answer_sha256": full,
           "oracle_seconds": round(time.perf_counter() - t0, 2)}
    if kind == "batched":
        rec.update({"n": g.n, "m": g.m, "graph_sha256": graph_sha256(g)})
    out_q.put((kind, i, rec))


def _save(data):
    tmp = OUT + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=0, sort_keys=True)
    os.replace(tmp, OUT)


def main(workers: int, max_seconds: float):
    from paper_2103_14688_gb300 import workloads as W
    wl = W.serving_workload(lam=100.0, n_queries=1, horizon_s=1.0)
    qs = W.batched_queries(count=512)
    data = {"what": "Oracle B answers of every batched query and every served-pool query, stored as hashes",
            "script": "tests/golden/make_mix_golden.py", "served_graph_sha256": graph_sha256(wl.graph),
            "served_n": wl.graph.n, "batched": {}, "served": {}, "too_slow_batched": [], "too_slow_served": []}
    if os.path.exists(OUT):
        old = json.load(open(OUT))
        if old.get("served_graph_sha256") == data["served_graph_sha256"]:
            data["batched"], data["served"] = old.get("batched", {}), old.get("served", {})
    data["max_seconds"] = max_seconds
    # the served pool first, then the batched queries, largest first
    big = sorted(range(512), key=lambda i: -qs[i][0].n * qs[i][1].n_states)
    tasks = [("served", j) for j in range(len(wl.pool)) if str(j) not in data["served"]]
    tasks += [("batched", i) for i in big if str(i) not in data["batched"]]
    ctx = mp.get_context("spawn")
    out_q = ctx.Queue()
    running = {}  # (kind, i) -> (process, start time)
    t0 = time.perf_counter()
    done = 0
    while tasks or running:
        while tasks and len(running) < workers:
            kind, i = tasks.pop(0)
            g, r = qs[i] if kind == "batched" else (wl.graph, wl.pool[i])
            p = ctx.Process(target=_worker, args=(kind, i, g, r, out_q), daemon=True)
            p.start()
            running[(kind, i)] = (p, time.perf_counter())
        try:
            kind, i, rec = out_q.get(timeout=1.0)
        except queue.Empty:
            kind = None
        if kind is not None and (kind, i) in running:
            data[kind][str(i)] = rec
            running.pop((kind, i))[0].join()
            done += 1
            if done % 32 == 0:
                _save(data)
                print(f"{done} queries stored, {len(tasks)} queued, {time.perf_counter() - t0:.0f} s", flush=True)
        now = time.perf_counter()
        for key, (p, start) in list(running.items()):
            if p.exitcode not in (None, 0):
                raise RuntimeError(f"the oracle's process for {key} failed (exit code {p.exitcode})")
            if now - start > max_seconds and p.is_alive():
                p.terminate()
                p.join()
                running.pop(key)
                kind, i = key
                g, r = (qs[i] if kind == "batched" else (wl.graph, wl.pool[i]))
                data["too_slow_" + kind].append({"index": i, "n": g.n, "states": r.n_states,
                                                 "seconds_limit": max_seconds})
                print(f"{kind} query {i} (n = {g.n}, {r.n_states} states) stopped after {max_seconds:.0f} s",
                      flush=True)
    for kind in ("batched", "served"):
        data["too_slow_" + kind].sort(key=lambda e: e["index"])
    _save(data)
    print(f"done: {len(data['batched'])} batched, {len(data['served'])} served stored; too slow: "
          f"{len(data['too_slow_batched'])} batched, {len(data['too_slow_served'])} served", flush=True)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--max-seconds", type=float, default=1800.0)
    a = ap.parse_args()
    main(a.workers, a.max_seconds)
