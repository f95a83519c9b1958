"""The stored Oracle B answers are the oracle's: a few of the cheapest
stored queries of every golden file are recomputed here with the oracle and
the input generator, and their hashes must equal the stored ones.  (The GPU
tests compare the CUDA path with every stored answer.)"""
import importlib.util
import json
import os

import pytest

import oracle
from paper_2103_14688_gb300 import workloads as W

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _script(name):
    spec = importlib.util.spec_from_file_location(name, os.path.join(HERE, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _mix():
    path = os.path.join(HERE, "mix_oracle_b.json")
    if not os.path.exists(path):
        pytest.skip("no stored answers of the batched and served workloads")
    return json.load(open(path))


def _cheapest(recs, count):
    """The `count` cheapest stored queries with a nonempty answer."""
    keep = [(v["oracle_seconds"], int(k)) for k, v in recs.items() if sum(v["pairs"]) > 0]
    return [i for _, i in sorted(keep)[:count]]


def test_batched_answers_are_oracle_b():
    gold = _mix()["batched"]
    if not gold:
        pytest.skip("no stored batched answers")
    mk = _script("make_mix_golden")
    qs = W.batched_queries(count=512)
    for i in _cheapest(gold, 6):
        g, r = qs[i]
        rec = gold[str(i)]
        assert mk.graph_sha256(g) == rec["graph_sha256"] and mk.rsm_sha256(r) == rec["rsm_sha256"]
        sha, pairs = mk.answer_digest(oracle.worklist_words(g, r))
        assert (sha, pairs) == (rec["answer_sha256"], rec["pairs"]), i


def test_served_answers_are_oracle_b():
    data = _mix()
    gold = data["served"]
    if not gold:
        pytest.skip("no stored served answers")
    mk = _script("make_mix_golden")
    wl = W.serving_workload(lam=100.0, n_queries=1, horizon_s=1.0)
    assert mk.graph_sha256(wl.graph) == data["served_graph_sha256"]
    for j in _cheapest(gold, 2):
        r = wl.pool[j]
        rec = gold[str(j)]
        assert mk.rsm_sha256(r) == rec["rsm_sha256"]
        sha, pairs = mk.answer_digest(oracle.worklist_words(wl.graph, r))
        assert (sha, pairs) == (rec["answer_sha256"], rec["pairs"]), j


def test_dyck_golden_graphs_are_the_generators():
    """The Dyck-4 answers take Oracle B minutes at n = 8192 and more, so only
    the stored graph hashes are recomputed here."""
    path = os.path.join(HERE, "dyck4_zipf_oracle_b.json")
    if not os.path.exists(path):
        pytest.skip("no stored Dyck-4 answers")
    gold = json.load(open(path))
    mk = _script("make_mix_golden")
    for n, case in gold["cases"].items():
        g, _ = W.dyck_zipf(int(n))
        assert mk.graph_sha256(g) == case["graph_sha256"], n
