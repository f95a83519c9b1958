"""The oracle's pins catch plausible mistakes: each case plants one mistake
in a copy of oracle/cfpq_oracle.c (a dropped rule, a transposed index, an
off-by-one bound, ...), and the CPU pin tests run against that copy must
fail.  The copy lives in a temporary directory; the oracle itself is not
touched."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_pins.py", "tests/test_golden_files.py", "tests/test_paths_host.py"]

# (what the mistake is, text of the oracle, the mistaken text)
MISTAKES = [
    ("Oracle A without the epsilon rule (Listing 1)",
     "        if (state_final[box_start[b]])\n            for (uint32_t i = 0; i < n; ++i) bset(M2ROW(n_term + b, i), i);",
     "        if (0 && state_final[box_start[b]])\n            for (uint32_t i = 0; i < n; ++i) bset(M2ROW(n_term + b, i), i);"),
    ("Oracle A with the Kronecker blocks transposed",
     "bset(M3 + ((uint64_t)s * n + x) * wN, (uint64_t)u * n + y)",
     "bset(M3 + ((uint64_t)u * n + x) * wN, (uint64_t)s * n + y)"),
    ("Oracle A with a reflexive closure",
     "            uint64_t sp = 0;\n            for (uint64_t e = off[u]; e < off[u + 1]; ++e) {",
     "            uint64_t sp = 0;\n            bset(row, u);\n            for (uint64_t e = off[u]; e < off[u + 1]; ++e) {"),
    ("Oracle A with a one-step closure",
     "            while (sp) {\n                uint32_t w = stack[--sp];",
     "            while (0 && sp) {\n                uint32_t w = stack[--sp];"),
    ("Oracle A extracting from non-final states",
     "                if (state_box[f] != b || !state_final[f]) continue;\n                for (uint32_t x = 0; x < n; ++x)",
     "                if (state_box[f] != b) continue;\n                for (uint32_t x = 0; x < n; ++x)"),
    ("Oracle A not counting the last iteration",
     "*out_iters = rc == 0 ? it : max_iter;", "*out_iters = rc == 0 ? it - 1 : max_iter;"),
    ("Oracle B never returning to waiting callers",
     "                        if (tr_kind[t] != ORC_NONTERM || tr_sym[t] != b) continue;\n                        uint64_t s2",
     "                        if (1) continue;\n                        uint64_t s2"),
    ("Oracle B accepting into the wrong box",
     "if (state_final[s]) ADD_SUM(state_box[s], x, y);", "if (state_final[s]) ADD_SUM(0, x, y);"),
    ("Oracle B calling at the entry vertex",
     "const uint64_t *sr = Sum + (b2 * n + y) * wn;", "const uint64_t *sr = Sum + (b2 * n + x) * wn;"),
    ("Oracle B reading terminals at the entry vertex",
     "uint64_t k = (uint64_t)tr_sym[t] * n + y;", "uint64_t k = (uint64_t)tr_sym[t] * n + x;"),
    ("Oracle B with the caller index transposed",
     "bset(PT + (_s * n + _y) * wn, _x);", "bset(PT + (_s * n + _x) * wn, _y);"),
    ("membership chart accepting the empty word in any state",
     "int v = (i == j) && r->state_final[s];", "int v = (i == j);"),
    ("membership chart with no empty callee",
     "for (uint32_t k = i; k <= j && !v; ++k)", "for (uint32_t k = i + 1; k <= j && !v; ++k)"),
    ("membership chart whose terminal step reads no symbol",
     "if (i < j && w[i] == r->tr_sym[t] && A[AIDX(to, i + 1, j)]) v = 1;",
     "if (i < j && w[i] == r->tr_sym[t] && A[AIDX(to, i, j)]) v = 1;"),
    ("Oracle C paths one edge short",
     "    if (len == d->max_len) return;\n    for (uint64_t e = d->E->off[v]; e < d->E->off[v + 1]; ++e) {\n        d->path[len]",
     "    if (len + 1 >= d->max_len) return;\n    for (uint64_t e = d->E->off[v]; e < d->E->off[v + 1]; ++e) {\n        d->path[len]"),
    ("Oracle C keeping duplicate edges",
     "if (k == 0 || cmp_triple(tr + 3 * e, tr + 3 * (k - 1)) != 0) {", "if (1) {"),
    ("Oracle C reach one edge short",
     "    if (len == d->max_len) return;\n    for (uint64_t e = d->E->off[v]; e < d->E->off[v + 1]; ++e) {\n"
     "        d->word[len] = d->E->el[e];\n        dfs_reach",
     "    if (len + 1 >= d->max_len) return;\n    for (uint64_t e = d->E->off[v]; e < d->E->off[v + 1]; ++e) {\n"
     "        d->word[len] = d->E->el[e];\n        dfs_reach"),
    ("closure rows holding their start vertex",
     "        uint64_t cur = start;", "        uint64_t cur = start;\n        bset(row, start);"),
    ("closure rows reading the wrong nonterminal row",
     "const uint64_t *mr = m2_nt + ((uint64_t)tr_sym[t] * n + x) * wn;",
     "const uint64_t *mr = m2_nt + ((uint64_t)tr_sym[t] * n + (x + 1) % n) * wn;"),
    ("closure rows ignoring terminal labels",
     "                        if (E.el[e] != tr_sym[t]) continue;\n                        uint64_t v = (uint64_t)to * n + E.ed[e];",
     "                        uint64_t v = (uint64_t)to * n + E.ed[e];"),
]


@pytest.mark.slow
@pytest.mark.parametrize("what,good,bad", MISTAKES, ids=[m[0] for m in MISTAKES])
def test_pins_catch_a_planted_mistake(tmp_path, what, good, bad):
    src = open(os.path.join(ROOT, "oracle", "cfpq_oracle.c")).read()
    assert src.count(good) == 1, "the text to change is not in the oracle any more"
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), pkg / "__init__.py")
    (pkg / "cfpq_oracle.c").write_text(src.replace(good, bad))
    # the copy comes first on the path: the working directory of `python -m`
    env = dict(os.environ, PYTHONPATH=ROOT)
    where = subprocess.run([sys.executable, "-c", "import oracle; print(oracle.__file__)"], cwd=tmp_path, env=env,
                           capture_output=True, text=True, check=True).stdout
    assert where.startswith(str(tmp_path)), where
    p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        "--rootdir", ROOT] + [os.path.join(ROOT, t) for t in PINS],
                       cwd=tmp_path, env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode == 1, f"the pins did not catch: {what}\n{p.stdout[-2000:]}"
