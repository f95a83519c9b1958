// Test driver for the host side of path extraction (Sec. 3.2, Listing 2):
// runs the library's enumerator (cfpq_paths_host.h) on the CPU, with the
// backward layers that the device computes in the library emulated here
// from their definition:
//   layer k = product vertices (s, x) from which some (f, y), f final in the
//   target's box, is reached over a path of M3 spelling at most k graph
//   edges, a nonterminal edge x -> z counting 1 edge when x != z and 0 when
//   x == z.
// Built by tests/test_paths_host.py with g++; test infrastructure only.
#include <stdint.h>

#include <cstdlib>
#include <cstring>
#include <vector>

#include "cfpq_paths_host.h"

namespace {

struct Rsm {
    uint32_t Q = 0, B = 0;
    std::vector<uint32_t> box_start, state_box;
    std::vector<uint8_t> final_;
    struct Tr {
        uint32_t from, kind, sym, to;
    };
    std::vector<Tr> tr;
};

}  // namespace

extern "C" int phd_paths(uint32_t n, uint64_t m, const uint32_t *tri, uint32_t Q, uint32_t B,
                         const uint32_t *box_start, const uint32_t *state_box, const uint8_t *fin, uint32_t T,
                         const uint32_t *tr_from, const uint32_t *tr_kind, const uint32_t *tr_sym,
                         const uint32_t *tr_to, const uint64_t *m2, uint32_t nq, const uint32_t *queries,
                         uint32_t *edges_out, uint64_t edge_cap, uint64_t *offs, uint64_t path_cap,
                         uint64_t *paths_per_query) {
    Rsm r;
    r.Q = Q;
    r.B = B;
    r.box_start.assign(box_start, box_start + B);
    r.state_box.assign(state_box, state_box + Q);
    r.final_.assign(fin, fin + Q);
    for (uint32_t i = 0; i < T; ++i) r.tr.push_back({tr_from[i], tr_kind[i], tr_sym[i], tr_to[i]});
    const size_t wn = (n + 63) / 64;
    cfpq::PathEnum<Rsm> P;
    P.r = &r;
    P.n = n;
    P.wn = wn;
    // a test can shrink the distance caches to a few entries (their eviction)
    if (const char *e = std::getenv("PHD_DIST_CACHE_ENTRIES")) P.dist_cache_bytes = (size_t)std::atoi(e) * n * 2;
    P.Qd = Q;
    P.Wd = (uint32_t)wn;
    P.eoff.assign(n + 1, 0);
    for (uint64_t i = 0; i < m; ++i) {
        P.es.push_back(tri[3 * i]);
        P.el.push_back(tri[3 * i + 1]);
        P.ed.push_back(tri[3 * i + 2]);
        P.eoff[tri[3 * i] + 1]++;
    }
    for (uint32_t v = 0; v < n; ++v) P.eoff[v + 1] += P.eoff[v];
    P.m2.resize(B);
    for (uint32_t b = 0; b < B; ++b) P.m2[b].assign(m2 + (size_t)b * n * wn, m2 + (size_t)(b + 1) * n * wn);

    auto bit = [&](const std::vector<uint64_t> &S, uint32_t s, uint32_t x) {
        return (S[(size_t)s * wn + (x >> 6)] >> (x & 63u)) & 1ull;
    };
    auto set = [&](std::vector<uint64_t> &S, uint32_t s, uint32_t x) {
        S[(size_t)s * wn + (x >> 6)] |= 1ull << (x & 63u);
    };
    auto diag = [&](uint32_t b, uint32_t z) { return (P.m2[b][(size_t)z * wn + (z >> 6)] >> (z & 63u)) & 1ull; };
    auto zero_close = [&](std::vector<uint64_t> &S) {
        for (bool ch = true; ch;) {
            ch = false;
            for (const auto &t : r.tr)
                if (t.kind)
                    for (uint32_t z = 0; z < n; ++z)
                        if (bit(S, t.to, z) && !bit(S, t.from, z) && diag(t.sym, z)) {
                            set(S, t.from, z);
                            ch = true;
                        }
        }
    };
    uint32_t L = 0;
    auto layers_of = [&](uint32_t N, uint32_t y, std::vector<uint64_t> *out) {
        const size_t words = (size_t)Q * wn;
        out->assign((size_t)(L + 1) * words, 0);
        std::vector<uint64_t> S(words, 0);
        for (uint32_t f = 0; f < Q; ++f)
            if (r.state_box[f] == N && r.final_[f]) set(S, f, y);
        zero_close(S);
        std::memcpy(out->data(), S.data(), words * 8);
        for (uint32_t k = 1; k <= L; ++k) {
            std::vector<uint64_t> S2 = S;
            for (const auto &t : r.tr) {
                if (t.kind == 0) {
                    for (uint64_t e = 0; e < m; ++e)
                        if (P.el[e] == t.sym && bit(S, t.to, P.ed[e])) set(S2, t.from, P.es[e]);
                } else {
                    for (uint32_t x = 0; x < n; ++x)
                        for (uint32_t z = 0; z < n; ++z)
                            if (x != z && ((P.m2[t.sym][(size_t)x * wn + (z >> 6)] >> (z & 63u)) & 1ull) &&
                                bit(S, t.to, z))
                                set(S2, t.from, x);
                }
            }
            zero_close(S2);
            S = S2;
            std::memcpy(out->data() + (size_t)k * words, S.data(), words * 8);
        }
    };
    P.fetch = [&](const std::vector<std::pair<uint32_t, uint32_t>> &ts, std::vector<std::vector<uint64_t>> *out) {
        out->resize(ts.size());
        for (size_t i = 0; i < ts.size(); ++i) layers_of(ts[i].first, ts[i].second, &(*out)[i]);
        return 0;
    };

    uint64_t np = 0, ne = 0;
    offs[0] = 0;
    for (uint32_t qi = 0; qi < nq; ++qi) {
        const uint32_t box = queries[4 * qi], vs = queries[4 * qi + 1], vf = queries[4 * qi + 2];
        const uint32_t max_len = queries[4 * qi + 3];
        // as in the library: layers of the largest bound asked so far
        if (max_len > P.Lmax) {
            P.Lmax = max_len;
            P.lay.clear();
            P.wanted.clear();
            P.fdist.clear();
        }
        L = P.Lmax;
        P.over = false;
        uint64_t here = 0;
        const bool reach = (P.m2[box][(size_t)vs * wn + (vf >> 6)] >> (vf & 63u)) & 1ull;
        for (uint32_t len = 0; reach && len <= max_len; ++len) {
            P.get(box, vs, vf, len);
            P.solve();
            if (P.over) return -2;
            for (const auto &p : P.memo[std::make_tuple(box, vs, vf, len)]) {
                if (np == path_cap) return -3;
                for (uint32_t e : p) {
                    if (ne == edge_cap) return -3;
                    edges_out[3 * ne] = P.es[e];
                    edges_out[3 * ne + 1] = P.el[e];
                    edges_out[3 * ne + 2] = P.ed[e];
                    ++ne;
                }
                offs[++np] = ne;
                ++here;
            }
        }
        paths_per_query[qi] = here;
    }
    return 0;
}

// The enumerator's table of word lengths: out[b * (L + 1) + j] = 1 iff box b
// derives a word of j terminals (j <= L).
extern "C" int phd_word_lengths(uint32_t Q, uint32_t B, const uint32_t *box_start, const uint32_t *state_box,
                                const uint8_t *fin, uint32_t T, const uint32_t *tr_from, const uint32_t *tr_kind,
                                const uint32_t *tr_sym, const uint32_t *tr_to, uint32_t L, uint8_t *out) {
    Rsm r;
    r.Q = Q;
    r.B = B;
    r.box_start.assign(box_start, box_start + B);
    r.state_box.assign(state_box, state_box + Q);
    r.final_.assign(fin, fin + Q);
    for (uint32_t i = 0; i < T; ++i) r.tr.push_back({tr_from[i], tr_kind[i], tr_sym[i], tr_to[i]});
    cfpq::PathEnum<Rsm> P;
    P.r = &r;
    P.Lmax = L;
    P.word_lengths();
    for (uint32_t b = 0; b < B; ++b)
        for (uint32_t j = 0; j <= L; ++j) out[(size_t)b * (L + 1) + j] = P.words[b][j];
    return 0;
}
