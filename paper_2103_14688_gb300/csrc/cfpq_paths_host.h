// cfpq_paths_host.h -- host enumeration of path extraction (Sec. 3.2, Listing 2).
//
// getPaths(vs, vf, N) follows product paths of M3 from (q0_N, vs) to (f, vf),
// f final in N's box; a product edge over a terminal is a graph edge, one over
// a nonterminal N' with M2^{N'}[v, v'] = 1 expands into getPaths(v, v', N').
// The sets are bounded by the number of graph edges (max_len) and computed as
// the least fixpoint of these equations over keys (N, x, y, length), so that
// recursion through nonterminals deriving the empty word terminates.
// The forward walk keeps a partial path of k edges ending at (s, v) only if
// (s, v) is in layer len - k of the backward search from the targets of
// (N, y), run on the device (PathsDev): the vertices that can still reach a
// target with the edges left; and, for RSMs with nonterminal transitions,
// only if the graph distance from v to y is at most len - k.  A nonterminal
// step v -> v2 asks for subpaths of j edges only from j = the graph distance
// from v to v2 on.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <deque>
#include <functional>
#include <map>
#include <set>
#include <tuple>
#include <unordered_map>
#include <unordered_set>
#include <utility>
#include <vector>

namespace cfpq {

// RSM: Q, box_start, state_box, final_ and tr (from, kind, sym, to; kind 0 =
// terminal) as in the engine's host copy of an RSM.
template <class RSM>
struct PathEnum {
    const RSM *r;
    uint32_t n;
    std::vector<uint32_t> es, el, ed;        // unique edges sorted by (src, label, dst)
    std::vector<uint32_t> eoff;              // per source vertex
    std::vector<std::vector<uint64_t>> m2;   // per box, n * wn words
    size_t wn;
    // Backward layers per target (N, y): (Lmax + 1) x Qd x Wd words.  The
    // targets of new keys are collected and fetched together the first time
    // one of them is needed (one device search for the batch).
    using Target = std::pair<uint32_t, uint32_t>;
    std::function<int(const std::vector<Target> &, std::vector<std::vector<uint64_t>> *)> fetch;
    std::map<Target, std::vector<uint64_t>> lay;
    std::set<Target> wanted;
    uint32_t Qd = 0, Wd = 0, Lmax = 0;
    int dev_rc = 0;

    const uint64_t *layers_for(uint32_t N, uint32_t y) {
        const Target key(N, y);
        auto it = lay.find(key);
        if (it == lay.end()) {
            wanted.insert(key);
            std::vector<Target> ts;
            for (const Target &t : wanted)
                if (!lay.count(t)) ts.push_back(t);
            wanted.clear();
            std::vector<std::vector<uint64_t>> vs;
            if (int rc = fetch(ts, &vs)) {
                dev_rc = rc;
                over = true;
                return nullptr;
            }
            for (size_t i = 0; i < ts.size(); ++i) lay.emplace(ts[i], std::move(vs[i]));
            it = lay.find(key);
        }
        return it->second.data();
    }
    // Word lengths of each box up to Lmax, from the RSM alone: words[b][j] is
    // set iff box b derives a word of j terminals.  A path of j edges derived
    // from b needs one, so a subcall of a length b cannot spell is empty.
    std::vector<std::vector<uint8_t>> words;
    uint32_t words_L = ~0u;
    void word_lengths() {
        if (words_L == Lmax) return;
        const uint32_t L1 = Lmax + 1;
        words.assign(r->B, std::vector<uint8_t>(L1, 0));
        // at[s][j]: state s is reached from its box's start state over j terminals
        std::vector<std::vector<uint8_t>> at(r->Q, std::vector<uint8_t>(L1, 0));
        for (uint32_t b = 0; b < r->B; ++b) at[r->box_start[b]][0] = 1;
        for (bool grew = true; grew;) {
            grew = false;
            for (const auto &t : r->tr)
                for (uint32_t j = 0; j < L1; ++j) {
                    if (!at[t.from][j]) continue;
                    for (uint32_t i = t.kind == 0 ? 1u : 0u; j + i < L1; ++i) {
                        if (t.kind == 0 ? i != 1u : !words[t.sym][i]) {
                            if (t.kind == 0) break;
                            continue;
                        }
                        if (!at[t.to][j + i]) {
                            at[t.to][j + i] = 1;
                            grew = true;
                        }
                    }
                }
            for (uint32_t f = 0; f < r->Q; ++f)
                if (r->final_[f])
                    for (uint32_t j = 0; j < L1; ++j)
                        if (at[f][j] && !words[r->state_box[f]][j]) {
                            words[r->state_box[f]][j] = 1;
                            grew = true;
                        }
        }
        words_L = Lmax;
    }

    // Graph distance from v over any labels, capped at Lmax + 1 (breadth-first,
    // depth Lmax): a subpath v -> v2 of j edges exists only if it is <= j.
    std::map<uint32_t, std::vector<uint16_t>> fdist;
    size_t dist_cache_bytes = (size_t)1 << 30;  // per distance cache
    const uint16_t *dist_from(uint32_t v) {
        auto it = fdist.find(v);
        if (it != fdist.end()) return it->second.data();
        const uint16_t far = (uint16_t)std::min<uint32_t>(Lmax + 1u, 65535u);
        std::vector<uint16_t> d(n, far);
        std::vector<uint32_t> cur{v}, nxt;
        d[v] = 0;
        for (uint32_t depth = 1; depth <= Lmax && !cur.empty(); ++depth) {
            nxt.clear();
            for (uint32_t a : cur)
                for (uint32_t e = eoff[a]; e < eoff[a + 1]; ++e)
                    if (d[ed[e]] == far) {
                        d[ed[e]] = (uint16_t)depth;
                        nxt.push_back(ed[e]);
                    }
            cur.swap(nxt);
        }
        // a pointer from an earlier call is not used after this one, so the
        // cache can be dropped when it outgrows its share of host memory
        if ((fdist.size() + 1) * (size_t)n * sizeof(uint16_t) > dist_cache_bytes) fdist.clear();
        return fdist.emplace(v, std::move(d)).first->second.data();
    }
    // Graph distance to y over any labels, capped like dist_from (breadth-first
    // over the reversed edges): a path of `len` edges ending at y passes a
    // vertex u after k edges only if the distance from u to y is <= len - k.
    // The layers give a weaker bound, as they count a nonterminal edge as one
    // edge whatever the graph distance it spans.
    std::vector<uint32_t> roff, rsrc;  // reversed terminal edges, by target
    std::map<uint32_t, std::vector<uint16_t>> bdist;
    uint32_t dist_L = ~0u;             // the bound the cached distances were taken to
    const uint16_t *dist_to(uint32_t y) {
        if (roff.size() != (size_t)n + 1) {
            roff.assign((size_t)n + 1, 0);
            for (uint32_t d : ed) ++roff[d + 1];
            for (uint32_t v = 0; v < n; ++v) roff[v + 1] += roff[v];
            rsrc.resize(ed.size());
            std::vector<uint32_t> fill(roff.begin(), roff.end() - 1);
            for (size_t e = 0; e < ed.size(); ++e) rsrc[fill[ed[e]]++] = es[e];
        }
        auto it = bdist.find(y);
        if (it != bdist.end()) return it->second.data();
        const uint16_t far = (uint16_t)std::min<uint32_t>(Lmax + 1u, 65535u);
        std::vector<uint16_t> d(n, far);
        std::vector<uint32_t> cur{y}, nxt;
        d[y] = 0;
        for (uint32_t depth = 1; depth <= Lmax && !cur.empty(); ++depth) {
            nxt.clear();
            for (uint32_t a : cur)
                for (uint32_t k = roff[a]; k < roff[a + 1]; ++k)
                    if (d[rsrc[k]] == far) {
                        d[rsrc[k]] = (uint16_t)depth;
                        nxt.push_back(rsrc[k]);
                    }
            cur.swap(nxt);
        }
        if ((bdist.size() + 1) * (size_t)n * sizeof(uint16_t) > dist_cache_bytes) bdist.clear();
        return bdist.emplace(y, std::move(d)).first->second.data();
    }
    // both distance caches hold distances capped at the current bound
    void check_dist_bound() {
        if (dist_L == Lmax) return;
        fdist.clear();
        bdist.clear();
        dist_L = Lmax;
    }
    // Without nonterminal transitions the layers are exact product distances,
    // at least the graph distance: the distance bound adds nothing there.
    std::vector<uint16_t> no_dist;
    int has_nt = -1;
    const uint16_t *target_dist(uint32_t y) {
        if (has_nt < 0) {
            has_nt = 0;
            for (const auto &t : r->tr) has_nt |= t.kind != 0 ? 1 : 0;
        }
        if (has_nt) return dist_to(y);
        if (no_dist.size() != n) no_dist.assign(n, 0);
        return no_dist.data();
    }
    using Key = std::tuple<uint32_t, uint32_t, uint32_t, uint32_t>;
    struct KeyHash {
        size_t operator()(const Key &k) const {
            uint64_t h = ((uint64_t)std::get<0>(k) << 32 | std::get<3>(k)) * 0x9E3779B97F4A7C15ull;
            h ^= ((uint64_t)std::get<1>(k) << 32 | std::get<2>(k)) * 0xC2B2AE3D27D4EB4Full;
            return (size_t)(h ^ (h >> 31));
        }
    };
    // the path set of every key (references stay valid when the map rehashes)
    std::unordered_map<Key, std::set<std::vector<uint32_t>>, KeyHash> memo;
    size_t stored = 0, cap = 4000000;
    bool over = false;

    size_t key_cap = 1u << 20;
    // Worklist of keys to (re)evaluate and, per key, the keys whose
    // evaluation read it: a key is evaluated again only when a set it reads
    // has grown.
    std::deque<Key> work;
    std::unordered_set<Key, KeyHash> queued;
    std::unordered_map<Key, std::vector<Key>, KeyHash> readers;
    const Key *reading = nullptr;                // key under evaluation
    std::unordered_set<Key, KeyHash> read_now;  // the keys its evaluation read

    const std::set<std::vector<uint32_t>> &get(uint32_t N, uint32_t x, uint32_t y, uint32_t len) {
        const Key key = std::make_tuple(N, x, y, len);
        auto it = memo.find(key);
        if (it == memo.end()) {
            it = memo.emplace(key, std::set<std::vector<uint32_t>>()).first;
            if (memo.size() > key_cap) over = true;
            work.push_back(key);
            queued.insert(key);
            if (!lay.count(Target(N, y))) wanted.insert(Target(N, y));
        }
        if (reading) read_now.insert(key);
        return it->second;
    }

    // One evaluation of Paths(N, x, y, len) from the current memo values.
    std::set<std::vector<uint32_t>> eval(uint32_t N, uint32_t x, uint32_t y, uint32_t len) {
        using PSet = std::set<std::vector<uint32_t>>;
        const uint64_t *D = layers_for(N, y);
        if (!D) return PSet();
        // (s, v) can reach a target of (N, y) over at most `rem` edges
        auto live = [&](uint32_t s, uint32_t v, uint32_t rem) {
            return (D[((size_t)rem * Qd + s) * Wd + (v >> 6)] >> (v & 63)) & 1ull;
        };
        // layer[k]: map (state, vertex) -> paths of k edges from (q0, x)
        std::vector<std::map<std::pair<uint32_t, uint32_t>, PSet>> layer(len + 1);
        const uint32_t q0 = r->box_start[N];
        word_lengths();
        check_dist_bound();
        const uint16_t *dy = target_dist(y);
        if (!words[N][len] || !live(q0, x, len) || dy[x] > len) return PSet();
        layer[0][{q0, x}].insert(std::vector<uint32_t>());
        for (uint32_t k = 0; k <= len; ++k) {
            bool grew = true;
            while (grew && !over) {
                grew = false;
                auto snapshot = layer[k];
                for (auto &kv : snapshot) {
                    const uint32_t s = kv.first.first, v = kv.first.second;
                    const PSet &S = kv.second;
                    for (const auto &t : r->tr) {
                        if (t.from != s) continue;
                        if (t.kind == 0) {
                            if (k + 1 > len) continue;
                            for (uint32_t e = eoff[v]; e < eoff[v + 1]; ++e) {
                                if (el[e] != t.sym || dy[ed[e]] > len - k - 1 || !live(t.to, ed[e], len - k - 1)) continue;
                                PSet &Dst = layer[k + 1][{t.to, ed[e]}];
                                for (const auto &p : S) {
                                    auto q = p;
                                    q.push_back(e);
                                    Dst.insert(std::move(q));
                                }
                            }
                        } else {
                            const uint64_t *row = m2[t.sym].data() + (size_t)v * wn;
                            // layers grow with the budget: layer len - k bounds every j
                            const uint64_t *reach = D + ((size_t)(len - k) * Qd + t.to) * Wd;
                            const uint16_t *dv = dist_from(v);
                            for (size_t w = 0; w < wn; ++w) {
                                uint64_t b = row[w] & reach[w];
                                while (b) {
                                    const uint32_t v2 = (uint32_t)(w * 64 + (uint64_t)__builtin_ctzll(b));
                                    b &= b - 1;
                                    // j <= len - k - (distance from v2 to y)
                                    if (dy[v2] > len - k) continue;
                                    for (uint32_t j = dv[v2]; k + j + dy[v2] <= len; ++j) {
                                        if (!words[t.sym][j] || !live(t.to, v2, len - k - j)) continue;
                                        const PSet &sub = get(t.sym, v, v2, j);
                                        if (sub.empty()) continue;
                                        PSet &Dst = layer[k + j][{t.to, v2}];
                                        const size_t before = Dst.size();
                                        for (const auto &p : S)
                                            for (const auto &s2 : sub) {
                                                auto q = p;
                                                q.insert(q.end(), s2.begin(), s2.end());
                                                Dst.insert(std::move(q));
                                            }
                                        if (j == 0 && Dst.size() != before) grew = true;
                                    }
                                }
                            }
                        }
                    }
                }
            }
        }
        PSet out;
        for (uint32_t f = 0; f < r->Q; ++f) {
            if (r->state_box[f] != N || !r->final_[f]) continue;
            auto it = layer[len].find({f, y});
            if (it != layer[len].end()) out.insert(it->second.begin(), it->second.end());
        }
        return out;
    }

    // Least fixpoint of the keys reachable from those requested: evaluate the
    // queued keys; a key whose set grew queues its readers.  The sets only
    // grow (evaluation is monotone in the memo) and are finite, so this ends.
    void solve() {
        while (!work.empty() && !over) {
            const Key k = work.front();
            work.pop_front();
            queued.erase(k);
            reading = &k;
            read_now.clear();
            auto v = eval(std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k));
            reading = nullptr;
            for (const Key &rk : read_now) readers[rk].push_back(k);
            auto &cur = memo[k];
            if (v.size() == cur.size()) continue;
            stored += v.size() - cur.size();
            cur = std::move(v);
            if (stored > cap) over = true;
            auto rd = readers.find(k);
            if (rd == readers.end()) continue;
            for (const Key &r2 : rd->second)
                if (queued.insert(r2).second) work.push_back(r2);
        }
    }
};


}  // namespace cfpq
