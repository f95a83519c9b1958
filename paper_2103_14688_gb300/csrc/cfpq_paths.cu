// cfpq_paths.cu -- device side of path extraction (Sec. 3.2, Listing 2).
//
// genPaths explores M3 from (q0, vs) one Boolean vector-matrix product at a
// time and keeps the paths that reach a target (f, vf), f final.  The host
// enumerator follows the product edges forward; this file gives it, per
// target (box N, vertex y), the backward layers of the search on the device:
//
//   D_k = { (s, x) : some target (f, y), f in F_N, is reached from (s, x)
//                    over a path of M3 that spells at most k graph edges }
//
// A product edge over a terminal spells one graph edge.  One over a
// nonterminal N' from (s, x) to (u, z) spells the edges of a path x -> z
// derived from N': at least one edge when x != z, possibly none when x == z
// (N' may derive the empty word).  Those lower bounds are the edge weights
// of the search, so D_k contains every product vertex that a path of at most
// k edges can pass through with the remaining budget, and the host may drop
// every partial path whose end (s, x) is outside D_{len - k}: no path of the
// answer is lost.
//
// One layer from the previous one:
//   - unit step: S_{k+1} = S_k, then every (u, z) new in layer k (Delta_k)
//     adds its M3 predecessors: (s, x) for x -l-> z in the graph and
//     s -l-> u in the RSM (reverse CSR of the terminals), and the rows x of
//     column z of M2^{N'} for s -N'-> u (the column is a row of M2^{N'}
//     transposed once per extraction call);
//   - zero step: per vertex z, the states s with s -N'-> u, (u, z) in the
//     layer and M2^{N'}[z, z] = 1, to a fixpoint (at most Q rounds);
//   - Delta_{k+1} = S_{k+1} and not S_k.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>

#include "cfpq_engine.cuh"

namespace cfpq {

namespace {

// Bit matrix transpose, one warp per 64 x 64 tile: rows r0..r0+63 of the
// n-row source (word wc) become rows 64*wc .. 64*wc+63 of the destination
// (word r0 / 64).  Lane i holds source rows r0+i and r0+32+i; output row j of
// the tile is the ballot of bit j over the 64 source rows.
__global__ void k_bit_transpose(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst, uint32_t n,
                                uint32_t W) {
    const uint32_t lane = threadIdx.x & 31u;
    const size_t warps = (size_t)gridDim.x * (blockDim.x >> 5);
    const size_t tiles = (size_t)W * W;
    for (size_t t = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < tiles; t += warps) {
        const uint32_t rt = (uint32_t)(t / W), wc = (uint32_t)(t % W);
        const uint32_t r0 = rt * 64u + lane, r1 = r0 + 32u;
        const uint64_t a = r0 < n ? src[(size_t)r0 * W + wc] : 0ull;
        const uint64_t b = r1 < n ? src[(size_t)r1 * W + wc] : 0ull;
        uint64_t o0 = 0, o1 = 0;
        for (uint32_t j = 0; j < 64u; ++j) {
            const uint32_t lo = __ballot_sync(0xffffffffu, (uint32_t)(a >> j) & 1u);
            const uint32_t hi = __ballot_sync(0xffffffffu, (uint32_t)(b >> j) & 1u);
            const uint64_t v = (uint64_t)lo | ((uint64_t)hi << 32);
            if (j == lane) o0 = v;
            if (j == lane + 32u) o1 = v;
        }
        dst[((size_t)wc * 64u + lane) * W + rt] = o0;
        dst[((size_t)wc * 64u + lane + 32u) * W + rt] = o1;
    }
}

struct BackDesc {
    const uint32_t *roff;    // reverse terminal CSR: [n_term * n + 1] over (label, target vertex)
    const uint32_t *rcol;    // sources
    const uint32_t *rt_off;  // [Q + 1] RSM transitions into each state
    const uint32_t *rt_from;
    const uint32_t *rt_kind; // 0 terminal, 1 nonterminal
    const uint32_t *rt_sym;
    const int32_t *mt_slot;  // [B] slot of box b's transposed M2 in mt (or -1)
    const uint64_t *mt;      // transposed M2 rows, n_pad * W words per slot
    const uint64_t *delta;   // [T * Q * W] vertices new in layer k, per target
    uint64_t *S;             // [T * Q * W] layer k + 1 (a copy of layer k on entry)
    uint32_t n, W, Q, T;     // T targets searched side by side
};

// Unit step: one warp per word of Delta_k; lanes split the predecessor lists.
__global__ void k_back_unit(BackDesc d) {
    const uint32_t lane = threadIdx.x & 31u;
    const size_t warps = (size_t)gridDim.x * (blockDim.x >> 5);
    const size_t total = (size_t)d.T * d.Q * d.W;
    for (size_t i = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < total; i += warps) {
        uint64_t f = d.delta[i];
        if (!f) continue;
        const size_t tq = i / d.W;  // target * Q + state
        const uint32_t u = (uint32_t)(tq % d.Q), w = (uint32_t)(i % d.W);
        uint64_t *const S = d.S + (tq - u) * d.W;  // this target's layer
        const uint32_t t0 = d.rt_off[u], t1 = d.rt_off[u + 1];
        while (f) {
            const uint32_t z = w * 64u + (uint32_t)(__ffsll((long long)f) - 1);
            f &= f - 1ull;
            for (uint32_t t = t0; t < t1; ++t) {
                uint64_t *row = S + (size_t)d.rt_from[t] * d.W;
                if (d.rt_kind[t] == 0) {
                    const size_t r = (size_t)d.rt_sym[t] * d.n + z;
                    const uint32_t e1 = d.roff[r + 1];
                    for (uint32_t e = d.roff[r] + lane; e < e1; e += 32u) {
                        const uint32_t x = d.rcol[e];
                        const unsigned long long bit = 1ull << (x & 63u);
                        if (!(__ldcg(row + (x >> 6)) & bit))
                            atomicOr(reinterpret_cast<unsigned long long *>(row + (x >> 6)), bit);
                    }
                } else {
                    const int32_t slot = d.mt_slot[d.rt_sym[t]];
                    const uint64_t *col = d.mt + ((size_t)slot * d.W * 64u + z) * d.W;
                    for (uint32_t k = lane; k < d.W; k += 32u) {
                        const uint64_t v = col[k];
                        if (v & ~__ldcg(row + k)) atomicOr(reinterpret_cast<unsigned long long *>(row + k), v);
                    }
                }
            }
        }
    }
}

// Zero step: thread per (target, vertex z); nonterminal transitions (from,
// box, to) in nt[3 * i ..]; diagonal bits read from M2 (n rows of W words per
// box).
__global__ void k_back_zero(uint64_t *S0, const uint32_t *nt, uint32_t n_nt, const uint64_t *m2, uint32_t n,
                            uint32_t W, uint32_t Q, uint32_t T) {
    const size_t total = (size_t)T * n;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t z = (uint32_t)(i % n);
        uint64_t *const S = S0 + (i / n) * Q * W;
        const uint32_t w = z >> 6;
        const uint64_t bit = 1ull << (z & 63u);
        bool changed = true;
        for (uint32_t pass = 0; changed && pass < Q; ++pass) {
            changed = false;
            for (uint32_t i = 0; i < n_nt; ++i) {
                const uint32_t s = nt[3 * i], b = nt[3 * i + 1], u = nt[3 * i + 2];
                if (!(m2[((size_t)b * n + z) * W + w] & bit)) continue;
                if (!(__ldcg(S + (size_t)u * W + w) & bit)) continue;
                if (__ldcg(S + (size_t)s * W + w) & bit) continue;
                atomicOr(reinterpret_cast<unsigned long long *>(S + (size_t)s * W + w), bit);
                changed = true;
            }
        }
    }
}

// Delta = cur and not prev; *any is set when Delta is not empty.
__global__ void k_back_delta(const uint64_t *cur, const uint64_t *prev, uint64_t *delta, size_t words,
                             unsigned int *any) {
    bool nz = false;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x) {
        const uint64_t v = prev ? (cur[i] & ~prev[i]) : cur[i];
        delta[i] = v;
        nz |= v != 0;
    }
    if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(any, 1u);
}

unsigned grid_for(size_t work, unsigned per_block) {
    return (unsigned)std::max<size_t>(1, std::min<size_t>((work + per_block - 1) / per_block, 4096));
}

}  // namespace

int PathsDev::prepare(Allocator *A, cudaStream_t st, const QueryDev &q, uint32_t n_term,
                      const std::vector<uint32_t> &h_roff, const std::vector<uint32_t> &h_rcol, std::string *err) {
    n = q.n;
    W = q.W;
    Q = q.Q;
    // RSM transitions grouped by target state (terminals the graph does not
    // have are left out: their matrices are empty); nonterminal triples.
    std::vector<HostRSM::Tr> tr;
    for (const auto &t : q.rsm.tr)
        if (t.kind != 0 || t.sym < n_term) tr.push_back(t);
    std::vector<uint32_t> off(Q + 1, 0), from, kind, sym, nt;
    for (const auto &t : tr) ++off[t.to + 1];
    for (uint32_t s = 0; s < Q; ++s) off[s + 1] += off[s];
    const uint32_t T = off[Q];
    from.resize(T);
    kind.resize(T);
    sym.resize(T);
    std::vector<uint32_t> fill(off.begin(), off.end() - 1);
    std::vector<int32_t> slot(q.B, -1);
    uint32_t n_mt = 0;
    for (const auto &t : tr) {
        const uint32_t k = fill[t.to]++;
        from[k] = t.from;
        kind[k] = t.kind;
        sym[k] = t.sym;
        if (t.kind != 0) {
            nt.push_back(t.from);
            nt.push_back(t.sym);
            nt.push_back(t.to);
            if (slot[t.sym] < 0) slot[t.sym] = (int32_t)n_mt++;
        }
    }
    n_nt = (uint32_t)(nt.size() / 3);
    const size_t tab_words = (Q + 1) + 3 * (size_t)T + q.B + nt.size() + 16;
    const size_t mt_words = (size_t)n_mt * W * 64u * W;
    if (!tables.ensure(A, tab_words * 4, err) || !rev_off.ensure(A, h_roff.size() * 4, err) ||
        !rev_col.ensure(A, std::max<size_t>(h_rcol.size(), 1) * 4, err) ||
        !mt.ensure(A, std::max<size_t>(mt_words, 1) * 8, err))
        return CFPQ_ERR_OUT_OF_MEMORY;
    std::vector<uint32_t> tab;
    tab.reserve(tab_words);
    tab.insert(tab.end(), off.begin(), off.end());
    tab.insert(tab.end(), from.begin(), from.end());
    tab.insert(tab.end(), kind.begin(), kind.end());
    tab.insert(tab.end(), sym.begin(), sym.end());
    for (int32_t v : slot) tab.push_back((uint32_t)v);
    tab.insert(tab.end(), nt.begin(), nt.end());
    host_tab = tab;
    ENG_CK(cudaMemcpyAsync(tables.p, host_tab.data(), host_tab.size() * 4, cudaMemcpyHostToDevice, st));
    ENG_CK(cudaMemcpyAsync(rev_off.p, h_roff.data(), h_roff.size() * 4, cudaMemcpyHostToDevice, st));
    if (!h_rcol.empty())
        ENG_CK(cudaMemcpyAsync(rev_col.p, h_rcol.data(), h_rcol.size() * 4, cudaMemcpyHostToDevice, st));
    for (uint32_t b = 0; b < q.B; ++b) {
        if (slot[b] < 0) continue;
        k_bit_transpose<<<grid_for((size_t)W * W, 8), 256, 0, st>>>(q.m2_ptr(b),
                                                                     mt.as<uint64_t>() + (size_t)slot[b] * W * 64u * W,
                                                                     n, W);
        ENG_CK(cudaGetLastError());
    }
    m2 = q.m2_ptr(0);
    B = q.B;
    return CFPQ_OK;
}

int PathsDev::layers(Allocator *A, cudaStream_t st, const HostRSM &rsm,
                     const std::vector<std::pair<uint32_t, uint32_t>> &targets, uint32_t L,
                     std::vector<std::vector<uint64_t>> *out, std::string *err) {
    const size_t words = (size_t)Q * W;
    out->resize(targets.size());
    // targets per batch: layers of at most 1 GiB on the device
    const size_t per = std::max<size_t>(1, ((size_t)1 << 30) / ((size_t)(L + 1) * words * 8));
    for (size_t b0 = 0; b0 < targets.size(); b0 += per) {
        const uint32_t T = (uint32_t)std::min(per, targets.size() - b0);
        if (int rc = layers_batch(A, st, rsm, targets.data() + b0, T, L, out->data() + b0, err)) return rc;
    }
    return CFPQ_OK;
}

int PathsDev::layers_batch(Allocator *A, cudaStream_t st, const HostRSM &rsm,
                           const std::pair<uint32_t, uint32_t> *targets, uint32_t T, uint32_t L,
                           std::vector<uint64_t> *out, std::string *err) {
    const size_t words = (size_t)T * Q * W;  // one layer of every target
    if (!lay.ensure(A, (size_t)(L + 1) * words * 8, err) || !delta.ensure(A, words * 8, err) ||
        !flag.ensure(A, 256, err))
        return CFPQ_ERR_OUT_OF_MEMORY;
    uint64_t *Lk = lay.as<uint64_t>();
    uint64_t *D = delta.as<uint64_t>();
    unsigned int *any = flag.as<unsigned int>();
    const uint32_t NTr = host_tab[Q];
    const uint32_t *tab = tables.as<uint32_t>();
    BackDesc d{rev_off.as<uint32_t>(), rev_col.as<uint32_t>(), tab, tab + (Q + 1), tab + (Q + 1) + NTr,
               tab + (Q + 1) + 2 * (size_t)NTr, reinterpret_cast<const int32_t *>(tab + (Q + 1) + 3 * (size_t)NTr),
               mt.as<uint64_t>(), D, nullptr, n, W, Q, T};
    const uint32_t *nt = tab + (Q + 1) + 3 * (size_t)NTr + B;
    // Layer 0: per target (box, y) the vertices (f, y), f final in the box,
    // closed under zero steps.
    std::vector<uint64_t> h0(words, 0);
    for (uint32_t t = 0; t < T; ++t) {
        const uint32_t box = targets[t].first, y = targets[t].second;
        for (uint32_t f = 0; f < Q; ++f)
            if (rsm.state_box[f] == box && rsm.final_[f])
                h0[((size_t)t * Q + f) * W + (y >> 6)] |= 1ull << (y & 63u);
    }
    ENG_CK(cudaMemcpyAsync(Lk, h0.data(), words * 8, cudaMemcpyHostToDevice, st));
    const unsigned gz = grid_for((size_t)T * n, 256), gw = grid_for(words, 8), gd = grid_for(words, 256);
    if (n_nt) {
        k_back_zero<<<gz, 256, 0, st>>>(Lk, nt, n_nt, m2, n, W, Q, T);
        ENG_CK(cudaGetLastError());
    }
    ENG_CK(cudaMemsetAsync(any, 0, 4, st));
    k_back_delta<<<gd, 256, 0, st>>>(Lk, nullptr, D, words, any);
    ENG_CK(cudaGetLastError());
    // A layer without new vertices repeats forever: the flag is read every
    // few layers and the rest copied on the host.
    constexpr uint32_t kLayersPerSync = 4;
    uint32_t done = 0;  // layers computed
    for (uint32_t k = 0; k < L; ++k) {
        uint64_t *cur = Lk + (size_t)k * words, *next = cur + words;
        ENG_CK(cudaMemcpyAsync(next, cur, words * 8, cudaMemcpyDeviceToDevice, st));
        d.S = next;
        k_back_unit<<<gw, 256, 0, st>>>(d);
        ENG_CK(cudaGetLastError());
        if (n_nt) {
            k_back_zero<<<gz, 256, 0, st>>>(next, nt, n_nt, m2, n, W, Q, T);
            ENG_CK(cudaGetLastError());
        }
        k_back_delta<<<gd, 256, 0, st>>>(next, cur, D, words, any);
        ENG_CK(cudaGetLastError());
        if ((k + 1) % kLayersPerSync == 0 || k + 1 == L) {
            // did any of the last layers add a vertex?
            unsigned int h_any = 0;
            ENG_CK(cudaMemcpyAsync(&h_any, any, 4, cudaMemcpyDeviceToHost, st));
            ENG_CK(cudaStreamSynchronize(st));
            done = k + 1;
            if (!h_any) break;
            ENG_CK(cudaMemsetAsync(any, 0, 4, st));
        }
    }
    std::vector<uint64_t> h((size_t)(done + 1) * words);
    ENG_CK(cudaMemcpyAsync(h.data(), Lk, h.size() * 8, cudaMemcpyDeviceToHost, st));
    ENG_CK(cudaStreamSynchronize(st));
    // per target: layers 0..L, layer-major (layers past `done` repeat it)
    const size_t tw = (size_t)Q * W;
    for (uint32_t t = 0; t < T; ++t) {
        std::vector<uint64_t> &o = out[t];
        o.resize((size_t)(L + 1) * tw);
        for (uint32_t k = 0; k <= L; ++k)
            std::memcpy(o.data() + (size_t)k * tw, h.data() + (size_t)std::min(k, done) * words + (size_t)t * tw,
                        tw * 8);
    }
    return CFPQ_OK;
}

}  // namespace cfpq
