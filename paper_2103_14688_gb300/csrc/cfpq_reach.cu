// cfpq_reach.cu -- rows of C3 a multiple-source query needs.
//
// The multiple-source version of the algorithm (named as future work in
// Sec. 6): for a source set S only the rows (s, x) of C3 reachable in the
// Kronecker product M3 from {(q0, x) : x in S} (q0 the start state of the
// start box) contribute to the answer rows of S, since C3 = M3^+ and row
// (q0, x) of C3 is the union of the rows reachable from it.  For RSMs whose
// transitions read only terminals, M3 = OR_l M1^l (x) M2^l is fixed, and one
// breadth-first search marks those rows: per state s a bit row R_s of the
// vertices x with (s, x) reachable, expanded one frontier at a time.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cfpq_engine.cuh"

namespace cfpq {

struct ReachDesc {
    const uint32_t *csr_off;  // [n_term * n + 1]
    const uint32_t *csr_col;
    const uint32_t *tr_off;   // [Q + 1] terminal transitions of each state
    const uint32_t *tr_lbl;
    const uint32_t *tr_to;
    uint64_t *R;              // [Q * W] reached rows
    const uint64_t *F;        // [Q * W] frontier of this round
    uint64_t *Fn;             // [Q * W] frontier of the next round (zero on entry)
    unsigned int *changed;
    uint32_t n, W, Q;
};

// One round: every (s, x) of the frontier follows its terminal transitions
// s -l-> u to (u, y) for the edges x -l-> y; newly reached pairs form the next
// frontier.
__global__ void k_reach_round(ReachDesc d) {
    const size_t total = (size_t)d.Q * d.W;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        uint64_t f = d.F[i];
        if (!f) continue;
        const uint32_t s = (uint32_t)(i / d.W), w = (uint32_t)(i % d.W);
        const uint32_t t0 = d.tr_off[s], t1 = d.tr_off[s + 1];
        while (f) {
            const uint32_t b = (uint32_t)__ffsll((long long)f) - 1u;
            f &= f - 1ull;
            const uint32_t x = w * 64u + b;
            for (uint32_t t = t0; t < t1; ++t) {
                const uint32_t l = d.tr_lbl[t], u = d.tr_to[t];
                const size_t r = (size_t)l * d.n + x;
                const uint32_t e1 = d.csr_off[r + 1];
                for (uint32_t e = d.csr_off[r]; e < e1; ++e) {
                    const uint32_t y = d.csr_col[e];
                    const size_t wi = (size_t)u * d.W + (y >> 6);
                    const unsigned long long bit = 1ull << (y & 63u);
                    const unsigned long long old = atomicOr(reinterpret_cast<unsigned long long *>(d.R + wi), bit);
                    if (!(old & bit)) {
                        atomicOr(reinterpret_cast<unsigned long long *>(d.Fn + wi), bit);
                        *d.changed = 1u;
                    }
                }
            }
        }
    }
}

// (q0, x) for the sources: reached and the first frontier.
__global__ void k_reach_init(uint64_t *R, uint64_t *F, const uint32_t *src, uint32_t ns, uint32_t q0, uint32_t W) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x) {
        const uint32_t x = src[i];
        const size_t wi = (size_t)q0 * W + (x >> 6);
        const unsigned long long bit = 1ull << (x & 63u);
        atomicOr(reinterpret_cast<unsigned long long *>(R + wi), bit);
        atomicOr(reinterpret_cast<unsigned long long *>(F + wi), bit);
    }
}

int QueryDev::compute_reach(Allocator *A, cudaStream_t st, const uint32_t *h_src, uint32_t ns, std::string *err) {
    const size_t words = (size_t)Q * W;
    // terminal transitions per state (the RSM reads no nonterminal here)
    std::vector<uint32_t> off(Q + 1, 0), lbl, to;
    for (const auto &tr : rsm.tr)
        if (tr.kind == 0) ++off[tr.from + 1];
    for (uint32_t s = 0; s < Q; ++s) off[s + 1] += off[s];
    lbl.resize(off[Q]);
    to.resize(off[Q]);
    std::vector<uint32_t> fill(off.begin(), off.end() - 1);
    for (const auto &tr : rsm.tr)
        if (tr.kind == 0) {
            lbl[fill[tr.from]] = tr.sym;
            to[fill[tr.from]] = tr.to;
            ++fill[tr.from];
        }
    const size_t tr_words = (Q + 1) + 2 * (size_t)off[Q];
    if (!reach_mem.ensure(A, words * 8, err) || !reach_f.ensure(A, 2 * words * 8, err) ||
        !reach_misc.ensure(A, (tr_words + (size_t)ns + 64) * 4, err))
        return CFPQ_ERR_OUT_OF_MEMORY;
    uint32_t *misc = reach_misc.as<uint32_t>();
    unsigned int *changed = reinterpret_cast<unsigned int *>(misc);  // word 0; tables from word 16
    uint32_t *d_off = misc + 16, *d_lbl = d_off + (Q + 1), *d_to = d_lbl + off[Q], *d_src = d_to + off[Q];
    ENG_CK(cudaMemcpyAsync(d_off, off.data(), (Q + 1) * 4, cudaMemcpyHostToDevice, st));
    if (off[Q]) {
        ENG_CK(cudaMemcpyAsync(d_lbl, lbl.data(), off[Q] * 4, cudaMemcpyHostToDevice, st));
        ENG_CK(cudaMemcpyAsync(d_to, to.data(), off[Q] * 4, cudaMemcpyHostToDevice, st));
    }
    if (ns) ENG_CK(cudaMemcpyAsync(d_src, h_src, (size_t)ns * 4, cudaMemcpyHostToDevice, st));
    uint64_t *R = reach_mem.as<uint64_t>(), *F = reach_f.as<uint64_t>(), *Fn = F + words;
    ENG_CK(cudaMemsetAsync(R, 0, words * 8, st));
    ENG_CK(cudaMemsetAsync(F, 0, 2 * words * 8, st));
    const uint32_t q0 = rsm.box_start[rsm.start_box];
    if (ns) {
        k_reach_init<<<(ns + 255u) / 256u < 1024u ? (ns + 255u) / 256u : 1024u, 256, 0, st>>>(R, F, d_src, ns, q0, W);
        ENG_CK(cudaGetLastError());
    }
    const unsigned grid = (unsigned)std::min<size_t>((words + 255) / 256, 4096);
    // Rounds are issued four at a time between reads of the changed flag (a
    // round on an empty frontier does nothing); every round that changes
    // something reaches a new pair, so the search ends.
    constexpr int kRoundsPerSync = 4;
    for (size_t round = 0; ns && round <= (size_t)Q * n; round += kRoundsPerSync) {
        ENG_CK(cudaMemsetAsync(changed, 0, 4, st));
        for (int k = 0; k < kRoundsPerSync; ++k) {
            ReachDesc d{g->csr_off.as<uint32_t>(), g->csr_col.as<uint32_t>(), d_off, d_lbl, d_to, R, F, Fn, changed,
                        n, W, Q};
            k_reach_round<<<grid, 256, 0, st>>>(d);
            ENG_CK(cudaGetLastError());
            std::swap(F, Fn);
            ENG_CK(cudaMemsetAsync(Fn, 0, words * 8, st));
        }
        unsigned int h_changed = 0;
        ENG_CK(cudaMemcpyAsync(&h_changed, changed, 4, cudaMemcpyDeviceToHost, st));
        ENG_CK(cudaStreamSynchronize(st));
        if (!h_changed) break;
    }
    return CFPQ_OK;
}

}  // namespace cfpq
