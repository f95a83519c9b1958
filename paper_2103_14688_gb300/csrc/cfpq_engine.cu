// cfpq_engine.cu -- host side of the index-creation engine: input staging,
// per-query planning of the closure blocks, and the executor that drives the
// fixpoint loop of Listing 1 (arXiv 2103.14688, Sec. 3.1) for one or many
// queries, as a CUDA graph with a device-side while loop or as host-driven
// passes.
#include <algorithm>
#include <cstring>
#include <string>
#include <type_traits>

#include "cfpq_engine.cuh"

namespace cfpq {


void *Allocator::get(size_t bytes, std::string *err) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (budget && in_use + bytes > budget) {
        if (err) *err = "device memory budget exceeded (" + std::to_string(in_use + bytes) + " > " +
                        std::to_string(budget) + " bytes)";
        return nullptr;
    }
    void *p = nullptr;
    if (alloc) {
        p = alloc(bytes, stream, user);
    } else if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (!p) {
        if (err) *err = "device allocation of " + std::to_string(bytes) + " bytes failed";
        return nullptr;
    }
    in_use += bytes;
    return p;
}

void Allocator::put(void *p, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (free) free(p, bytes, stream, user);
    else cudaFreeAsync(p, stream);
    in_use -= std::min(in_use, bytes);
}

void *SlabArena::take(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    while (chunk < chunks.size()) {
        if (chunks[chunk].second - used >= bytes) {
            void *p = static_cast<char *>(chunks[chunk].first) + used;
            used += bytes;
            return p;
        }
        ++chunk;  // (the rest of this chunk stays unused until reset)
        used = 0;
    }
    const size_t cb = std::max(chunk_bytes, bytes);
    void *p = parent->get(cb, nullptr);
    if (!p) return nullptr;
    chunks.push_back({p, cb});
    chunk = chunks.size() - 1;
    used = bytes;
    return p;
}

void SlabArena::release() {
    for (auto &c : chunks)
        if (parent) parent->put(c.first, c.second);
    chunks.clear();
    reset();
}

static void *slab_alloc(size_t bytes, void *, void *user) { return static_cast<SlabArena *>(user)->take(bytes); }
static void slab_free(void *, size_t, void *, void *) {}

void bind_slab(SlabArena *s, Allocator *parent, cudaStream_t st) {
    s->parent = parent;
    s->A.alloc = slab_alloc;
    s->A.free = slab_free;
    s->A.user = s;
    s->A.stream = st;
    s->A.budget = 0;  // the parent's budget applies to the chunks
}

// ---------------------------------------------------------------------------
// RSM validation (Sec. 2.3, Def. of an RSM).
// ---------------------------------------------------------------------------
int copy_rsm(const cfpq_rsm *r, HostRSM *out, std::string *err) {
    if (!r) { *err = "rsm is NULL"; return CFPQ_ERR_INVALID_ARG; }
    if (r->n_states == 0 || r->n_boxes == 0 || r->start_box >= r->n_boxes) {
        *err = "rsm needs at least one state and one box, and start_box < n_boxes";
        return CFPQ_ERR_INVALID_ARG;
    }
    if (!r->box_start || !r->state_box || !r->state_final || (r->n_trans && (!r->tr_from || !r->tr_kind ||
                                                                              !r->tr_sym || !r->tr_to))) {
        *err = "rsm has a NULL array";
        return CFPQ_ERR_INVALID_ARG;
    }
    HostRSM h;
    h.Q = r->n_states;
    h.B = r->n_boxes;
    h.start_box = r->start_box;
    h.box_start.assign(r->box_start, r->box_start + h.B);
    h.state_box.assign(r->state_box, r->state_box + h.Q);
    h.final_.assign(r->state_final, r->state_final + h.Q);
    for (uint32_t s = 0; s < h.Q; ++s)
        if (h.state_box[s] >= h.B) { *err = "state_box out of range"; return CFPQ_ERR_INVALID_ARG; }
    for (uint32_t b = 0; b < h.B; ++b)
        if (h.box_start[b] >= h.Q || h.state_box[h.box_start[b]] != b) {
            *err = "box_start[b] must be a state of box b";
            return CFPQ_ERR_INVALID_ARG;
        }
    for (uint32_t k = 0; k < r->n_trans; ++k) {
        HostRSM::Tr t{r->tr_from[k], r->tr_kind[k], r->tr_sym[k], r->tr_to[k]};
        if (t.from >= h.Q || t.to >= h.Q || h.state_box[t.from] != h.state_box[t.to]) {
            *err = "transition " + std::to_string(k) + " leaves its box or names a bad state";
            return CFPQ_ERR_INVALID_ARG;
        }
        if (t.kind > 1 || (t.kind == 1 && t.sym >= h.B)) {
            *err = "transition " + std::to_string(k) + " has a bad kind or box symbol";
            return CFPQ_ERR_INVALID_ARG;
        }
        if (t.kind == 0) h.max_terminal_plus1 = std::max(h.max_terminal_plus1, t.sym + 1);
        h.tr.push_back(t);
    }
    std::sort(h.tr.begin(), h.tr.end(), [](const HostRSM::Tr &a, const HostRSM::Tr &b) {
        if (a.from != b.from) return a.from < b.from;
        if (a.kind != b.kind) return a.kind < b.kind;
        if (a.sym != b.sym) return a.sym < b.sym;
        return a.to < b.to;
    });
    h.tr.erase(std::unique(h.tr.begin(), h.tr.end(),
                           [](const HostRSM::Tr &a, const HostRSM::Tr &b) {
                               return a.from == b.from && a.kind == b.kind && a.sym == b.sym && a.to == b.to;
                           }),
               h.tr.end());
    *out = std::move(h);
    return CFPQ_OK;
}

// ---------------------------------------------------------------------------
// Graph staging (edge list -> per-label deduplicated CSR), on the device.
// ---------------------------------------------------------------------------
int stage_graph(GraphDev *g, Allocator *A, cudaStream_t st, uint32_t n, uint32_t n_term, size_t m, const uint32_t *src,
                const uint32_t *lbl, const uint32_t *dst, bool device_ptrs, std::string *err) {
    if (n == 0 || n_term == 0) { *err = "graph needs n_vertices > 0 and n_terminals > 0"; return CFPQ_ERR_INVALID_ARG; }
    if (m && (!src || !lbl || !dst)) { *err = "edge arrays are NULL"; return CFPQ_ERR_INVALID_ARG; }
    if (m >= 0xffffffffull) { *err = "more than 2^32-1 edges"; return CFPQ_ERR_UNSUPPORTED; }
    const uint32_t n_pad = (n + 127u) & ~127u, W = n_pad / 64u;
    if (vpl_for_words(W) == 0) { *err = "graphs above 65536 vertices are not supported"; return CFPQ_ERR_UNSUPPORTED; }
    const size_t rows = (size_t)n_term * n;
    if (rows + 1 >= 0xffffffffull) { *err = "n_vertices * n_terminals too large"; return CFPQ_ERR_UNSUPPORTED; }
    const size_t mm = m ? m : 1;
    const bool realloc = !(g->csr_off.p && g->csr_off.bytes >= (rows + 1) * 4 && g->csr_col.bytes >= mm * 4);
    const size_t nb = (rows + 4095) / 4096 + 2;
    if (!g->csr_off.ensure(A, (rows + 1) * 4, err) || !g->csr_col.ensure(A, mm * 4, err) ||
        !g->cnt.ensure(A, rows * 4, err) || !g->off.ensure(A, (rows + 1) * 4, err) || !g->col.ensure(A, mm * 4, err) ||
        !g->ucnt.ensure(A, rows * 4, err) || !g->scan_tmp.ensure(A, nb * 4, err) ||
        !g->label_map.ensure(A, (size_t)n_term * 4, err) || !g->err.ensure(A, 16, err))
        return CFPQ_ERR_OUT_OF_MEMORY;
    const uint32_t *s = src, *l = lbl, *d = dst;
    if (!device_ptrs && m) {
        if (!g->e_src.ensure(A, m * 4, err) || !g->e_lbl.ensure(A, m * 4, err) || !g->e_dst.ensure(A, m * 4, err))
            return CFPQ_ERR_OUT_OF_MEMORY;
        ENG_CK(cudaMemcpyAsync(g->e_src.p, src, m * 4, cudaMemcpyHostToDevice, st));
        ENG_CK(cudaMemcpyAsync(g->e_lbl.p, lbl, m * 4, cudaMemcpyHostToDevice, st));
        ENG_CK(cudaMemcpyAsync(g->e_dst.p, dst, m * 4, cudaMemcpyHostToDevice, st));
        s = g->e_src.as<uint32_t>();
        l = g->e_lbl.as<uint32_t>();
        d = g->e_dst.as<uint32_t>();
    }
    if (g->n_term != n_term || realloc) {
        std::vector<int32_t> lm(n_term);
        for (uint32_t i = 0; i < n_term; ++i) lm[i] = (int32_t)i;
        ENG_CK(cudaMemcpyAsync(g->label_map.p, lm.data(), n_term * 4, cudaMemcpyHostToDevice, st));
        ENG_CK(cudaStreamSynchronize(st));
    }
    uint32_t *cnt = g->cnt.as<uint32_t>(), *off = g->off.as<uint32_t>(), *col = g->col.as<uint32_t>();
    uint32_t *ucnt = g->ucnt.as<uint32_t>(), *tmp = g->scan_tmp.as<uint32_t>();
    int *errf = g->err.as<int>();
    ENG_CK(cudaMemsetAsync(cnt, 0, rows * 4, st));
    ENG_CK(cudaMemsetAsync(errf, 0, 16, st));
    ENG_CK(launch_stage_count(s, l, d, m, n, n_term, g->label_map.as<int32_t>(), cnt, errf, st));
    ENG_CK(scan_exclusive(cnt, off, rows, tmp, st));
    ENG_CK(cudaMemsetAsync(ucnt, 0, rows * 4, st));
    ENG_CK(launch_stage_fill(s, l, d, m, n, n_term, g->label_map.as<int32_t>(), off, ucnt, col, st));
    ENG_CK(launch_stage_unique(off, col, ucnt, rows, st));
    ENG_CK(scan_exclusive(ucnt, g->csr_off.as<uint32_t>(), rows, tmp, st));
    ENG_CK(launch_stage_compact(off, col, g->csr_off.as<uint32_t>(), g->csr_col.as<uint32_t>(), rows, st));
    int herr = 0;
    uint32_t total = 0;
    ENG_CK(cudaMemcpyAsync(&herr, errf, 4, cudaMemcpyDeviceToHost, st));
    ENG_CK(cudaMemcpyAsync(&total, g->csr_off.as<uint32_t>() + rows, 4, cudaMemcpyDeviceToHost, st));
    ENG_CK(cudaStreamSynchronize(st));
    if (herr) {
        *err = "an edge names a vertex >= n_vertices or a label >= n_terminals";
        g->n = 0;
        return CFPQ_ERR_INVALID_ARG;
    }
    if (realloc || g->n != n || g->n_term != n_term) g->generation += 1;
    g->content += 1;
    g->n = n;
    g->n_pad = n_pad;
    g->W = W;
    g->n_term = n_term;
    g->m_in = m;
    g->m_unique = total;
    g->host_valid = false;
    return CFPQ_OK;
}

int GraphDev::ensure_nonempty(Allocator *A, cudaStream_t st, std::string *err) {
    if (nonempty.p && nonempty_content == content) return CFPQ_OK;
    if (!nonempty.ensure(A, std::max<size_t>((size_t)n_term * W * 8, 64), err)) return CFPQ_ERR_OUT_OF_MEMORY;
    ENG_CK(launch_nonempty_bits(csr_off.as<uint32_t>(), n, n_term, W, nonempty.as<uint64_t>(), st));
    nonempty_content = content;
    return CFPQ_OK;
}

int GraphDev::ensure_term_bits(Allocator *A, cudaStream_t st, std::string *err) {
    if (term_bits.p && term_bits_content == content) return CFPQ_OK;
    const size_t rows = (size_t)n_term * n;
    if (!term_bits.ensure(A, rows * W * 8, err)) return CFPQ_ERR_OUT_OF_MEMORY;
    ENG_CK(cudaMemsetAsync(term_bits.p, 0, rows * W * 8, st));
    ENG_CK(launch_csr_to_bits(csr_off.as<uint32_t>(), csr_col.as<uint32_t>(), rows, W, term_bits.as<uint64_t>(), st));
    term_bits_content = content;
    return CFPQ_OK;
}

// ---------------------------------------------------------------------------
// Query planning: which n x n state blocks of C3 can be nonzero.
// ---------------------------------------------------------------------------
static uint32_t next_pow2(uint32_t x) {
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

int QueryDev::plan(std::string *err) {
    if (!g || g->n == 0) { *err = "no graph loaded"; return CFPQ_ERR_STATE; }
    if (rsm.max_terminal_plus1 > g->n_term) {
        *err = "the RSM reads a terminal >= the graph's n_terminals";
        return CFPQ_ERR_INVALID_ARG;
    }
    n = g->n;
    W = g->W;
    Q = rsm.Q;
    B = rsm.B;
    vpl = (uint32_t)vpl_for_words(W);
    if (!vpl) { *err = "unsupported row width"; return CFPQ_ERR_UNSUPPORTED; }
    lpr = std::min<uint32_t>(32u, next_pow2(((W / 2) + vpl - 1) / vpl));
    // reach[s][t]: t reachable from s by one or more RSM transitions (any
    // symbol).  Block (s,t) of M3 is OR over transitions s -l-> t of M2^l, so
    // block (s,t) of C3 = M3^+ can only be nonzero when reach[s][t].
    std::vector<uint8_t> reach((size_t)Q * Q, 0);
    for (const auto &t : rsm.tr) reach[(size_t)t.from * Q + t.to] = 1;
    for (uint32_t k = 0; k < Q; ++k)
        for (uint32_t i = 0; i < Q; ++i)
            if (reach[(size_t)i * Q + k])
                for (uint32_t j = 0; j < Q; ++j)
                    if (reach[(size_t)k * Q + j]) reach[(size_t)i * Q + j] = 1;
    blk_of.assign((size_t)Q * Q, -1);
    blocks.clear();
    for (uint32_t s = 0; s < Q; ++s)
        for (uint32_t t = 0; t < Q; ++t)
            if (reach[(size_t)s * Q + t]) {
                blk_of[(size_t)s * Q + t] = (int32_t)blocks.size();
                blocks.push_back({s, t});
            }
    // Levels (see cfpq_dev.cuh): strongly connected components of the state
    // graph, level = 1 + max level of the components a component has
    // transitions into; levels without blocks are dropped.
    std::vector<uint32_t> comp(Q);
    for (uint32_t s = 0; s < Q; ++s) {
        comp[s] = s;
        for (uint32_t t = 0; t < s; ++t)
            if (reach[(size_t)s * Q + t] && reach[(size_t)t * Q + s]) { comp[s] = comp[t]; break; }
    }
    std::vector<int32_t> clevel(Q, -1);
    // components in an order where every successor component comes first:
    // repeat relaxation (Q is small)
    bool changed_lv = true;
    for (uint32_t s = 0; s < Q; ++s) clevel[comp[s]] = 0;
    while (changed_lv) {
        changed_lv = false;
        for (const auto &t : rsm.tr) {
            const uint32_t a = comp[t.from], b = comp[t.to];
            if (a == b) continue;
            if (clevel[a] < clevel[b] + 1) { clevel[a] = clevel[b] + 1; changed_lv = true; }
        }
    }
    std::vector<int32_t> used(Q + 1, 0);
    for (const auto &bk : blocks) used[clevel[comp[bk.first]]] = 1;
    std::vector<int32_t> remap(Q + 1, -1);
    n_levels = 0;
    for (uint32_t L = 0; L <= Q; ++L)
        if (used[L]) remap[L] = (int32_t)n_levels++;
    if (n_levels == 0) n_levels = 1;
    if (n_levels > 64) { *err = "more than 64 block levels"; return CFPQ_ERR_UNSUPPORTED; }
    blk_level.assign(blocks.size(), 0);
    cyclic_mask = 0;
    for (size_t b = 0; b < blocks.size(); ++b) {
        const uint32_t s = blocks[b].first;
        blk_level[b] = (uint32_t)remap[clevel[comp[s]]];
        if (reach[(size_t)s * Q + s]) cyclic_mask |= 1ull << blk_level[b];
    }
    // Sources of block (s,t): transitions s -l-> u with u == t or t reachable from u.
    srcs.clear();
    n_tc_src = 0;
    // compacted inner dimension: every row up to n = 8192 (operands of at
    // most 2 n^2 bytes per source), half of the rows above, a multiple of 128
    // (full_kcap: every row, so that a product covering the new edges, whose
    // list can grow to n, stays compacted)
    kcap = (W * 64u <= 8192u || full_kcap) ? W * 64u : std::max<uint32_t>(128u, ((W * 32u) + 127u) & ~127u);
    if (tile_fp4) kcap = std::max<uint32_t>(kcap, 256u);  // E2M1 operand rows of at least one 128-byte TMA box
    blk_src0.assign(blocks.size(), 0);
    blk_nsrc.assign(blocks.size(), 0);
    for (size_t b = 0; b < blocks.size(); ++b) {
        const uint32_t s = blocks[b].first, t = blocks[b].second;
        blk_src0[b] = (uint32_t)srcs.size();
        for (const auto &tr : rsm.tr) {
            if (tr.from != s) continue;
            const uint32_t u = tr.to;
            const bool ident = (u == t);
            const int32_t rb = blk_of[(size_t)u * Q + t];
            if (!ident && rb < 0) continue;
            const uint32_t same = (rb >= 0 && blk_level[(size_t)rb] == blk_level[b]) ? 1u : 0u;
            srcs.push_back({tr.kind, tr.sym, ident ? 1u : 0u, rb, same, 0u, 0u, -1, 0u});
        }
        blk_nsrc[b] = (uint32_t)srcs.size() - blk_src0[b];
    }
    // Boxes read by some transition (bit 63: a box >= 63 is read).
    nt_read_mask = 0;
    for (const auto &tr : rsm.tr)
        if (tr.kind == 1) nt_read_mask |= tr.sym < 63u ? (1ull << tr.sym) : (1ull << 63);
    // Pure-terminal blocks: every source a direct terminal transition u -l-> t
    // (no closure block read), at most two labels.  Such a block equals the
    // union of those adjacencies, so its readers expand CSR rows.
    blk_pure_n.assign(blocks.size(), 0);
    blk_pure_lbl.assign(blocks.size() * 2, 0);
    for (size_t b = 0; b < blocks.size(); ++b) {
        bool pure = blk_nsrc[b] > 0 && blk_nsrc[b] <= 2;
        for (uint32_t k = 0; k < blk_nsrc[b] && pure; ++k) {
            const Src &sd = srcs[blk_src0[b] + k];
            pure = sd.rblk < 0 && sd.label_kind == 0 && sd.ident;
        }
        if (!pure) continue;
        blk_pure_n[b] = blk_nsrc[b];
        for (uint32_t k = 0; k < blk_nsrc[b]; ++k) blk_pure_lbl[b * 2 + k] = srcs[blk_src0[b] + k].label;
    }
    for (auto &sd : srcs) {
        sd.pure_rb = (sd.rblk >= 0 && !sd.ident && sd.label_kind == 1 && blk_pure_n[(size_t)sd.rblk] > 0) ? 1u : 0u;
        const bool tiles_ok = sd.rblk >= 0 && !sd.pure_rb;
        // tensor-core mode: the dirty-row channels of every source that reads
        // a (non-pure) closure block are tile products; new edges stay on the
        // row gather
        sd.dense = (closure_all_tiles(closure_mode) && tiles_ok) ? 1u : 0u;
        // AUTO: the same for a nonterminal source while its box's matrix is
        // dense (large queries only: a tile is 128 x 256)
        sd.box_switch =
            (closure_mode == CFPQ_CLOSURE_AUTO && sd.label_kind == 1 && tiles_ok && n >= kAutoTilesMinN) ? 1u : 0u;
        sd.tc_slot = (sd.dense || sd.box_switch) ? (int32_t)n_tc_src++ : -1;
        // the new edges of a nonterminal tile source get a job of their own
        // (channel 1, run when the tiles beat the gather: new_tiles_pay)
        sd.tc_slot_new = (sd.tc_slot >= 0 && sd.label_kind == 1 && !sd.same_level) ? (int32_t)n_tc_src++ : -1;
    }
    // a context's query holds full-size slots (2 n^2 bytes each) only up to
    // 96 GiB of them (at n = 65536: 11 slots; Dyck-4 in TC_FP8 mode has 10)
    if (full_kcap && W * 64u > 8192u && (uint64_t)n_tc_src * tc_slot_bytes() > (96ull << 30))
        kcap = std::max<uint32_t>(128u, ((W * 32u) + 127u) & ~127u);
    // Extraction blocks: (q0_b, f) for f final in box b.
    fblocks.clear();
    box_f0.assign(B, 0);
    box_nf.assign(B, 0);
    for (uint32_t b = 0; b < B; ++b) {
        box_f0[b] = (uint32_t)fblocks.size();
        const uint32_t q0 = rsm.box_start[b];
        for (uint32_t f = 0; f < Q; ++f)
            if (rsm.state_box[f] == b && rsm.final_[f] && blk_of[(size_t)q0 * Q + f] >= 0)
                fblocks.push_back((uint32_t)blk_of[(size_t)q0 * Q + f]);
        box_nf[b] = (uint32_t)fblocks.size() - box_f0[b];
    }
    n_eps = 0;
    for (uint32_t b = 0; b < B; ++b) n_eps += rsm.final_[rsm.box_start[b]] ? 1u : 0u;
    return CFPQ_OK;
}

uint64_t QueryDev::tc_slot_bytes() const {
    return (uint64_t)W * 64 * 8 + 256 + ((uint64_t)n + (uint64_t)W * 64) * tc_kstride();
}

uint64_t QueryDev::footprint() const {
    const uint64_t nblk = std::max<uint64_t>(blocks.size(), 1), bw = (uint64_t)n * W * 8;
    return nblk * bw + nblk * n * 4 + nblk * 4 + 2ull * B * bw + (uint64_t)B * n * 4 + B * 4 + 4096 +
           (uint64_t)n_tc_src * tc_slot_bytes();
}

int QueryDev::prepare(Allocator *A, std::string *err) {
    int rc = plan(err);
    if (rc) return rc;
    const size_t nblk = blocks.size();
    const size_t bw = (size_t)n * W * 8;
    if (!blk_mem.ensure(A, std::max<size_t>(nblk, 1) * bw, err) ||
        !stamp_mem.ensure(A, std::max<size_t>(nblk, 1) * n * 4, err) ||
        !last_mem.ensure(A, std::max<size_t>(nblk, 1) * 4, err) || !m2_mem.ensure(A, (size_t)B * bw, err) ||
        !a2_mem.ensure(A, (size_t)B * bw, err) || !a2it_mem.ensure(A, (size_t)B * n * 4, err) ||
        !boxit_mem.ensure(A, (size_t)B * 4, err) || !ctl_mem.ensure(A, sizeof(QCtl), err) ||
        !boxedge_mem.ensure(A, (size_t)B * 8, err) ||
        !ctl_ptr_mem.ensure(A, sizeof(QCtl *), err) ||
        !eps_mem.ensure(A, std::max<size_t>(n_eps, 1) * eps_desc_size(), err) ||
        !tc_mem.ensure(A, std::max<size_t>(n_tc_src * tc_slot_bytes(), 64), err))
        return CFPQ_ERR_OUT_OF_MEMORY;
    device_bytes = blk_mem.bytes + stamp_mem.bytes + last_mem.bytes + m2_mem.bytes + a2_mem.bytes + a2it_mem.bytes +
                   boxit_mem.bytes + (n_tc_src ? tc_mem.bytes : 0);
    std::vector<unsigned char> he(std::max<size_t>(n_eps, 1) * eps_desc_size());
    uint32_t k = 0;
    for (uint32_t b = 0; b < B; ++b) {
        if (!rsm.final_[rsm.box_start[b]]) continue;
        fill_eps_desc(he.data() + (size_t)k * eps_desc_size(), m2_ptr(b), a2_ptr(b),
                      a2it_mem.as<uint32_t>() + (size_t)b * n, boxit_mem.as<uint32_t>() + b, ctl(),
                      boxedge_mem.as<unsigned long long>() + b, n, W);
        ++k;
    }
    QCtl *cp = ctl();
    ENG_CK(cudaMemcpyAsync(eps_mem.p, he.data(), he.size(), cudaMemcpyHostToDevice, A->stream));
    ENG_CK(cudaMemcpyAsync(ctl_ptr_mem.p, &cp, sizeof(cp), cudaMemcpyHostToDevice, A->stream));
    ENG_CK(cudaStreamSynchronize(A->stream));
    prepared = true;
    graph_generation = g->generation;
    return CFPQ_OK;
}

int QueryDev::refresh_graph_caches(Allocator *A, cudaStream_t st, std::string *err, bool *moved) {
    bool need_term_bits = false, need_nonempty = false;
    for (const auto &sdesc : srcs) {
        need_term_bits |= (sdesc.dense && sdesc.label_kind == 0);
        need_nonempty |= sdesc.pure_rb != 0;
    }
    const void *p_ne = g->nonempty.p, *p_tb = g->term_bits.p;
    if (need_nonempty)
        if (int rc = g->ensure_nonempty(A, st, err)) return rc;
    if (need_term_bits)
        if (int rc = g->ensure_term_bits(A, st, err)) return rc;
    *moved = (need_nonempty && g->nonempty.p != p_ne) || (need_term_bits && g->term_bits.p != p_tb);
    return CFPQ_OK;
}

int QueryDev::prepare_small(Allocator *A, cudaStream_t st, uint32_t max_iter, uint32_t max_passes,
                            std::string *err) {
    small_ok = false;
    const uint32_t nblk = (uint32_t)blocks.size();
    if (W > 8 || closure_all_tiles(closure_mode)) return CFPQ_OK;
    const size_t smem = small_smem_bytes(n, W, B, nblk);
    const size_t limit = small_smem_limit();
    if (smem == 0 || smem > limit) return CFPQ_OK;
    // arrays: level, src0, nsrc (per block), f0, nf, nullable (per box), fblocks
    std::vector<uint32_t> arr;
    const size_t off_level = arr.size();
    arr.insert(arr.end(), blk_level.begin(), blk_level.end());
    const size_t off_src0 = arr.size();
    arr.insert(arr.end(), blk_src0.begin(), blk_src0.end());
    const size_t off_nsrc = arr.size();
    arr.insert(arr.end(), blk_nsrc.begin(), blk_nsrc.end());
    const size_t off_f0 = arr.size();
    arr.insert(arr.end(), box_f0.begin(), box_f0.end());
    const size_t off_nf = arr.size();
    arr.insert(arr.end(), box_nf.begin(), box_nf.end());
    const size_t off_null = arr.size();
    for (uint32_t b = 0; b < B; ++b) arr.push_back(rsm.final_[rsm.box_start[b]] ? 1u : 0u);
    const size_t off_fb = arr.size();
    arr.insert(arr.end(), fblocks.begin(), fblocks.end());
    while (arr.size() % 4) arr.push_back(0);  // 16-byte alignment of the sources that follow
    const size_t ssz = small_src_size();
    std::vector<unsigned char> blob(arr.size() * 4 + std::max<size_t>(srcs.size(), 1) * ssz);
    memcpy(blob.data(), arr.data(), arr.size() * 4);
    for (size_t k = 0; k < srcs.size(); ++k)
        fill_small_src(blob.data() + arr.size() * 4 + k * ssz, srcs[k].label_kind, srcs[k].label, srcs[k].ident,
                       srcs[k].same_level, srcs[k].rblk);
    if (!small_arrays.ensure(A, blob.size(), err) || !small_desc.ensure(A, small_desc_size(), err))
        return CFPQ_ERR_OUT_OF_MEMORY;
    const uint32_t *dev_arr = small_arrays.as<uint32_t>();
    const SmallSrc *dev_src = reinterpret_cast<const SmallSrc *>(small_arrays.as<unsigned char>() + arr.size() * 4);
    std::vector<unsigned char> desc(small_desc_size());
    build_small_desc(desc.data(), n, W, B, nblk, n_levels, cyclic_mask, max_iter, max_passes, dev_arr, dev_src,
                     off_level, off_src0, off_nsrc, off_f0, off_nf, off_fb, off_null, g->csr_off.as<uint32_t>(),
                     g->csr_col.as<uint32_t>(), blk_mem.as<uint64_t>(), m2_mem.as<uint64_t>(), ctl());
    ENG_CK(cudaMemcpyAsync(small_arrays.p, blob.data(), blob.size(), cudaMemcpyHostToDevice, st));
    ENG_CK(cudaMemcpyAsync(small_desc.p, desc.data(), desc.size(), cudaMemcpyHostToDevice, st));
    ENG_CK(cudaStreamSynchronize(st));
    small_smem = smem;
    small_ok = true;
    return CFPQ_OK;
}

int QueryDev::enqueue_init(cudaStream_t st, uint32_t max_iter, uint32_t max_rounds, uint32_t max_passes) {
    std::string *err = nullptr;
    const size_t nblk = blocks.size();
    if (nblk) {
        ENG_CK(cudaMemsetAsync(blk_mem.p, 0, nblk * (size_t)n * W * 8, st));
        ENG_CK(cudaMemsetAsync(stamp_mem.p, 0, nblk * (size_t)n * 4, st));
        ENG_CK(cudaMemsetAsync(last_mem.p, 0, nblk * 4, st));
    }
    ENG_CK(cudaMemsetAsync(m2_mem.p, 0, (size_t)B * n * W * 8, st));
    ENG_CK(cudaMemsetAsync(a2it_mem.p, 0, (size_t)B * n * 4, st));
    ENG_CK(cudaMemsetAsync(boxit_mem.p, 0, (size_t)B * 4, st));
    ENG_CK(cudaMemsetAsync(boxedge_mem.p, 0, (size_t)B * 8, st));
    for (uint32_t k = 0; k < n_tc_src; ++k) ENG_CK(cudaMemsetAsync(tc_kcount(k), 0, 8, st));
    // per-box edge counts: the dense-box mask drives AUTO's tile switch and
    // the column slices of the row gather in every mode
    ENG_CK(launch_ctl_reset(ctl_ptr_mem.as<QCtl *>(), 1, max_iter, max_rounds, max_passes, n_levels, cyclic_mask,
                            boxedge_mem.as<unsigned long long>(), B, n, boxit_mem.as<uint32_t>(), nt_read_mask, st));
    ENG_CK(launch_eps_init(eps_mem.p, n_eps, 152, st));
    if (seeded)
        ENG_CK(launch_seed_apply(seed_mem.as<uint64_t>(), m2_mem.as<uint64_t>(), a2_mem.as<uint64_t>(),
                                 a2it_mem.as<uint32_t>(), boxit_mem.as<uint32_t>(), ctl(),
                                 boxedge_mem.as<unsigned long long>(), n, W, B, st));
    return CFPQ_OK;
}

// ---------------------------------------------------------------------------
// Executor.
// ---------------------------------------------------------------------------
static int vpl_index(uint32_t vpl) {
    switch (vpl) {
        case 1: return 0;
        case 2: return 1;
        case 4: return 2;
        case 8: return 3;
        default: return 4;
    }
}
static const int kVplOf[5] = {1, 2, 4, 8, 16};

int Executor::assemble(Allocator *A, cudaStream_t st, std::string *err) {
    const uint32_t nq = (uint32_t)qs.size();
    if (!ctl_ptrs.ensure(A, std::max<uint32_t>(nq, 1) * sizeof(QCtl *), err) ||
        !mirror.ensure(A, std::max<uint32_t>(nq, 1) * sizeof(QCtl), err) || !running.ensure(A, 16, err) ||
        !tc_err.ensure(A, 16, err) || !done_counter.ensure(A, 16, err))
        return CFPQ_ERR_OUT_OF_MEMORY;
    uint32_t maxL1 = 2;
    for (QueryDev *q : qs) maxL1 = std::max(maxL1, q->n_levels + 1);
    std::vector<QCtl *> hp;
    std::vector<SrcDesc> hs;
    std::vector<GItem> hi[kClasses];
    std::vector<FDesc> hf;
    std::vector<XItem> hx[kClasses];
    std::vector<TcJob> hj;
    // static tables
    std::vector<uint32_t> g_lvl[kClasses], x_rng[kClasses];
    for (int v = 0; v < kClasses; ++v) {
        g_lvl[v].assign((size_t)nq * maxL1, 0);
        x_rng[v].assign((size_t)nq + 1, 0);
    }
    std::vector<uint32_t> t_lvl((size_t)nq * maxL1, 0), t_lvl_tiles((size_t)nq * maxL1, 0);
    max_tc_tiles = 0;
    max_tc_w = 0;
    // one tile kernel per executor: the product kernel is launched for it
    tile_kind = kTileFp8Pair;
    bool kind_set = false;
    for (QueryDev *q : qs) {
        if (!q->n_tc_src) continue;
        if (kind_set && q->tile_kind != tile_kind) {
            *err = "queries of one executor use different tile kernels";
            return CFPQ_ERR_INVALID_ARG;
        }
        tile_kind = q->tile_kind;
        kind_set = true;
    }
    uint32_t n_maps = 0;
    size_t n_newcols = 0;  // words of the channel-1 jobs' column bitmaps and counts
    std::vector<size_t> newcols_of;
    uint32_t live_bound[kClasses] = {0};
    for (uint32_t qi = 0; qi < nq; ++qi) {
        QueryDev &q = *qs[qi];
        GraphDev &g = *q.g;
        QCtl *cp = q.ctl();
        hp.push_back(cp);
        bool moved = false;
        if (int rc = q.refresh_graph_caches(A, st, err, &moved)) return rc;
        const uint32_t base = (uint32_t)hs.size();
        for (const auto &sd : q.srcs) {
            SrcDesc d;
            memset(&d, 0, sizeof(d));
            if (sd.label_kind == 0) {
                d.csr_off = g.csr_off.as<uint32_t>() + (size_t)sd.label * q.n;
                d.csr_col = g.csr_col.as<uint32_t>();
            } else {
                d.nt_all = q.m2_ptr(sd.label);
                d.nt_new = q.a2_ptr(sd.label);
                d.nt_new_it = q.a2it_mem.as<uint32_t>() + (size_t)sd.label * q.n;
                d.box_new_it = q.boxit_mem.as<uint32_t>() + sd.label;
            }
            if (sd.rblk >= 0) {
                d.rblk = q.blk_ptr((uint32_t)sd.rblk);
                d.rstamp = q.stamp_ptr((uint32_t)sd.rblk);
                d.rlast = q.last_mem.as<uint32_t>() + sd.rblk;
            }
            if (sd.pure_rb) {
                const size_t rb = (size_t)sd.rblk;
                d.pure_n = q.blk_pure_n[rb];
                for (uint32_t p = 0; p < d.pure_n; ++p) {
                    d.pure_off[p] = g.csr_off.as<uint32_t>() + (size_t)q.blk_pure_lbl[rb * 2 + p] * q.n;
                    d.pure_mask[p] = g.nonempty.as<uint64_t>() + (size_t)q.blk_pure_lbl[rb * 2 + p] * q.W;
                }
                d.pure_col = g.csr_col.as<uint32_t>();
            }
            d.ident = sd.ident;
            d.same_level = sd.same_level;
            d.dense = sd.dense;
            d.box_switch = sd.box_switch;
            d.label_box = sd.label_kind == 1 ? sd.label : 0u;
            if (sd.tc_slot_new >= 0) {
                // the channel-1 job's column bitmap and counts: W + 8 words of
                // the executor's newcols buffer (offsets, made pointers below)
                d.tile_new = 1u;
                d.tc_kcap = q.kcap;
                d.tc_ratio = q.tile_ratio;
                d.tc_kcount = q.tc_kcount((uint32_t)sd.tc_slot_new);
                d.tc_mcount = reinterpret_cast<const unsigned long long *>((size_t)(n_newcols + q.W));
                d.tc_ecount = reinterpret_cast<const unsigned long long *>((size_t)(n_newcols + q.W + 1));
                newcols_of.push_back(n_newcols);
                n_newcols += q.W + 8u;
            }
            hs.push_back(d);
        }
        const int vi = vpl_index(q.vpl);
        const uint32_t rows_per_step = 8u * (32u / q.lpr);
        // rows per work item (extraction; the gather's narrow rows), times the
        // executor's item scale (the server's larger items keep its frequent
        // re-assembly cheap), at most 1024
        const uint32_t rpi = std::min<uint32_t>(1024u, std::max<uint32_t>(64u, rows_per_step * 4u) * item_scale);
        // product jobs: tcgen05 tiles of 128 rows x 256 columns
        const uint32_t tiles_m = (q.n + 127u) / 128u, tiles_n = (q.n + 255u) / 256u;
        for (uint32_t L = 0; L <= q.n_levels; ++L) {
            for (int v = 0; v < kClasses; ++v) g_lvl[v][(size_t)qi * maxL1 + L] = (uint32_t)hi[v].size();
            t_lvl[(size_t)qi * maxL1 + L] = (uint32_t)hj.size();
            if (L == q.n_levels) break;
            uint32_t lvl_tiles = 0;
            for (size_t b = 0; b < q.blocks.size(); ++b) {
                if (q.blk_level[b] != L || q.blk_nsrc[b] == 0) continue;
                bool has_nt = false;
                for (uint32_t k = 0; k < q.blk_nsrc[b]; ++k) {
                    const auto &sd = q.srcs[q.blk_src0[b] + k];
                    // the general kernel variant: nonterminal adjacency rows, pure-terminal blocks
                    has_nt |= (sd.label_kind != 0) || sd.pure_rb;
                }
                const int cls = 2 * vi + (has_nt ? 1 : 0);
                // wide rows of nonterminal blocks: the adjacency columns are
                // split over several items, so that rows with thousands of new
                // edges (hubs) spread over several CTAs
                const uint32_t nvec = q.W / 2u;
                // Boxes (first 32) whose dense adjacency this block's row gather
                // enumerates into OR-ed closure rows: nonterminal sources reading a
                // closure block (not a pure-terminal one) with no tile job.  A hub
                // row of such a box costs thousands of row ORs, which the column
                // slices spread over several units.  (Measured on Dyck-4 n = 65536:
                // slicing every block with a nonterminal source cost AUTO
                // 1.22 -> 1.28 s with 4 slices and 1.46 s with 8, as the warp units
                // already balance the lighter blocks.)
                uint32_t nt_boxes = 0;
                for (uint32_t k = 0; k < q.blk_nsrc[b]; ++k) {
                    const auto &sd = q.srcs[q.blk_src0[b] + k];
                    if (sd.label_kind != 0 && sd.label < 32u && sd.rblk >= 0 && !sd.pure_rb && sd.tc_slot < 0)
                        nt_boxes |= 1u << sd.label;
                }
                const bool sliceable = has_nt && q.W >= 128u && nt_boxes != 0u;
                // 4 slices: measured on Dyck-4 n = 65536 (1: 2.93 s, 2: 2.56, 3: 2.53,
                // 4: 2.50, 8: 2.72, 16: 3.33); more slices cost atomic merges
                uint32_t n_slices = sliceable ? 4u : 1u;
                if (q.gather_slices) n_slices = sliceable ? std::min<uint32_t>(q.gather_slices, 16u) : 1u;
                // nonterminal blocks of wide rows: 128-row items (measured on
                // Dyck-4; the CSR blocks of the RPQ bench prefer 64)
                const uint32_t rows_item =
                    (has_nt && q.W >= 256u) ? std::min<uint32_t>(1024u, std::max<uint32_t>(rpi, 128u * item_scale)) : rpi;
                // the gather keeps an item's row mask in 16 words of shared memory
                if (rows_item > 1024u || rows_item % 64u != 0u) {
                    *err = "gather items: rows per item must be a multiple of 64 and at most 1024";
                    return CFPQ_ERR_INVALID_ARG;
                }
                // slice-major: CTAs running side by side enumerate the same
                // columns of the adjacency, so the closure rows they read (a
                // 1/n_slices share of the block read) stay in L2
                for (uint32_t sl = 0; sl < n_slices; ++sl)
                for (uint32_t r0 = 0; r0 < q.n; r0 += rows_item) {
                    GItem it;
                    it.out = q.blk_ptr((uint32_t)b);
                    it.out_stamp = q.stamp_ptr((uint32_t)b);
                    it.out_last = q.last_mem.as<uint32_t>() + b;
                    it.ctl = cp;
                    it.rmask = q.restricted ? q.reach_ptr(q.blocks[b].first) : nullptr;
                    it.src0 = base + q.blk_src0[b];
                    it.nsrc = q.blk_nsrc[b];
                    it.row0 = r0;
                    it.row1 = std::min(q.n, r0 + rows_item);
                    it.W = q.W;
                    it.lpr = q.lpr;
                    it.level = L;
                    it.slice = (nvec * sl / n_slices) | ((nvec * (sl + 1) / n_slices) << 16);
                    it.nt_boxes = nt_boxes;
                    it.pad = 0;
                    hi[cls].push_back(it);
                }
                // tile sources of this block: one product job for the dirty-row
                // channel (4 on a cyclic level's own blocks, else 2)
                for (uint32_t k = 0; k < q.blk_nsrc[b]; ++k) {
                    const auto &sd = q.srcs[q.blk_src0[b] + k];
                    if (sd.tc_slot < 0) continue;
                    const SrcDesc &d = hs[base + q.blk_src0[b] + k];
                    TcJob j;
                    memset(&j, 0, sizeof(j));
                    j.out = q.blk_ptr((uint32_t)b);
                    j.out_stamp = q.stamp_ptr((uint32_t)b);
                    j.out_last = q.last_mem.as<uint32_t>() + b;
                    if (sd.label_kind == 0) {
                        j.A = g.term_bits.as<uint64_t>() + (size_t)sd.label * q.n * q.W;
                        j.box_new_it = nullptr;
                    } else {
                        j.A = q.m2_ptr(sd.label);
                        j.box_new_it = d.box_new_it;
                    }
                    j.a_it = nullptr;
                    j.B = d.rblk;
                    j.b_stamp = d.rstamp;
                    j.rlast = d.rlast;
                    j.ctl = cp;
                    j.n = q.n;
                    j.W = q.W;
                    j.ident = 0u;
                    j.chan = sd.same_level ? 4u : 2u;
                    j.level = L;
                    j.same_level = sd.same_level;
                    j.tiles_m = tiles_m;
                    j.tiles_n = tiles_n;
                    j.box = sd.label_kind == 1 ? sd.label : 0u;
                    j.switchable = sd.box_switch;
                    j.kcap = q.kcap;
                    j.kstride = q.tc_kstride();
                    j.fp4 = q.tile_fp4 ? 1u : 0u;
                    j.tile_ratio = q.tile_ratio;
                    j.ys = q.tc_ys((uint32_t)sd.tc_slot);
                    j.kcount = q.tc_kcount((uint32_t)sd.tc_slot);
                    j.a8 = q.tc_a8((uint32_t)sd.tc_slot);
                    j.b8 = q.tc_b8((uint32_t)sd.tc_slot);
                    j.map = n_maps++;
                    j.tile0 = lvl_tiles;
                    lvl_tiles += tiles_m * tiles_n;
                    hj.push_back(j);
                    max_tc_w = std::max(max_tc_w, q.W);
                    if (sd.tc_slot_new >= 0) {
                        // channel 1: A2 rows (new in the iteration) x whole rows of B
                        const size_t off = reinterpret_cast<size_t>(d.tc_mcount) - q.W;
                        j.chan = 1u;
                        j.A = q.a2_ptr(sd.label);
                        j.a_it = q.a2it_mem.as<uint32_t>() + (size_t)sd.label * q.n;
                        j.b_stamp = nullptr;
                        j.covers_new = 1u;
                        j.newcols = reinterpret_cast<uint64_t *>(off);
                        j.mcount = reinterpret_cast<unsigned long long *>(off + q.W);
                        j.ecount = reinterpret_cast<unsigned long long *>(off + q.W + 1);
                        j.xs = q.tc_xs((uint32_t)sd.tc_slot_new);
                        j.ys = q.tc_ys((uint32_t)sd.tc_slot_new);
                        j.kcount = q.tc_kcount((uint32_t)sd.tc_slot_new);
                        j.a8 = q.tc_a8((uint32_t)sd.tc_slot_new);
                        j.b8 = q.tc_b8((uint32_t)sd.tc_slot_new);
                        j.map = n_maps++;
                        j.tile0 = lvl_tiles;
                        lvl_tiles += tiles_m * tiles_n;
                        hj.push_back(j);
                    }
                }
            }
            t_lvl_tiles[(size_t)qi * maxL1 + L] = lvl_tiles;
        }
        for (uint32_t L = q.n_levels + 1; L < maxL1; ++L) {
            for (int v = 0; v < kClasses; ++v)
                g_lvl[v][(size_t)qi * maxL1 + L] = g_lvl[v][(size_t)qi * maxL1 + q.n_levels];
            t_lvl[(size_t)qi * maxL1 + L] = t_lvl[(size_t)qi * maxL1 + q.n_levels];
        }
        uint32_t qtiles = 0;
        for (uint32_t L = 0; L < q.n_levels; ++L) qtiles = std::max(qtiles, t_lvl_tiles[(size_t)qi * maxL1 + L]);
        max_tc_tiles += qtiles;
        for (int c = 0; c < kClasses; ++c) {
            uint32_t mx = 0;
            for (uint32_t L = 0; L < q.n_levels; ++L)
                mx = std::max(mx, g_lvl[c][(size_t)qi * maxL1 + L + 1] - g_lvl[c][(size_t)qi * maxL1 + L]);
            live_bound[c] += mx;
        }
        const uint32_t fbase = (uint32_t)hf.size();
        for (uint32_t fb : q.fblocks) hf.push_back(FDesc{q.blk_ptr(fb), q.stamp_ptr(fb)});
        for (int v = 0; v < kClasses; ++v) x_rng[v][qi] = (uint32_t)hx[v].size();
        for (uint32_t b = 0; b < q.B; ++b) {
            if (q.box_nf[b] == 0) continue;
            for (uint32_t r0 = 0; r0 < q.n; r0 += rpi) {
                XItem x;
                x.box_edges = q.boxedge_mem.as<unsigned long long>() + b;
                x.m2 = q.m2_ptr(b);
                x.a2 = q.a2_ptr(b);
                x.a2_it = q.a2it_mem.as<uint32_t>() + (size_t)b * q.n;
                x.box_new_it = q.boxit_mem.as<uint32_t>() + b;
                x.ctl = cp;
                x.f0 = fbase + q.box_f0[b];
                x.nf = q.box_nf[b];
                x.row0 = r0;
                x.row1 = std::min(q.n, r0 + rpi);
                x.W = q.W;
                x.lpr = q.lpr;
                hx[2 * vi].push_back(x);
            }
        }
    }
    for (int v = 0; v < kClasses; ++v) x_rng[v][nq] = (uint32_t)hx[v].size();
    auto upload = [&](DBuf &buf, const void *h, size_t bytes) -> int {
        if (!buf.ensure(A, std::max<size_t>(bytes, 64), err)) return CFPQ_ERR_OUT_OF_MEMORY;
        if (bytes) ENG_CK(cudaMemcpyAsync(buf.p, h, bytes, cudaMemcpyHostToDevice, st));
        return CFPQ_OK;
    };
    int rc;
    newcols_words = n_newcols;
    if (n_newcols) {
        if (!newcols.ensure(A, n_newcols * 8, err)) return CFPQ_ERR_OUT_OF_MEMORY;
        uint64_t *nb = newcols.as<uint64_t>();
        auto fix = [nb](auto *&p) {
            using T = std::remove_pointer_t<std::remove_reference_t<decltype(p)>>;
            p = reinterpret_cast<T *>(nb + reinterpret_cast<size_t>(p));
        };
        for (auto &j : hj)
            if (j.covers_new) {
                fix(j.newcols);
                fix(j.mcount);
                fix(j.ecount);
            }
        for (auto &d : hs)
            if (d.tile_new) {
                fix(d.tc_mcount);
                fix(d.tc_ecount);
            }
    }
    if ((rc = upload(ctl_ptrs, hp.data(), hp.size() * sizeof(QCtl *)))) return rc;
    if ((rc = upload(srcs, hs.data(), hs.size() * sizeof(SrcDesc)))) return rc;
    if ((rc = upload(fds, hf.data(), hf.size() * sizeof(FDesc)))) return rc;
    if ((rc = upload(tcjobs, hj.data(), hj.size() * sizeof(TcJob)))) return rc;
    n_tcjobs = (uint32_t)hj.size();
    // TMA descriptors of the jobs' FP8 operands (a8, b8 per job)
    if (n_maps) {
        std::vector<unsigned char> hm((size_t)n_maps * 2 * tc_map_bytes());
        ENG_CK(tc_encode_maps(hj.data(), (uint32_t)hj.size(), hm.data()));
        if ((rc = upload(tcmaps, hm.data(), hm.size()))) return rc;
    }
    for (int v = 0; v < kClasses; ++v) {
        max_live[v] = live_bound[v];
        n_items[v] = (uint32_t)hi[v].size();
        n_xitems[v] = (uint32_t)hx[v].size();
        if ((rc = upload(items[v], hi[v].data(), hi[v].size() * sizeof(GItem)))) return rc;
        if ((rc = upload(xitems[v], hx[v].data(), hx[v].size() * sizeof(XItem)))) return rc;
    }
    // tables: one buffer, static part then the per-pass part
    const size_t nqa = std::max<uint32_t>(nq, 1), lv = nqa * maxL1;
    const size_t words = kClasses * lv + kClasses * (nqa + 1) + 2 * lv  // static
                         + 2 * kClasses + 2 * kClasses * nqa              // gather lists and unit counters
                         + kClasses + 2 * kClasses * nqa                  // extraction lists
                         + 1 + 3 * nqa                                    // tensor-core lists
                         + 1 + hj.size();                                 // active tile jobs
    std::vector<uint32_t> ht(words, 0);
    size_t o = 0;
    memset(&T, 0, sizeof(T));
    T.nq = nq;
    T.maxL1 = maxL1;
    uint32_t *dbase = nullptr;
    if (!tables.ensure(A, words * 4, err)) return CFPQ_ERR_OUT_OF_MEMORY;
    dbase = tables.as<uint32_t>();
    auto take = [&](size_t cnt) {
        uint32_t *p = dbase + o;
        o += cnt;
        return p;
    };
    for (int v = 0; v < kClasses; ++v) {
        std::copy(g_lvl[v].begin(), g_lvl[v].end(), ht.begin() + o);
        T.g_lvl[v] = take(lv);
    }
    for (int v = 0; v < kClasses; ++v) {
        std::copy(x_rng[v].begin(), x_rng[v].end(), ht.begin() + o);
        T.x_rng[v] = take(nqa + 1);
    }
    std::copy(t_lvl.begin(), t_lvl.end(), ht.begin() + o);
    T.t_lvl = take(lv);
    std::copy(t_lvl_tiles.begin(), t_lvl_tiles.end(), ht.begin() + o);
    T.t_lvl_tiles = take(lv);
    T.g_total = take(kClasses);
    T.g_next = take(kClasses);
    for (int v = 0; v < kClasses; ++v) T.g_pre[v] = take(nqa);
    for (int v = 0; v < kClasses; ++v) T.g_beg[v] = take(nqa);
    T.x_total = take(kClasses);
    for (int v = 0; v < kClasses; ++v) T.x_pre[v] = take(nqa);
    for (int v = 0; v < kClasses; ++v) T.x_beg[v] = take(nqa);
    T.t_total = take(1);
    T.t_pre = take(nqa);
    T.t_job_beg = take(nqa);
    T.t_job_end = take(nqa);
    T.aj_n = take(1);
    T.aj = take(hj.size());
    T.jobs = hj.empty() ? nullptr : tcjobs.as<TcJob>();
    ENG_CK(cudaMemcpyAsync(dbase, ht.data(), words * 4, cudaMemcpyHostToDevice, st));
    ENG_CK(cudaMemsetAsync(tc_err.p, 0, 16, st));
    ENG_CK(cudaMemsetAsync(done_counter.p, 0, 16, st));
    if (n_tcjobs) ENG_CK(prepare_tc_launch());
    ENG_CK(prepare_gather_launch());
    ENG_CK(cudaStreamSynchronize(st));
    drop_graph();
    built = true;
    return CFPQ_OK;
}

int Executor::enqueue_prologue(cudaStream_t st, uint32_t max_iter, uint32_t max_rounds, uint32_t max_passes) {
    for (QueryDev *q : qs)
        if (int rc = q->enqueue_init(st, max_iter, max_rounds, max_passes)) return rc;
    return enqueue_lists(st);
}

int Executor::enqueue_lists(cudaStream_t st) {
    std::string *err = nullptr;
    ENG_CK(launch_control(ctl_ptrs.as<QCtl *>(), (uint32_t)qs.size(), mirror.as<QCtl>(), 0, 0, nullptr, T, 0, st));
    return CFPQ_OK;
}

int Executor::enqueue_pass(cudaStream_t st, cudaGraphConditionalHandle h, int use_handle, int *running_out,
                           const cudaEvent_t *ev) {
    std::string *err = nullptr;
    // Tile operands first: the rows the tile jobs multiply were final before
    // this pass (lower levels, or the previous pass of a cyclic level), and a
    // gather whose source's new edges the tiles take needs the job's list.
    if (ev) ENG_CK(cudaEventRecord(ev[0], st));
    if (n_tcjobs) {
        if (newcols_words) ENG_CK(cudaMemsetAsync(newcols.p, 0, newcols_words * 8, st));
        ENG_CK(launch_tc_compact(tcjobs.as<TcJob>(), T, max_tc_w, tc_err.as<int>(), st));
    }
    if (ev) ENG_CK(cudaEventRecord(ev[1], st));
    for (int c = 0; c < kClasses; ++c)
        ENG_CK(launch_gather(kVplOf[c / 2], (c & 1) != 0, items[c].as<GItem>(), max_live[c], srcs.as<SrcDesc>(), T, c,
                             st));
    if (ev) ENG_CK(cudaEventRecord(ev[2], st));
    if (n_tcjobs) {
        ENG_CK(launch_tc_product(false, tcjobs.as<TcJob>(), max_tc_tiles, T, tc_err.as<int>(), st));
        ENG_CK(launch_tc_product_tma(tcjobs.as<TcJob>(), tcmaps.p, max_tc_tiles, T, tc_err.as<int>(), st, tile_kind));
    }
    if (ev) ENG_CK(cudaEventRecord(ev[3], st));
    // the last extraction launch of the pass also runs the loop control
    int last_x = -1;
    for (int c = 0; c < kClasses; c += 2)
        if (n_xitems[c]) last_x = c;
    for (int c = 0; c < kClasses; c += 2) {
        const bool fuse = c == last_x;
        ENG_CK(launch_extract(kVplOf[c / 2], xitems[c].as<XItem>(), n_xitems[c], fds.as<FDesc>(), T, c,
                              fuse ? ctl_ptrs.as<QCtl *>() : nullptr, (uint32_t)qs.size(), mirror.as<QCtl>(), h,
                              use_handle, running_out, done_counter.as<unsigned int>(), st));
    }
    if (last_x < 0)
        ENG_CK(launch_control(ctl_ptrs.as<QCtl *>(), (uint32_t)qs.size(), mirror.as<QCtl>(), h, use_handle,
                              running_out, T, 1, st));
    return CFPQ_OK;
}

int Executor::build_graph(cudaStream_t st, uint32_t max_iter, uint32_t max_rounds, uint32_t max_passes,
                          std::string *err) {
    drop_graph();
    if (!cap_stream) ENG_CK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    // Everything the graph reads was uploaded on `st`; order the capture after it.
    ENG_CK(cudaStreamSynchronize(st));
    const cudaStream_t cs = cap_stream;
    cudaGraph_t prologue = nullptr;
    ENG_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_prologue(cs, max_iter, max_rounds, max_passes);
    const uint32_t kPassesPerLoop = kLoopUnroll;
    cudaError_t ce = cudaStreamEndCapture(cs, &prologue);
    if (rc || ce != cudaSuccess) {
        if (prologue) cudaGraphDestroy(prologue);
        if (err) *err = std::string("prologue capture failed: ") + cudaGetErrorString(ce);
        return CFPQ_ERR_CUDA;
    }
    ENG_CK(cudaGraphCreate(&graph, 0));
    cudaGraphNode_t pro_node, loop_node;
    ce = cudaGraphAddChildGraphNode(&pro_node, graph, nullptr, 0, prologue);
    cudaGraphDestroy(prologue);
    ENG_CK(ce);
    cudaGraphConditionalHandle handle;
    ENG_CK(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
    // cudaGraphNodeParams holds a union with a deleted default constructor.
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    memset(cp_raw, 0, sizeof(cp_raw));
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    ENG_CK(cudaGraphAddNode(&loop_node, graph, &pro_node, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ENG_CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    // kPassesPerLoop passes per evaluation of the while node: a pass after the
    // loop finished finds no live work and leaves the control state unchanged
    for (uint32_t p = 0; p < kPassesPerLoop && rc == 0; ++p) rc = enqueue_pass(cs, handle, 1, nullptr);
    cudaGraph_t body_out = body;
    ce = cudaStreamEndCapture(cs, &body_out);
    if (rc || ce != cudaSuccess) {
        if (err) *err = std::string("loop body capture failed: ") + cudaGetErrorString(ce);
        drop_graph();
        return CFPQ_ERR_CUDA;
    }
    ENG_CK(cudaGraphInstantiate(&exec, graph, 0));
    return CFPQ_OK;
}

int Executor::read_ctls(cudaStream_t st, std::vector<QCtl> *out, int *tc_error) {
    std::string *err = nullptr;
    out->resize(qs.size());
    if (qs.empty()) return CFPQ_OK;
    ENG_CK(cudaMemcpyAsync(out->data(), mirror.p, qs.size() * sizeof(QCtl), cudaMemcpyDeviceToHost, st));
    int te = 0;
    if (tc_error && n_tcjobs) ENG_CK(cudaMemcpyAsync(&te, tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    ENG_CK(cudaStreamSynchronize(st));
    if (tc_error) *tc_error = te;
    return CFPQ_OK;
}

}  // namespace cfpq
