// cfpq_engine.cuh -- host-side engine of libcfpq (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/cfpq.h"
#include "cfpq_dev.cuh"

// CUDA call inside a function returning a CFPQ status (with std::string *err in scope).
#define ENG_CK(call)                                                                          \
    do {                                                                                      \
        cudaError_t _e = (call);                                                              \
        if (_e != cudaSuccess) {                                                              \
            if (err) *err = std::string(#call) + ": " + cudaGetErrorString(_e);               \
            return CFPQ_ERR_CUDA;                                                             \
        }                                                                                     \
    } while (0)

namespace cfpq {

// ---- kernel launchers (cfpq_kernels.cu) ----
int vpl_for_words(uint32_t W);
cudaError_t launch_gather(int vpl, bool nt, const GItem *items, uint32_t n_items, const SrcDesc *srcs,
                          const ExecTables &T, int cls, cudaStream_t st);
cudaError_t launch_extract(int vpl, const XItem *items, uint32_t n_items, const FDesc *fds, const ExecTables &T,
                           int cls, QCtl *const *ctls, uint32_t nq, QCtl *mirror, cudaGraphConditionalHandle h,
                           int use_handle, int *running_out, unsigned int *done_counter, cudaStream_t st);
cudaError_t launch_control(QCtl *const *ctls, uint32_t nq, QCtl *mirror, cudaGraphConditionalHandle h, int use_handle,
                           int *running_out, const ExecTables &T, int advance, cudaStream_t st);
cudaError_t launch_tc_product(bool int8, const TcJob *jobs, uint32_t max_tiles, const ExecTables &T, int *err_flag,
                              cudaStream_t st);
// Per pass, before the products: list each live job's dirty B rows and
// expand A's columns and B's rows at them to FP8 (max_w = the largest W).
cudaError_t launch_tc_compact(const TcJob *jobs, const ExecTables &T, uint32_t max_w, int *err_flag, cudaStream_t st);
// Products of the compacted jobs: TMA-fed tcgen05 pipeline (maps = the
// jobs' tensor maps, two per job, from tc_encode_maps).
cudaError_t launch_tc_product_tma(const TcJob *jobs, const void *maps, uint32_t max_tiles, const ExecTables &T,
                                  int *err_flag, cudaStream_t st, uint32_t tile_kind);
// Bytes of one tensor map; encode the a8/b8 maps of every job with buffers
// (job.map indexes pairs) into host memory.
size_t tc_map_bytes();
cudaError_t tc_encode_maps(const TcJob *jobs, uint32_t n_jobs, void *out);
cudaError_t prepare_tc_launch();
// One thread waits on an mbarrier nothing arrives at, with the tile kernels'
// bounded wait (limit limit_ns); *timed_out (device) = 1 when it gave up.
cudaError_t launch_wait_selftest(uint64_t limit_ns, int *timed_out, cudaStream_t st);
cudaError_t prepare_gather_launch();
cudaError_t launch_csr_to_bits(const uint32_t *off, const uint32_t *col, size_t rows, uint32_t W, uint64_t *bits,
                               cudaStream_t st);
cudaError_t launch_ctl_reset(QCtl *const *ctls, uint32_t nq, uint32_t max_iter, uint32_t max_rounds,
                             uint32_t max_passes, uint32_t n_levels, unsigned long long cyclic_mask,
                             unsigned long long *box_edges, uint32_t n_boxes, uint32_t n,
                             const uint32_t *box_new_it, unsigned long long nt_read_mask, cudaStream_t st);
cudaError_t launch_eps_init(const void *eds, uint32_t ned, uint32_t grid, cudaStream_t st);
// Resume: OR seed (n_boxes x n rows of W words) into M2, A2 := M2 on the
// rows it touches, those rows new in iteration 1.
cudaError_t launch_seed_apply(const uint64_t *seed, uint64_t *m2, uint64_t *a2, uint32_t *a2_it, uint32_t *box_new_it,
                              QCtl *ctl, unsigned long long *box_edges, uint32_t n, uint32_t W, uint32_t n_boxes,
                              cudaStream_t st);
size_t eps_desc_size();
void fill_eps_desc(void *dst, uint64_t *m2, uint64_t *a2, uint32_t *a2_it, uint32_t *box_new_it, QCtl *ctl,
                   unsigned long long *box_edges, uint32_t n, uint32_t W);
cudaError_t scan_exclusive(const uint32_t *in, uint32_t *out, size_t n, uint32_t *tmp, cudaStream_t st);
cudaError_t launch_stage_count(const uint32_t *src, const uint32_t *lbl, const uint32_t *dst, size_t m, uint32_t n,
                               uint32_t n_term, const int32_t *label_map, uint32_t *cnt, int *err, cudaStream_t st);
cudaError_t launch_stage_fill(const uint32_t *src, const uint32_t *lbl, const uint32_t *dst, size_t m, uint32_t n,
                              uint32_t n_term, const int32_t *label_map, const uint32_t *off, uint32_t *fill,
                              uint32_t *col, cudaStream_t st);
cudaError_t launch_stage_unique(const uint32_t *off, uint32_t *col, uint32_t *ucnt, size_t rows, cudaStream_t st);
cudaError_t launch_stage_compact(const uint32_t *off, const uint32_t *col, const uint32_t *uoff, uint32_t *ucol,
                                 size_t rows, cudaStream_t st);
cudaError_t launch_popcount(const uint64_t *p, size_t nwords, unsigned long long *out, cudaStream_t st);
cudaError_t launch_nonempty_bits(const uint32_t *off, uint32_t n, uint32_t n_term, uint32_t W, uint64_t *bits,
                                 cudaStream_t st);
cudaError_t launch_copy_rows(const uint64_t *const *ptrs, const uint32_t *rows, uint32_t njobs, uint32_t W,
                             uint64_t *out, cudaStream_t st);

// ---- column sharding (cfpq_shard.cu) ----
cudaError_t launch_shard_setup(QCtl *ctl, uint32_t v0, uint32_t v1, cudaStream_t st);
cudaError_t launch_shard_export(const uint64_t *a2, const uint32_t *a2_it, uint32_t n, uint32_t W, uint32_t B,
                                uint32_t w0, uint32_t w1, uint32_t iter, uint64_t *out, cudaStream_t st);
cudaError_t launch_shard_apply(const uint64_t *full, uint64_t *m2, uint64_t *a2, uint32_t *a2_it, uint32_t n,
                               uint32_t W, uint32_t B, uint32_t iter, unsigned long long *cnt, QCtl *ctl,
                               uint32_t *box_new_it, cudaStream_t st);

// ---- single-CTA fixpoint (cfpq_small.cu) ----
struct SmallSrc;
size_t small_smem_bytes(uint32_t n, uint32_t W, uint32_t B, uint32_t nblk);
size_t small_desc_size();
size_t small_src_size();
size_t small_smem_limit();
cudaError_t launch_small_fixpoint(const void *descs, uint32_t count, size_t smem, cudaStream_t st);
void build_small_desc(void *desc_out, uint32_t n, uint32_t W, uint32_t B, uint32_t nblk, uint32_t n_levels,
                      unsigned long long cyclic_mask, uint32_t max_iter, uint32_t max_passes,
                      const uint32_t *dev_arrays, const SmallSrc *dev_srcs, size_t off_level, size_t off_src0,
                      size_t off_nsrc, size_t off_f0, size_t off_nf, size_t off_fb, size_t off_null,
                      const uint32_t *csr_off, const uint32_t *csr_col, uint64_t *blk_out, uint64_t *m2_out,
                      QCtl *ctl);
void fill_small_src(void *dst, uint32_t kind, uint32_t label, uint32_t ident, uint32_t same_level, int32_t rblk);

// ---- device memory ----
struct Allocator {
    cfpq_alloc_fn alloc = nullptr;
    cfpq_free_fn free = nullptr;
    void *user = nullptr;
    cudaStream_t stream = nullptr;
    size_t budget = 0;
    size_t in_use = 0;
    void *get(size_t bytes, std::string *err);
    void put(void *p, size_t bytes);
};

// A bump allocator over large chunks taken from a parent allocator, for the
// many buffers of a batch of queries (one parent call per chunk instead of
// one per buffer; the parent may be a caller's callback, e.g. into
// PyTorch).  Buffers handed out are never freed one by one: reset() rewinds
// to the start and keeps the chunks for the next batch, release() returns
// them to the parent.  `A` is an Allocator that draws from it.
struct SlabArena {
    Allocator *parent = nullptr;
    std::vector<std::pair<void *, size_t>> chunks;
    size_t chunk = 0, used = 0;  // current chunk and bytes used in it
    size_t chunk_bytes = (size_t)1 << 30;
    Allocator A;
    void *take(size_t bytes);
    void reset() { chunk = 0; used = 0; A.in_use = 0; }
    void release();
    ~SlabArena() { release(); }
};
void bind_slab(SlabArena *s, Allocator *parent, cudaStream_t st);

// An owned device buffer.
struct DBuf {
    Allocator *A = nullptr;
    void *p = nullptr;
    size_t bytes = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { reset(); }
    void reset() {
        if (p && A) A->put(p, bytes);
        p = nullptr;
        bytes = 0;
    }
    // (Re)allocate to at least `want` bytes; returns false on failure.
    bool ensure(Allocator *a, size_t want, std::string *err) {
        if (p && bytes >= want) return true;
        reset();
        A = a;
        if (want == 0) want = 256;
        p = a->get(want, err);
        if (!p) return false;
        bytes = want;
        return true;
    }
    template <class T>
    T *as() const { return static_cast<T *>(p); }
};

// Host copy of an RSM (validated).
struct HostRSM {
    uint32_t Q = 0, B = 0, start_box = 0;
    std::vector<uint32_t> box_start, state_box;
    std::vector<uint8_t> final_;
    struct Tr { uint32_t from, kind, sym, to; };
    std::vector<Tr> tr;  // deduplicated, sorted
    uint32_t max_terminal_plus1 = 0;
};
int copy_rsm(const cfpq_rsm *r, HostRSM *out, std::string *err);

// A staged graph on the device: per terminal label, deduplicated CSR rows.
struct GraphDev {
    uint32_t n = 0, n_pad = 0, W = 0, n_term = 0;
    size_t m_in = 0, m_unique = 0;
    DBuf csr_off;  // [n_term * n + 1]
    DBuf csr_col;  // [m_unique]
    // Row bitmaps derived from the CSR, rebuilt when `content` moves on:
    DBuf term_bits;  // [n_term * n * W] bit rows of the terminal labels (tensor-core sources only)
    uint64_t term_bits_content = ~0ull;
    int ensure_term_bits(Allocator *A, cudaStream_t st, std::string *err);
    DBuf nonempty;  // [n_term * W] bit y of label l: row (l, y) of the CSR has an edge (pure-terminal reads)
    uint64_t nonempty_content = ~0ull;
    int ensure_nonempty(Allocator *A, cudaStream_t st, std::string *err);
    // staging scratch
    DBuf e_src, e_lbl, e_dst, cnt, off, col, ucnt, scan_tmp, label_map, err;
    std::vector<uint32_t> h_off;  // host copies on demand (paths)
    std::vector<uint32_t> h_col;
    bool host_valid = false;
    // `generation` moves on when the shape of the staged graph changes (n,
    // n_terminals, reallocated buffers): plans and work lists hold its
    // pointers and sizes.  `content` moves on with every successful load,
    // also a same-size one: everything derived from the edges is stale then.
    uint64_t generation = 0;
    uint64_t content = 0;
};

// Device state and descriptors of one query (graph + RSM).
struct QueryDev {
    GraphDev *g = nullptr;
    HostRSM rsm;
    uint32_t n = 0, W = 0, Q = 0, B = 0, vpl = 0, lpr = 0;
    std::vector<int32_t> blk_of;  // Q*Q -> block or -1
    std::vector<std::pair<uint32_t, uint32_t>> blocks;
    DBuf blk_mem, stamp_mem, last_mem, m2_mem, a2_mem, a2it_mem, boxit_mem, ctl_mem, eps_mem, ctl_ptr_mem, boxedge_mem;
    uint32_t n_eps = 0;
    uint64_t device_bytes = 0;
    // host descriptors (pointers filled once buffers exist; ctl set by the executor)
    uint32_t closure_mode = CFPQ_CLOSURE_AUTO;
    uint32_t tile_kind = kTileFp8Pair;  // product kernel of the tiles (TileKind)
    bool tile_fp4 = false;              // tile operands are E2M1 nibbles (tile_kind_fp4(tile_kind))
    uint32_t tile_ratio = (uint32_t)kTileEdgeRatio;  // new_tiles_pay's ratio for this tile kind
    uint32_t gather_slices = 0;  // cfpq_options::gather_slices
    // Multiple-source runs: per state the rows reachable from the sources
    // (compute_reach); the work items of block (s, t) then skip the rows of
    // state s outside them.
    bool restricted = false;
    DBuf reach_mem, reach_f, reach_misc;
    // Resume: a given M2 (B x n rows of W words) applied after the epsilon
    // rows by every enqueue_init while `seeded`.
    bool seeded = false;
    DBuf seed_mem;
    uint64_t *reach_ptr(uint32_t s) const { return reach_mem.as<uint64_t>() + (size_t)s * W; }
    int compute_reach(Allocator *A, cudaStream_t st, const uint32_t *h_src, uint32_t ns, std::string *err);
    struct Src {
        uint32_t label_kind, label, ident;
        int32_t rblk;
        uint32_t same_level, dense, box_switch;
        int32_t tc_slot;  // compaction buffers of the source's product job, or -1
        int32_t tc_slot_new;  // ... of its channel-1 job (new edges; nonterminal, not same level), or -1
        uint32_t pure_rb; // the block read is pure-terminal: expand CSR rows
    };
    std::vector<uint32_t> blk_pure_n, blk_pure_lbl;  // per block: labels of a pure-terminal block (<= 2)
    // Product jobs' compaction buffers, one slot per tile job: the dirty
    // row list (n_pad entries), its pass-stamped count, the row list of a
    // channel-1 job (n_pad entries), A's columns at the listed rows as FP8
    // bytes (n rows of kcap; E2M1 nibbles: kcap/2) and the listed B rows
    // transposed (n_pad rows of the same).  Every part starts 128-byte
    // aligned.
    DBuf tc_mem;
    uint32_t n_tc_src = 0, kcap = 0;
    bool full_kcap = false;  // tile jobs' inner dimension may hold every row (else half above n = 8192)
    uint64_t tc_slot_bytes() const;
    uint32_t tc_kstride() const { return tile_fp4 ? kcap / 2u : kcap; }  // bytes per operand row
    unsigned char *tc_slot(uint32_t k) const { return tc_mem.as<unsigned char>() + (size_t)k * tc_slot_bytes(); }
    uint32_t *tc_ys(uint32_t k) const { return reinterpret_cast<uint32_t *>(tc_slot(k)); }
    unsigned long long *tc_kcount(uint32_t k) const {
        return reinterpret_cast<unsigned long long *>(tc_slot(k) + (size_t)W * 64 * 4);
    }
    uint32_t *tc_xs(uint32_t k) const { return reinterpret_cast<uint32_t *>(tc_slot(k) + (size_t)W * 64 * 4 + 256); }
    uint8_t *tc_a8(uint32_t k) const { return tc_slot(k) + (size_t)W * 64 * 8 + 256; }
    uint8_t *tc_b8(uint32_t k) const { return tc_a8(k) + (size_t)n * tc_kstride(); }
    std::vector<uint32_t> blk_src0, blk_nsrc;  // per block
    std::vector<uint32_t> blk_level;           // per block, 0..n_levels-1
    uint32_t n_levels = 1;
    uint64_t cyclic_mask = 0;
    unsigned long long nt_read_mask = 0;  // boxes read by some transition (bit 63: some box >= 63)
    std::vector<Src> srcs;
    std::vector<uint32_t> box_f0, box_nf;
    std::vector<uint32_t> fblocks;  // per box list of block ids (q0, f)
    bool prepared = false;
    uint64_t graph_generation = 0;
    int plan(std::string *err);                    // blocks, sources, extraction lists (host only)
    uint64_t footprint() const;                    // device bytes prepare() will hold
    int prepare(Allocator *A, std::string *err);  // plan + buffers
    // The row bitmaps this query's sources read (pure-terminal masks, terminal
    // bit rows), rebuilt for the graph's current content; *moved is set when a
    // buffer was reallocated (the work lists hold its address).
    int refresh_graph_caches(Allocator *A, cudaStream_t st, std::string *err, bool *moved);
    // Reset this query's device state and loop control (start of its fixpoint).
    int enqueue_init(cudaStream_t st, uint32_t max_iter, uint32_t max_rounds, uint32_t max_passes);
    // single-CTA path: eligible when rows are <= 512 bits and the state fits one SM
    DBuf small_arrays, small_desc;
    size_t small_smem = 0;
    bool small_ok = false;
    int prepare_small(Allocator *A, cudaStream_t st, uint32_t max_iter, uint32_t max_passes, std::string *err);
    QCtl *ctl() const { return ctl_mem.as<QCtl>(); }
    uint64_t *blk_ptr(uint32_t b) const { return blk_mem.as<uint64_t>() + (size_t)b * n * W; }
    uint32_t *stamp_ptr(uint32_t b) const { return stamp_mem.as<uint32_t>() + (size_t)b * n; }
    uint64_t *m2_ptr(uint32_t b) const { return m2_mem.as<uint64_t>() + (size_t)b * n * W; }
    uint64_t *a2_ptr(uint32_t b) const { return a2_mem.as<uint64_t>() + (size_t)b * n * W; }
};

// Closure modes that put every dirty-row product of a closure block on tiles.
inline bool closure_all_tiles(uint32_t mode) {
    return mode == CFPQ_CLOSURE_TC_FP8 || mode == CFPQ_CLOSURE_TC_FP4;
}

// ---- autotuner (cfpq_tune.cu) ----
// Measured on a probe query per device: the rate of each tile kind and of
// the row gather, the kind AUTO uses by default, and the cost-model ratio
// for that kind (the channel-1 tiles run while M * K < ratio * new edges).
struct Tuning {
    bool tuned = false;
    uint32_t kind = kTileFp4Pair;
    double gather_gbs = 0, tflops[kTileKinds] = {0, 0, 0, 0}, probe_ms = 0;
    double read_l2_gbs = 0, read_hbm_gbs = 0;  // device reads of an L2-sized / HBM-sized buffer
    uint64_t l2_bytes = 0;
    uint32_t ratio_l2 = 0;  // the searched cost-model ratio of `kind` (L2-resident queries)
    int status = 0;  // CFPQ status of the probe (0 = ok)
    // the gather's rate for closure blocks of `block_bytes`: measured on
    // L2-resident blocks, scaled by the read bandwidths beyond half the L2
    double gather_rate(uint64_t block_bytes) const { return gather_gbs * memory_scale(block_bytes); }
    double memory_scale(uint64_t block_bytes) const {
        if (block_bytes * 2 <= l2_bytes || read_l2_gbs <= 0 || read_hbm_gbs <= 0) return 1.0;
        return std::min(1.0, read_hbm_gbs / read_l2_gbs);
    }
};
// The device's tuning; runs the probe first when `run` and it has not run
// (or when `force`).  `like` gives the allocator and stream of the probe.
Tuning device_tuning(const cfpq_options &like, cudaStream_t st, bool run, bool force);
// Set q's tile kernel, operand format and ratio for a run with options o on
// a graph of n vertices (cfpq_api.cu).
void set_tiles(QueryDev &q, const cfpq_options &o, cudaStream_t st, uint32_t n);
// The tile kind of a query in closure mode `mode` with tile_format `fmt`
// (CFPQ_TILES_DEFAULT: the tuned kind).
uint32_t tile_kind_of(uint32_t mode, uint32_t fmt, const Tuning &t);
// new_tiles_pay's ratio for a kind and a query of n vertices: from the
// measured rates when tuned, else the built-in constant of its format.
uint32_t tile_ratio_of(uint32_t kind, const Tuning &t, uint32_t n);

// Closure passes per iteration of the CUDA graph's while node.
constexpr uint32_t kLoopUnroll = 2;

// Runs the fixpoint of a set of queries with shared launches.
struct Executor {
    std::vector<QueryDev *> qs;
    DBuf ctl_ptrs, mirror, items[kClasses], xitems[kClasses], srcs, fds, running;
    DBuf tcjobs, tcmaps, tables, tc_err, done_counter;
    DBuf newcols;              // new-edge column bitmaps of the jobs covering new edges (zeroed every pass)
    size_t newcols_words = 0;
    ExecTables T;
    uint32_t n_items[kClasses] = {0}, n_xitems[kClasses] = {0};
    uint32_t max_live[kClasses] = {0};  // bound on live items of a pass: sum over queries of the largest level
    uint32_t n_tcjobs = 0, max_tc_tiles = 0, max_tc_w = 0;
    uint32_t tile_kind = kTileFp8Pair;  // the tile jobs' kernel (every query of an executor shares it)
    uint32_t item_scale = 1;            // work items span item_scale times the usual rows (a power of 2)
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream: capture is not allowed on the legacy default stream
    bool built = false;
    ~Executor() {
        drop_graph();
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    int assemble(Allocator *A, cudaStream_t st, std::string *err);
    int enqueue_prologue(cudaStream_t st, uint32_t max_iter, uint32_t max_rounds, uint32_t max_passes);
    int enqueue_lists(cudaStream_t st);  // recompute the live lists without advancing any query
    // ev (profiling, may be null): four events recorded before the tile
    // operands, after them (before the row gathers), after the gathers and
    // after the tile products.
    int enqueue_pass(cudaStream_t st, cudaGraphConditionalHandle h, int use_handle, int *running_out,
                     const cudaEvent_t *ev = nullptr);
    int build_graph(cudaStream_t st, uint32_t max_iter, uint32_t max_rounds, uint32_t max_passes, std::string *err);
    int read_ctls(cudaStream_t st, std::vector<QCtl> *out, int *tc_error = nullptr);
};

// Backward layers of path extraction (Sec. 3.2): for a target (box N,
// vertex y), layer k holds the product vertices (s, x) from which some (f, y),
// f final in N, is reached in M3 over at most k graph edges (a nonterminal
// edge counts one edge unless it stays on its vertex).  prepare() uploads the
// reverse terminal CSR and the RSM transitions grouped by target state, and
// transposes M2 of every box a nonterminal transition reads; layers() runs
// the search for a list of targets and copies, per target, layers 0..L to
// the host ((L + 1) * Q * W words: layer-major, then state, then the
// vertex's word).
struct PathsDev {
    uint32_t n = 0, W = 0, Q = 0, B = 0, n_nt = 0;
    const uint64_t *m2 = nullptr;
    std::vector<uint32_t> host_tab;
    DBuf tables, rev_off, rev_col, mt, lay, delta, flag;
    int prepare(Allocator *A, cudaStream_t st, const QueryDev &q, uint32_t n_term, const std::vector<uint32_t> &h_roff,
                const std::vector<uint32_t> &h_rcol, std::string *err);
    // Layers of several targets (box, vertex), searched side by side in
    // batches of at most 1 GiB; out[i] gets target i's layers.
    int layers(Allocator *A, cudaStream_t st, const HostRSM &rsm,
               const std::vector<std::pair<uint32_t, uint32_t>> &targets, uint32_t L,
               std::vector<std::vector<uint64_t>> *out, std::string *err);
    int layers_batch(Allocator *A, cudaStream_t st, const HostRSM &rsm, const std::pair<uint32_t, uint32_t> *targets,
                     uint32_t T, uint32_t L, std::vector<uint64_t> *out, std::string *err);
};

int stage_graph(GraphDev *g, Allocator *A, cudaStream_t st, uint32_t n, uint32_t n_term, size_t m, const uint32_t *src,
                const uint32_t *lbl, const uint32_t *dst, bool device_ptrs, std::string *err);

}  // namespace cfpq
