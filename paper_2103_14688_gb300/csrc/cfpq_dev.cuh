// cfpq_dev.cuh -- device data structures of libcfpq (shared by host and kernels).
//
// Layout of one query on the device (Sec. 3.1, Listing 1; Kronecker index
// state * n + vertex of Sec. 2.4):
//   - the closure C3 is held as n x n state blocks C[s,t], one per pair of RSM
//     states with t reachable from s by one or more RSM transitions (all other
//     blocks of C3 are zero because M3's block (s,t) is OR_{l: s-l->t} M2^l);
//     a block is n rows of W = n_pad/64 uint64 words, bit y of row x is
//     word y/64, bit y%64; n_pad is n rounded up to 128 so that rows are
//     16-byte aligned for 128-bit loads;
//   - every block has a uint32 stamp per row (the closure pass that last
//     changed the row) and one "last changed pass" word: the dirty flags;
//   - terminal labels are CSR adjacency lists (static, deduplicated);
//   - nonterminal labels are bit rows M2^b (all edges) and A2^b (edges new in
//     this iteration, valid where the row's stamp equals the iteration).
#pragma once
#include <stdint.h>

namespace cfpq {

// Passes are scheduled by level: the RSM's states are grouped into strongly
// connected components, a component's level is one more than the highest
// level among the components it has transitions into, and block C[s,t]
// takes the level of s.  C[s,t] depends only on blocks C[u,t] of successors
// u of s, so on lower levels or (inside a cyclic component) its own level.
// Every iteration processes the levels in increasing order; a level gets one
// FIRST pass, and a level whose component has a cycle repeats (REPEAT) until
// a pass changes no row.
constexpr uint32_t kModeNew = 0;   // FIRST pass of a level
constexpr uint32_t kModeProp = 1;  // REPEAT pass of a cyclic level
constexpr uint32_t kPhaseRun = 0;
constexpr uint32_t kPhaseDone = 1;
constexpr uint32_t kPhasePause = 2;  // column sharding: iteration done, new edges not yet exchanged
constexpr uint32_t kStatusOk = 0;
constexpr uint32_t kStatusIterCap = 1;
constexpr uint32_t kStatusRoundCap = 2;
constexpr uint32_t kStatusPassCap = 3;

// Per-query loop state, in device memory.  Written only by the control
// kernel (and the counters by atomics), read by every kernel of a pass.
struct QCtl {
    uint32_t g;               // id of the closure pass in progress (starts at 2)
    uint32_t iter;            // fixpoint iteration, 1-based
    uint32_t mode;            // kModeNew / kModeProp
    uint32_t phase;           // kPhaseRun / kPhaseDone
    uint32_t g_iter_start;    // pass id of the iteration's first pass
    uint32_t rounds_in_iter;  // passes done in this iteration
    uint32_t status;          // kStatus*
    uint32_t max_iter;        // 0 = no cap
    uint32_t max_rounds;      // 0 = no cap
    uint32_t max_passes;      // hard cap on passes (safety)
    uint32_t iters_done;      // completed iterations
    uint32_t passes;          // passes done
    uint32_t level;           // level being processed
    uint32_t n_levels;        // levels of this query (>= 1)
    unsigned long long cyclic_mask;   // bit L: level L has a cycle (REPEAT passes)
    // Density switch of nonterminal sources (closure mode AUTO): bit b set when
    // box b's matrix M2^b holds at least n^2 / kDenseDiv edges; decided at the
    // end of every iteration, so a pass never mixes the two forms of a source.
    unsigned long long *box_edges;    // per box: edges of M2^b (null: no switch)
    // Boxes some transition of the query reads (bit b; all bits when a box >=
    // 63 is read) and the per-box iteration mark written by extraction: an
    // iteration whose new edges all lie in boxes nobody reads is the last one
    // that changes anything, so the next (which adds nothing) is counted
    // without running its passes.
    const uint32_t *box_new_it;
    unsigned long long nt_read_mask;
    uint32_t dense_mask;
    uint32_t n_boxes;
    uint32_t n;
    uint32_t pad2;
    unsigned long long changed_rows;  // rows changed by the pass in progress
    unsigned long long new_edges;     // edges added by the extraction in progress
    unsigned long long edges_total;   // edges added so far (epsilon edges included)
    unsigned long long row_ors;       // source rows ORed (all passes)
    unsigned long long tile_mmas;     // dense tiles multiplied (all passes)
    unsigned long long tile_kstages;  // K stages of those tiles run on the tensor cores (128 x 256 x 128 MACs each)
    unsigned long long rounds_total;
    unsigned long long rows_changed_total;  // summed over passes
    // Column sharding (one query over several ranks): the closure is
    // computed on the 128-bit column vectors [col_v0, col_v1) of every block
    // only (all columns: 0, ~0), and with `shard` set the loop pauses after
    // every iteration (kPhasePause) until the new edges of all ranks are
    // installed; shard_new = this rank's new edges of that iteration.
    uint32_t shard;
    uint32_t col_v0, col_v1;
    uint32_t pad4;
    unsigned long long shard_new;
    unsigned long long tile_operand_bytes;  // 0/1 operand bytes the tile jobs expanded (all passes)
};

// One source of an output block C[s,t]: a transition s -l-> u with t = u or
// t reachable from u.  Product edges (s,x) -> (u,y) for every edge (x,y) of
// the graph matrix M2^l (the Kronecker product M1^l (x) M2^l, row by row).
struct SrcDesc {
    const uint32_t *csr_off;   // terminal l: CSR offsets [n+1]; else null
    const uint32_t *csr_col;   // terminal l: CSR columns
    const uint64_t *nt_all;    // nonterminal l = box b: M2^b rows
    const uint64_t *nt_new;    // nonterminal: A2^b rows
    const uint32_t *nt_new_it; // nonterminal: A2 row valid iff == iteration
    const uint32_t *box_new_it;// nonterminal: box has new edges iff == iteration
    const uint64_t *rblk;      // C[u,t] rows or null (u == t without a cycle)
    const uint32_t *rstamp;    // row stamps of C[u,t]
    const uint32_t *rlast;     // last pass that changed C[u,t]
    uint32_t ident;            // u == t: the product edge itself lands in C[s,t]
    uint32_t same_level;       // C[u,t] is on the level of C[s,t] (same cyclic component)
    uint32_t dense;            // label matrix handled by dense tiles (not here)
    uint32_t box_switch;       // nonterminal source that moves to dense tiles when its box is dense
    uint32_t label_box;        // box of a nonterminal source
    // C[u,t] is the union of at most two terminal adjacencies (every source of
    // block (u,t) is a direct terminal transition u -l-> t): its row y is read
    // as those labels' CSR rows of y instead of n bits.  rblk/rstamp/rlast
    // still give the dirty state of the block.
    uint32_t pure_n;
    const uint32_t *pure_off[2];
    const uint32_t *pure_col;
    const uint64_t *pure_mask[2];  // per label: bit y set iff y has an edge of it (W words)
    // Tile source with a product job for the iteration's new edges
    // (TcJob::covers_new): while its tiles are on and that job runs in this
    // pass (new_tiles_pay on its counts: tc_kcount, tagged with the pass, at
    // most tc_kcap rows; tc_mcount; tc_ecount), the row gather leaves the new
    // edges' row ORs to the tiles and keeps only the product edges
    // themselves (ident).
    uint32_t tile_new;
    uint32_t tc_kcap;
    uint32_t tc_ratio;         // new_tiles_pay's ratio for the job's tile format
    const unsigned long long *tc_kcount;
    const unsigned long long *tc_mcount;
    const unsigned long long *tc_ecount;
};

// Gather work item: rows [row0, row1) of one output block.
struct GItem {
    uint64_t *out;
    uint32_t *out_stamp;
    uint32_t *out_last;
    QCtl *ctl;
    const uint64_t *rmask;  // multiple-source runs: rows to compute (bit per row), else null
    uint32_t src0, nsrc;
    uint32_t row0, row1;
    uint32_t W;    // words per row
    uint32_t lpr;  // lanes per row (power of two <= 32)
    uint32_t level;
    // Column slice of the nonterminal adjacency rows this item enumerates,
    // in 128-bit vectors: [slice & 0xFFFF, slice >> 16).  Items of one row
    // range with different slices share the output rows and merge them with
    // atomicOr; the CSR sources are taken by the slice that starts at 0.
    // Slices take part only while a box in nt_boxes (the boxes whose dense
    // adjacency the block's gather enumerates into closure-row ORs: sources
    // reading a closure block that is not pure-terminal, without a tile job)
    // is dense (QCtl::dense_mask); otherwise the first slice covers every
    // column and the others do nothing.
    uint32_t slice;
    uint32_t nt_boxes;
    uint32_t pad;
};

// Final-state block used by extraction: C[q0(b), f] with f final in box b.
struct FDesc {
    const uint64_t *blk;
    const uint32_t *stamp;
};

// Extraction work item: rows [row0, row1) of box b's M2^b.
struct XItem {
    uint64_t *m2;
    uint64_t *a2;
    uint32_t *a2_it;
    uint32_t *box_new_it;
    unsigned long long *box_edges;  // edge counter of the box (density switch)
    QCtl *ctl;
    uint32_t f0, nf;
    uint32_t row0, row1;
    uint32_t W;
    uint32_t lpr;
};

// One dense product job: out |= A * B over the square n x n state block,
// with A rows optionally valid only in one iteration (A2 semantics) and B
// rows taking part only when their stamp is >= thr.
struct TcJob {
    uint64_t *out;
    uint32_t *out_stamp;
    uint32_t *out_last;
    const uint64_t *A;
    const uint32_t *a_it;      // if set: A row x is used only when a_it[x] == iter
    const uint64_t *B;
    const uint32_t *b_stamp;   // stamps of B rows (null: all rows)
    QCtl *ctl;                 // null: standalone product (iter = 0, thr = 0, g = 0)
    uint32_t n, W;
    uint32_t ident;            // also OR the A rows themselves into out (product edge u == t)
    uint32_t chan;             // 1, 2 or 4 (see src_channels); 0 = always, thr 0
    uint32_t level, same_level;
    const uint32_t *box_new_it;
    const uint32_t *rlast;
    uint32_t tiles_m, tiles_n;  // tiles of this job
    uint32_t tile0;             // first global tile index of this job
    uint32_t box;               // nonterminal label (switchable jobs)
    uint32_t switchable;        // active only while the box is dense (closure mode AUTO)
    uint32_t kcap;              // most compacted rows (a multiple of 128)
    // Dirty-row compaction (channels 2 and 4): before the products of a pass,
    // the B rows with stamp >= thr are listed in `ys`; A's columns at those
    // rows and the listed B rows are expanded to 0/1 FP8 bytes, A as
    // a8[x][k] (n rows of kcap bytes), B transposed as b8[z][k] (n_pad rows
    // of kcap bytes), and the product runs its inner dimension over the
    // listed rows only, operands brought in by TMA.  kcount = (pass stamp <<
    // 32) | count.  A job whose list is longer than kcap runs uncompacted.
    // With fp4 set the operands are 0/1 E2M1 nibbles instead, two per byte
    // (element k in byte k/2, even k in the low nibble), for the block-scaled
    // FP4 products; kstride = bytes per operand row (kcap, or kcap/2 for fp4).
    uint32_t *ys;
    unsigned long long *kcount;
    uint8_t *a8;
    uint8_t *b8;
    uint32_t map;               // index of the job's pair of tensor maps (a8, b8)
    uint32_t kstride;
    uint32_t fp4;
    uint32_t tile_ratio;        // new_tiles_pay's ratio (channel-1 jobs)
    // Channel-1 job (covers_new): the iteration's new edges A2 (A = A2 rows,
    // a_it = their iteration marks) times whole rows of B, compacted on both
    // sides: M to the rows x with a new edge (xs, count *mcount), K to the
    // columns y of some new edge (newcols, a bitmap of W words, then ys).
    // *ecount = the number of new edges.  mcount, ecount and newcols are
    // zeroed before every pass.  The job runs only when new_tiles_pay says
    // the tiles beat the row gather on those counts; the gather then skips
    // the channel's row ORs.
    uint32_t covers_new;
    uint64_t *newcols;
    uint32_t *xs;
    unsigned long long *mcount;
    unsigned long long *ecount;
};

// Does the channel-1 tile job beat the row gather?  The gather reads one
// closure row (n/8 bytes) per new edge (e of them); the compacted product
// issues 2 * M * K * n multiply-adds (M and K rounded up to whole 128-row
// tiles).  With the gather's measured ~3.5 TB/s and the FP8 tiles' ~2.5
// PFLOP/s, the tiles win when M * K < e * 2.5e15 / (16 * 3.5e12), i.e.
// about 44 * e; n cancels.  The ratio scales with the tile format's rate
// (kTileEdgeRatio for FP8, kTileEdgeRatioFp4 for FP4).  listed_k = K for
// this pass (0 if the list was not built), kcap = the job's room for it.
constexpr unsigned long long kTileEdgeRatio = 44;
constexpr unsigned long long kTileEdgeRatioFp4 = 88;

// Tile products (TMA-fed tcgen05 kernels): 0/1 FP8 operands in 256 x 256
// output tiles (two 128-row accumulators per CTA) or in 128 x 256 tiles
// (double-buffered accumulator), or 0/1 E2M1 operands in 256 x 192 tiles
// (kind::mxf4 with 32-element UE8M0 scales, or kind::mxf4nvf4 with
// 16-element UE4M3 scales; the operands are the same).
constexpr uint32_t kTileFp8Pair = 0, kTileFp8Single = 1, kTileFp4Pair = 2, kTileFp4NvPair = 3, kTileKinds = 4;
__host__ __device__ constexpr bool tile_kind_fp4(uint32_t k) { return k == kTileFp4Pair || k == kTileFp4NvPair; }
__host__ __device__ inline bool new_tiles_pay(uint32_t listed_k, uint32_t kcap, unsigned long long m,
                                              unsigned long long e, unsigned long long ratio) {
    if (listed_k == 0 || listed_k > kcap || m == 0) return false;
    const unsigned long long pm = (m + 127ull) & ~127ull, pk = ((unsigned long long)listed_k + 127ull) & ~127ull;
    return pm * pk < ratio * e;
}

constexpr uint32_t kDenseDiv = 32;  // a box is dense from n^2 / 32 edges on (one bit in two words)
constexpr uint32_t kAutoTilesMinN = 2048;  // AUTO switches boxes to tile products only from this n on

// Per-executor work tables.  Items of each kind are sorted by (query, level);
// the static tables give, for query q and level L, the first item of that
// level (entry L = n_levels gives the end).  Before every pass the control
// kernel writes, for each running query, the range of items of its current
// level and an exclusive prefix over queries, so that persistent kernels walk
// only the live items.
constexpr int kVplClasses = 5;
// Item classes: row width class (VPL 1, 2, 4, 8, 16) x kernel variant: the
// general variant (nt = 1) serves blocks with sources over nonterminal
// (bit-row) adjacency or reading pure-terminal blocks; class = 2 * vpl_index + nt.
constexpr int kClasses = 2 * kVplClasses;
struct ExecTables {
    uint32_t nq;
    uint32_t maxL1;                          // max levels over queries + 1
    const uint32_t *g_lvl[kClasses];         // [nq * maxL1] gather items per (q, level)
    const uint32_t *x_rng[kClasses];         // [nq + 1] extraction items per query
    const uint32_t *t_lvl;                   // [nq * maxL1] TC jobs per (q, level)
    const uint32_t *t_lvl_tiles;             // [nq * maxL1] TC tiles of the jobs at (q, level)
    // written by the control kernel for the next pass
    uint32_t *g_total;                       // [kClasses]
    uint32_t *g_next;                        // [kClasses] dynamic gather units taken in the pass
    uint32_t *g_pre[kClasses];               // [nq] exclusive prefix of live items
    uint32_t *g_beg[kClasses];               // [nq] first live item
    uint32_t *x_total;                       // [kClasses]
    uint32_t *x_pre[kClasses];
    uint32_t *x_beg[kClasses];
    uint32_t *t_total;                       // [1] live TC tiles
    uint32_t *t_pre;                         // [nq] prefix of live tiles
    uint32_t *t_job_beg;                     // [nq]
    uint32_t *t_job_end;                     // [nq]
    // The tile jobs that take part in the next pass (tc_job_active), listed
    // by the control kernel in any order: the operand kernels walk only these.
    const TcJob *jobs;                       // the executor's jobs (null: none)
    uint32_t *aj;                            // [number of jobs]
    uint32_t *aj_n;                          // [1]
};

// Decide whether the job takes part in this pass and with which threshold.
__device__ inline bool tc_job_active(const TcJob &j, uint32_t *thr, uint32_t *iter, uint32_t *g) {
    if (!j.ctl) {
        *thr = 0;
        *iter = 0;
        *g = 0;
        return true;
    }
    const QCtl *c = j.ctl;
    if (c->phase != kPhaseRun || c->level != j.level) return false;
    if (j.switchable && (j.box >= 32u || !((c->dense_mask >> j.box) & 1u))) return false;
    *iter = c->iter;
    *g = c->g;
    const uint32_t g0 = c->g_iter_start;
    if (j.chan == 1u) {
        if (c->mode != kModeNew) return false;
        if (j.box_new_it && *j.box_new_it != c->iter) return false;
        if (!j.box_new_it && c->iter != 1) return false;
        *thr = 0;
        return true;
    }
    if (j.chan == 2u) {
        if (c->mode != kModeNew || j.same_level || !j.rlast || *j.rlast < g0) return false;
        if (!j.box_new_it && c->iter == 1) return false;  // terminals: iteration 1 is covered by channel 1
        *thr = g0;
        return true;
    }
    if (j.chan == 4u) {
        if (c->mode != kModeProp || !j.same_level || !j.rlast || *j.rlast + 1u < c->g) return false;
        *thr = c->g - 1u;
        return true;
    }
    return false;
}


// Find q with pre[q] <= i < pre[q+1] (pre exclusive, non-decreasing).
__host__ __device__ inline uint32_t find_owner(const uint32_t *pre, uint32_t nq, uint32_t i) {
    uint32_t lo = 0, hi = nq;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

}  // namespace cfpq
