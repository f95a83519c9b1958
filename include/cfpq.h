/*
 * cfpq.h -- C ABI of libcfpq: Kronecker-product context-free and regular path
 * querying on one GB300 GPU (sm_103a).
 *
 * Method: Shemetova, Azimov, Orachev, Epelbaum, Grigorev, "One Algorithm to
 * Evaluate Them All: Unified Linear Algebra Based Approach to Evaluate Both
 * Regular and Context-Free Path Queries" (arXiv 2103.14688).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns an int status: CFPQ_OK (0) or a negative CFPQ_ERR_*
 *    code; cfpq_status_string() names it and cfpq_last_error() gives the
 *    context's last message.  No C++ exception crosses this boundary.
 *  - The caller owns every buffer it passes.  Inputs are copied before the
 *    call returns (host pointers) or read on the context's stream (device
 *    pointers, *_device calls).  Output buffers follow a two-call protocol:
 *    passing NULL (or a capacity too small) reports the required count and
 *    returns CFPQ_ERR_BUFFER_TOO_SMALL when the buffer was too small.
 *  - A context is used by one host thread at a time.  It owns its device
 *    memory, obtained through the optional allocator callbacks in
 *    cfpq_options (else cudaMallocAsync on the context's stream), and issues
 *    all its work on the stream given to cfpq_create (a cudaStream_t; NULL
 *    selects the legacy default stream).
 *  - Vertices are 0-based (Sec. 2.1, Def. of an edge-labelled graph:
 *    V = {0..|V|-1}).  Terminal labels are 0..n_terminals-1; nonterminals are
 *    the RSM's boxes 0..n_boxes-1, a namespace disjoint from the terminals
 *    (Sec. 2.3, Def. of an RSM: Sigma and B are disjoint).
 *  - Product-graph index (Sec. 2.4, Def. of the Kronecker product, and the
 *    getStates/getCoordinates helpers of Listing 1): a product vertex
 *    (state s, vertex x) has index s * n + x.
 */
#ifndef CFPQ_H
#define CFPQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define CFPQ_OK 0
#define CFPQ_ERR_INVALID_ARG (-1)      /* bad pointer, id out of range, malformed RSM */
#define CFPQ_ERR_OUT_OF_MEMORY (-2)    /* device or host allocation failed / budget exceeded */
#define CFPQ_ERR_BUFFER_TOO_SMALL (-3) /* output capacity too small; the count was reported */
#define CFPQ_ERR_TIMEOUT (-4)          /* iteration or round cap reached before the fixpoint */
#define CFPQ_ERR_NOT_READY (-5)        /* result asked for before it exists */
#define CFPQ_ERR_CUDA (-6)             /* a CUDA runtime call failed */
#define CFPQ_ERR_STATE (-7)            /* calls in the wrong order (e.g. run before load) */
#define CFPQ_ERR_UNSUPPORTED (-8)      /* size or mode the library does not handle */

typedef struct cfpq_ctx cfpq_ctx;

/* Device allocator callbacks.  alloc returns a device pointer of at least
 * `bytes` bytes usable on `stream` (aligned to 256 bytes) or NULL; free
 * releases it.  Both run on the calling host thread inside cfpq_* calls. */
typedef void *(*cfpq_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*cfpq_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

/* Closure kernels (Listing 1, incremental transitive closure). */
/* AUTO: bit-packed rows; from n = 2048 on, a nonterminal whose matrix M2
 * holds >= n^2/32 edges (checked after every iteration) moves its products
 * with the dirty closure rows to tensor-core tiles as in TC_FP8 / TC_FP4,
 * in the format cfpq_options::tile_format selects. */
#define CFPQ_CLOSURE_AUTO 0
#define CFPQ_CLOSURE_BITPACKED 1 /* bit-packed uint64 rows only */
/* TC_FP8: products of whole label matrices with the closure rows changed in
 * the previous pass run as 0/1 FP8-E4M3 tcgen05 tiles (FP32 accumulate,
 * count > 0), the inner dimension compacted to the changed rows; products of
 * the new edges of an iteration stay on bit-packed rows. */
#define CFPQ_CLOSURE_TC_FP8 2
#define CFPQ_CLOSURE_TC_I8 3     /* 0/1 INT8 tcgen05 products: CFPQ_ERR_UNSUPPORTED on sm_103a (no kind::i8) */
/* TC_FP4: as TC_FP8, with 0/1 E2M1 operands (two per byte) multiplied by the
 * block-scaled FP4 MMA (tcgen05 kind::mxf4, every scale factor 1.0, FP32
 * accumulate, count > 0); tiles of 256 x 192 output bits.  Exact for the
 * same reason: counts never exceed the inner dimension (< 2^24). */
#define CFPQ_CLOSURE_TC_FP4 4

/* Tile kernel of the tensor-core products (cfpq_options::tile_format): the
 * operand format and the output tile of one CTA.  DEFAULT is the
 * autotuner's choice for AUTO (see cfpq_tune), FP8 pairs for TC_FP8. */
#define CFPQ_TILES_DEFAULT 0
#define CFPQ_TILES_FP8 1     /* 0/1 FP8, 256 x 256 output bits per CTA (two 128-row accumulators) */
#define CFPQ_TILES_FP4 2     /* 0/1 E2M1, 256 x 192 output bits per CTA */
#define CFPQ_TILES_FP8_128 3 /* 0/1 FP8, 128 x 256 output bits per CTA (double-buffered accumulator) */
#define CFPQ_TILES_NVFP4 4   /* as FP4, multiplied by kind::mxf4nvf4 (16-element UE4M3 scales, all 1.0) */

/* Fixpoint loop control (Listing 1, "while M2 is changing"). */
#define CFPQ_LOOP_DEVICE 0 /* one CUDA-graph launch; device-side convergence flags */
#define CFPQ_LOOP_HOST 1   /* host reads the convergence flags after every pass */

typedef struct {
    uint32_t struct_size;    /* sizeof(cfpq_options); set by cfpq_default_options */
    int32_t device;          /* CUDA device ordinal */
    uint32_t max_iterations; /* fixpoint iteration cap; 0 = no cap (the loop always ends) */
    uint32_t max_rounds;     /* closure passes per iteration cap; 0 = no cap */
    uint32_t closure_mode;   /* CFPQ_CLOSURE_* */
    uint32_t loop_mode;      /* CFPQ_LOOP_* */
    uint32_t profile;        /* 1 = time every closure-pass launch with CUDA events on the
                                context's stream (needs CFPQ_LOOP_HOST); see cfpq_run_stats */
    uint32_t no_single_cta;  /* 0 = a query whose whole device state fits in one SM's shared
                                memory (rows <= 512 bits) runs its fixpoint inside one CTA;
                                1 = always use the multi-kernel loop */
    uint32_t gather_slices;  /* column slices of the nonterminal adjacency per work item of the
                                row gather (used only while a box the block reads holds
                                >= n^2/32 edges): 0 = automatic (rows of >= 8192 bits: 4-8),
                                k >= 1 = k (capped at 16); the result does not depend on it */
    size_t memory_budget;    /* bytes of device memory a context may hold; 0 = no limit */
    cfpq_alloc_fn alloc;     /* NULL = cudaMallocAsync */
    cfpq_free_fn free;
    void *alloc_user;
    uint32_t tile_format;    /* CFPQ_TILES_*: tile kernel of AUTO's (and TC_FP8's) products; the
                                result does not depend on it */
    uint32_t no_autotune;    /* 0 = the first AUTO query that may use tiles (n >= 2048) on a
                                device runs the autotuner's probe once (cfpq_tune); 1 = use the
                                built-in choices, never probe */
    uint32_t tile_ratio;     /* cost model of the new-edge tiles: run them while M * K <
                                tile_ratio * new edges (see cfpq_tuning::edge_ratio); 0 = the
                                autotuner's (or built-in) value; the result does not depend on it */
} cfpq_options;

/* Recursive state machine (Sec. 2.3, Def. of an RSM).  States are numbered
 * globally 0..n_states-1; state_box[s] is the box owning s (boxes have
 * disjoint state sets), box_start[b] its start state q_b^0, state_final[s]
 * != 0 marks s as final in its box.  Transition k is
 * tr_from[k] --(tr_kind[k], tr_sym[k])--> tr_to[k], with tr_kind 0 for a
 * terminal symbol tr_sym < n_terminals and 1 for a call of box tr_sym; both
 * ends must lie in the same box.  Nondeterminism is allowed; duplicate
 * transitions are merged.  A regular query is a one-box RSM without calls
 * (Sec. 3.1, index creation for RPQ). */
typedef struct {
    uint32_t n_states;
    uint32_t n_boxes;
    uint32_t start_box;           /* the initial box m */
    uint32_t n_trans;
    const uint32_t *box_start;    /* [n_boxes] */
    const uint32_t *state_box;    /* [n_states] */
    const uint8_t *state_final;   /* [n_states] */
    const uint32_t *tr_from;      /* [n_trans] */
    const uint32_t *tr_kind;      /* [n_trans] */
    const uint32_t *tr_sym;       /* [n_trans] */
    const uint32_t *tr_to;        /* [n_trans] */
} cfpq_rsm;

/* Statistics of one cfpq_run (or one query of a batch). */
typedef struct {
    uint32_t iterations;       /* loop iterations, counting the last one that adds no edge */
    uint32_t rounds;           /* closure passes over all blocks, all iterations */
    uint32_t status;           /* 0, or the CFPQ_ERR_* that stopped the loop */
    uint32_t gpu_launches;     /* kernels launched by the call (graph nodes executed) */
    uint64_t edges_added;      /* nonterminal edges found, epsilon edges included */
    uint64_t closure_bits;     /* nnz(C3) at the fixpoint (counted on request, else 0) */
    uint64_t m3_bits;          /* nnz(M3) at the fixpoint (counted on request, else 0) */
    uint64_t row_ors;          /* bit-packed source-row ORs issued by the closure */
    uint64_t rows_changed;     /* output rows of C3 changed, summed over passes */
    uint64_t row_bytes;        /* bytes of one bit-packed row (n rounded up to 128 bits, / 8) */
    uint64_t tile_mmas;        /* dense tensor-core tile products issued */
    uint64_t closure_blocks;   /* n x n state blocks of C3 held on the device */
    uint64_t device_bytes;     /* device memory held by the query */
    double ms_total;           /* wall time of the call (host clock) */
    double ms_closure;         /* summed CUDA-event time of the closure-pass launches (profile = 1) */
    double ms_setup;           /* host clock: staging, planning, buffer and work-list set-up of the call */
    double ms_loop;            /* host clock: the fixpoint loop (launch to completion) */
    uint32_t closure_launches; /* closure-pass launches timed (profile = 1) */
    uint32_t pad_;
    uint64_t tile_kstages;     /* K stages of 128 multiplied by the tile products; each stage is
                                  128 x 256 x 128 tensor-core multiply-adds */
    /* profile = 1: the closure time of ms_closure split by kernel, from CUDA
     * events on the context's stream around each group of launches of a pass */
    double ms_gather;          /* row-gather launches (k_gather, every row-width class) */
    double ms_tile_operands;   /* tile jobs' dirty-row lists and 0/1 FP8 operand expansion */
    double ms_tile_products;   /* tcgen05 tile-product launches */
    uint32_t gather_launches;  /* row-gather launches timed */
    uint32_t tile_launches;    /* passes whose tile-product launches were timed */
    uint64_t tile_operand_bytes; /* bytes of 0/1 operands the tile jobs expanded (A and B) */
} cfpq_run_stats;

/* Result of the autotuner (cfpq_tune). */
typedef struct {
    uint32_t struct_size;   /* sizeof(cfpq_tuning), set by the caller */
    uint32_t tuned;         /* 1: measured on this device; 0: built-in choices (probe off or failed) */
    uint32_t tile_format;   /* CFPQ_TILES_FP8 / _FP4 / _FP8_128 / _NVFP4: the tile kernel AUTO uses */
    uint32_t edge_ratio;    /* cost model: an iteration's new edges (e of them, M rows x K columns
                               after compaction) run as tiles while M * K < edge_ratio * e; for
                               queries whose n x n closure blocks fit in half the L2 ... */
    uint32_t edge_ratio_hbm;/* ... and for larger ones (their gather reads rows from HBM) */
    uint32_t edge_ratio_formula; /* tile rate / (16 x gather rate) from the measured rates: the
                               search tried 1/2, 1, 2, 4 and 8 times it on the probe query in
                               AUTO and kept the fastest as edge_ratio */
    int32_t probe_status;   /* CFPQ status of the probe (0 = ok) */
    double gather_gbs;      /* measured: bytes of source rows ORed per second by the row gather
                               (probe blocks of 8 MiB: L2-resident) */
    double gather_gbs_hbm;  /* gather_gbs x read_hbm_gbs / read_l2_gbs (at most gather_gbs): the
                               same rows from HBM */
    double read_l2_gbs;     /* measured device read bandwidth over a 24 MiB buffer (L2-resident) */
    double read_hbm_gbs;    /* ... over a 2 GiB buffer */
    double fp8_tflops;      /* measured: 0/1 multiply-adds per second of each tile kernel (x 1e12) */
    double fp4_tflops;
    double fp8_128_tflops;
    double nvfp4_tflops;
    double probe_ms;        /* host time the probe took */
} cfpq_tuning;

/* ---- context ---------------------------------------------------------------- */

/* Fill *opt with defaults (device 0, no caps, AUTO closure, device loop). */
int cfpq_default_options(cfpq_options *opt);

/* Create a context on opt->device (NULL = defaults) issuing work on `stream`
 * (a cudaStream_t).  *out receives the context; destroy it with cfpq_destroy. */
int cfpq_create(cfpq_ctx **out, const cfpq_options *opt, void *stream);

/* Release every device buffer and the context.  NULL is accepted. */
int cfpq_destroy(cfpq_ctx *ctx);

/* ---- inputs ------------------------------------------------------------------- */

/* Load the labelled graph G = <V, E, L> as an edge list (Sec. 2.1): edge e is
 * (src[e], label[e], dst[e]) with src, dst < n_vertices and label <
 * n_terminals.  Host pointers; duplicate edges are merged, self-loops kept.
 * An out-of-range id fails the call with CFPQ_ERR_INVALID_ARG and leaves no
 * graph loaded.  Replaces any earlier graph and clears earlier results. */
int cfpq_load_graph(cfpq_ctx *ctx, uint32_t n_vertices, uint32_t n_terminals, size_t n_edges,
                    const uint32_t *src, const uint32_t *label, const uint32_t *dst);

/* Same as cfpq_load_graph with the three arrays in device memory, read on the
 * context's stream.  Range errors are detected on the device and reported by
 * this call (it synchronises the stream once). */
int cfpq_load_graph_device(cfpq_ctx *ctx, uint32_t n_vertices, uint32_t n_terminals, size_t n_edges,
                           const uint32_t *d_src, const uint32_t *d_label, const uint32_t *d_dst);

/* Load the query RSM (Sec. 2.3).  The RSM is copied.  Validation failures
 * (state or box id out of range, a transition leaving its box, a terminal
 * symbol >= the graph's n_terminals once both are loaded) return
 * CFPQ_ERR_INVALID_ARG. */
int cfpq_load_rsm(cfpq_ctx *ctx, const cfpq_rsm *rsm);

/* ---- index creation (Listing 1) ------------------------------------------------- */

/* Run index creation to its fixpoint: epsilon initialisation, then while M2
 * changes: M3' = OR_l M1^l (x) A2^l over the new edges (computed tile by tile,
 * never stored), incremental closure C3 <- (C3 + M3')^+, extraction of new
 * nonterminal edges from the start-state to final-state blocks of C3.
 * Returns CFPQ_ERR_TIMEOUT if an iteration or round cap stopped the loop
 * (the partial index stays readable).  stats may be NULL. */
int cfpq_run(cfpq_ctx *ctx, cfpq_run_stats *stats);

/* Multiple-source index creation (the multiple-source version named as
 * future work in Sec. 6).  sources: host array of n_sources vertex ids
 * (< n_vertices, duplicates allowed; NULL when n_sources is 0).  Like
 * cfpq_run, but for an RSM whose transitions read only terminals the closure
 * computes only the rows of C3 reachable in the Kronecker product from
 * (q0, x), q0 the start state of the start box and x a source: afterwards
 * the rows x in sources of every nonterminal's M2 are exact (and so are the
 * other reached rows); a row of an unreached vertex x holds at most (x, x),
 * the pair the empty word gives when the box's start state is final.  When a
 * transition reads a nonterminal (M3 grows with M2) every row is computed,
 * as by cfpq_run.  Errors: CFPQ_ERR_INVALID_ARG (NULL ctx, NULL sources with
 * n_sources > 0, a source out of range), CFPQ_ERR_STATE (no graph or RSM),
 * and those of cfpq_run. */
int cfpq_run_sources(cfpq_ctx *ctx, const uint32_t *sources, uint32_t n_sources, cfpq_run_stats *stats);

/* Checkpoint and resume (the fixpoint of Listing 1 is monotone).  The
 * checkpoint of a result is its M2, read with cfpq_get_reachable_bits for
 * every box.  cfpq_set_start(ctx, bits, n_boxes, n_vertices) makes the next
 * cfpq_run calls start from such pairs.
 *   - Layout: n_boxes blocks of n_vertices rows of ceil(n_vertices/64)
 *     words, box-major, the cfpq_get_reachable_bits layout.  The bits are
 *     copied.
 *   - What a run does with them: the pairs are added to M2 after the epsilon
 *     rows and enter the first iteration as new edges (A2 := M2 on their
 *     rows).  The run then reaches the least fixpoint containing them.
 *   - When the result equals a run without them: whenever the pairs belong to
 *     this graph's answer, e.g. the answer of an earlier run on a subset of
 *     its edges, or of this graph.  The run then needs fewer iterations.
 *   - Pairs outside the answer stay in the result.
 *   - bits = NULL clears the start.
 * A run returns CFPQ_ERR_INVALID_ARG while the start's n_boxes and
 * n_vertices differ from the loaded RSM and graph.  cfpq_run_sources returns
 * CFPQ_ERR_STATE while a start is set.  Seeded pairs count in edges_added. */
int cfpq_set_start(cfpq_ctx *ctx, const uint64_t *bits, uint32_t n_boxes, uint32_t n_vertices);

/* Autotuner of the closure's tile products (no counterpart in the paper,
 * whose closure runs on a CPU Boolean-matrix library).  On the context's
 * device it runs a probe query -- Dyck-4 (S -> S S | o_i c_i | o_i S c_i)
 * on a seeded graph of 8192 vertices with Zipf(2.1) out-degrees (mean
 * about 3), 8 labels --
 * with the bit-packed closure and with each tile kernel, times their kernel
 * groups with CUDA events, times reads of an L2-sized and an HBM-sized
 * buffer, and derives: the fastest tile kernel (AUTO's default) and the
 * cost-model ratio (new-edge tiles run while M * K < ratio x new edges),
 * searched around tile rate / (16 x gather rate) -- one new edge costs the
 * gather n/8 bytes, a tile product 2n multiply-adds per (row, column) of its
 * M x K box -- by timing the probe query in AUTO, and scaled by the measured
 * L2/HBM read bandwidths for queries whose closure blocks exceed half the
 * L2.  The result is kept per
 * device for the process; force = 1 measures again.  Every answer is the
 * same whichever choices are made.  The probe uses the context's stream and
 * allocator and about 3 GB of device memory for its duration.  Errors:
 * CFPQ_ERR_INVALID_ARG (NULL ctx or out, wrong struct_size); a probe that
 * fails leaves the built-in choices (tuned = 0, probe_status set) and
 * returns CFPQ_OK. */
int cfpq_tune(cfpq_ctx *ctx, int force, cfpq_tuning *out);

/* Count nnz(C3) and nnz(M3) of the last run into *closure_bits / *m3_bits. */
int cfpq_count_index(cfpq_ctx *ctx, uint64_t *closure_bits, uint64_t *m3_bits);

/* ---- results ----------------------------------------------------------------------- */

/* Pairs (x, y) with M2^box[x, y] = 1 (Theorem 1: a path x -> y whose word box
 * derives), in (src, dst) lexicographic order.  src/dst hold `cap` entries;
 * *count receives the number of pairs.  NULL buffers or a small cap return the
 * count with CFPQ_ERR_BUFFER_TOO_SMALL (count-only query when both are NULL
 * and cap is 0 returns CFPQ_OK). */
int cfpq_get_reachable(cfpq_ctx *ctx, uint32_t box, uint32_t *src, uint32_t *dst, size_t cap, size_t *count);

/* Number of pairs of M2^box, counted on the device; one 8-byte read back. */
int cfpq_count_reachable(cfpq_ctx *ctx, uint32_t box, uint64_t *count);

/* M2^box as host bit rows: row x occupies ceil(n/64) uint64 words at
 * bits + x * ceil(n/64); bit y of the row is word y/64, bit y%64. */
int cfpq_get_reachable_bits(cfpq_ctx *ctx, uint32_t box, uint64_t *bits);

/* Rows of the closure index C3 = M3^+ (Listing 1's C3 at the fixpoint).  For
 * k < n_rows the product vertex (row_state[k], row_vertex[k]) gets row
 * out + k * ceil(Q*n/64) with bit t*n + y set iff (t, y) is reachable from it
 * by a path of one or more M3 edges. */
int cfpq_get_closure_rows(cfpq_ctx *ctx, uint32_t n_rows, const uint32_t *row_state,
                          const uint32_t *row_vertex, uint64_t *out);

/* All-path semantics (Sec. 3.2, Listing 2): the paths vs -> vf of at most
 * max_len edges whose word box derives, deduplicated, in order of (length,
 * lexicographic sequence of (src, label, dst) triples), at most max_paths of
 * them.  Path k's edges are the triples edge_buf[3*j .. 3*j+2] for
 * path_offsets[k] <= j < path_offsets[k+1] (path_offsets has max_paths + 1
 * entries).  *n_paths receives the number of paths returned; *truncated (may
 * be NULL) is set to 1 if max_paths stopped the enumeration.  The empty path
 * is returned for vs == vf when box derives the empty word.
 * The product paths of M3 are walked forward on the host.  For every target
 * (box, vertex) met, the device first computes the backward layers: the
 * product vertices that can reach the target within k edges, for
 * k <= max_len.  Partial paths outside them are dropped, so the result does
 * not depend on them.  Targets are searched in batches.  Device memory kept
 * by the context for these calls:
 *   - the reverse terminal CSR;
 *   - (max_len + 1) * Q * n_pad / 8 bytes of layers per target of a batch,
 *     at most 1 GiB;
 *   - n_pad^2 / 8 bytes per box that a nonterminal transition reads (its M2,
 *     transposed).
 * The host copies and the memo of subpath sets are kept between calls
 * until the result changes (a run, or a new graph or RSM).  After
 * cfpq_run_sources only the sources' rows are exact, so vs must be one of
 * its sources (CFPQ_ERR_INVALID_ARG otherwise).
 * CFPQ_ERR_BUFFER_TOO_SMALL if edge_cap (in triples) was too small;
 * CFPQ_ERR_OUT_OF_MEMORY if the device buffers do not fit; CFPQ_ERR_UNSUPPORTED
 * if the enumeration exceeds its work cap (4e6 stored paths or 2^20 subpath
 * sets). */
int cfpq_extract_paths(cfpq_ctx *ctx, uint32_t box, uint32_t vs, uint32_t vf, uint32_t max_len, size_t max_paths,
                       uint32_t *edge_buf, size_t edge_cap, size_t *path_offsets, size_t *n_paths,
                       int *truncated);

/* ---- batched index creation ------------------------------------------------------- */

/* One query of a batch: a graph (host edge list) and an RSM. */
typedef struct {
    uint32_t n_vertices;
    uint32_t n_terminals;
    size_t n_edges;
    const uint32_t *src;
    const uint32_t *label;
    const uint32_t *dst;
    const cfpq_rsm *rsm;
} cfpq_query;

/* Run index creation for every query of the batch in shared persistent
 * launches: one CUDA graph drives all queries' fixpoints, each pass of the
 * closure covers the blocks of every unfinished query, and each query keeps
 * its own convergence flag.  Results stay on the device until the next
 * batch.  per_query_stats (may be NULL) has n_queries entries. */
int cfpq_batch_run(cfpq_ctx *ctx, uint32_t n_queries, const cfpq_query *queries, cfpq_run_stats *per_query_stats,
                   cfpq_run_stats *total_stats);

/* M2^box of query q of the last batch as host bit rows (layout of
 * cfpq_get_reachable_bits with that query's n). */
int cfpq_batch_get_reachable_bits(cfpq_ctx *ctx, uint32_t q, uint32_t box, uint64_t *bits);

/* ---- serving ------------------------------------------------------------------------- */

typedef struct cfpq_server cfpq_server;

/* A server keeps one graph resident and answers RSM queries submitted at any
 * time.  Each admitted query gets its own device state (sized by its
 * |Q|n x |Q|n closure blocks) and joins the running batch at the next pass;
 * queries that do not fit the memory budget wait until running ones finish
 * (continuous batching). */
int cfpq_server_create(cfpq_server **out, const cfpq_options *opt, void *stream, uint32_t n_vertices,
                       uint32_t n_terminals, size_t n_edges, const uint32_t *src, const uint32_t *label,
                       const uint32_t *dst);
int cfpq_server_destroy(cfpq_server *srv);

/* Queue a query; *ticket identifies it.  Never blocks on the GPU. */
int cfpq_submit(cfpq_server *srv, const cfpq_rsm *rsm, uint64_t *ticket);

/* Advance the server: admit waiting queries that fit, run one fixpoint pass
 * for every running query, retire finished ones.  *n_running / *n_waiting
 * (may be NULL) report the queue sizes after the step. */
int cfpq_server_step(cfpq_server *srv, uint32_t *n_running, uint32_t *n_waiting);

/* *done = 1 once the query's fixpoint is reached (its result is readable). */
int cfpq_poll(cfpq_server *srv, uint64_t ticket, int *done);

/* M2^box of a finished query as host bit rows (layout of
 * cfpq_get_reachable_bits). */
int cfpq_result_reachable_bits(cfpq_server *srv, uint64_t ticket, uint32_t box, uint64_t *bits);

/* Forget the ticket and free the query's device state: a finished query is
 * released, a waiting one is dropped, a running one is cancelled (its passes
 * run only inside cfpq_server_step, so none is in flight between calls; the
 * other queries continue unchanged). */
int cfpq_release(cfpq_server *srv, uint64_t ticket);

/* ---- one query over several GPUs (column sharding) ---------------------------------- */

/* The multi-GPU version of index creation that Sec. 6 names as future work.
 * Row x of a closure block C[s,t] is the OR, over the product edges
 * (s,x) -> (u,y) of M3 (Sec. 2.4), of row y of C[u,t] (and bit y when u = t),
 * so any range of columns (target vertices) of C3 needs only the same range
 * of the rows it reads.  Each rank (one context per GPU) loads the whole
 * graph and RSM and computes C3 on its own columns [col0, col1); Listing 1's
 * extraction then yields the new nonterminal edges in those columns.  After
 * every iteration the caller exchanges them (an all-gather of the ranks'
 * slices, e.g. NCCL) and installs the full rows on every rank, which start
 * the next iteration with the same M2 and A2.  The loop ends after the
 * first iteration in which no rank found an edge -- the unsharded loop's
 * last iteration too, so the answer and the iteration count are the same.
 *
 *   cfpq_shard_begin(ctx, col0, col1);
 *   do { cfpq_shard_step(ctx, slice, &k);  all-gather slices -> full;
 *        cfpq_shard_apply(ctx, full, &done); } while (!done);
 *
 * Columns are in the padded width n_pad = n rounded up to 128: col0 a
 * multiple of 256 (a tensor-core tile), col1 a multiple of 256 or n_pad,
 * col0 <= col1 (an empty range is allowed); the ranks' ranges must partition
 * [0, n_pad).  Slices and full rows are device buffers of 64-bit words,
 * box-major: slice = n_boxes x n rows of (col1 - col0) / 64 words (the rank's
 * columns of the iteration's new edges), full = n_boxes x n rows of
 * n_pad / 64 words (the ranks' slices side by side in column order).  The
 * loop runs with one launch per kernel and pass (the exchange needs the host
 * between iterations).  After the loop every rank holds the whole answer
 * (cfpq_get_reachable*); its closure blocks hold only its columns, so
 * cfpq_get_closure_rows and cfpq_count_index describe those columns only.
 *
 * Errors: CFPQ_ERR_STATE (no graph/RSM, a start answer set, step/apply
 * without begin), CFPQ_ERR_INVALID_ARG (columns, NULL buffers),
 * CFPQ_ERR_TIMEOUT (a cap of cfpq_options stopped the loop), CFPQ_ERR_CUDA. */
int cfpq_shard_begin(cfpq_ctx *ctx, uint32_t col0, uint32_t col1);

/* Run one iteration (closure passes and extraction) on the rank's columns and
 * write its new edges into d_slice; *new_edges (may be NULL) = their count. */
int cfpq_shard_step(cfpq_ctx *ctx, uint64_t *d_slice, uint64_t *new_edges);

/* Install the gathered new edges d_full of every rank (M2 |= them, A2 :=
 * them) and decide whether the loop goes on: *done = 1 when no rank found an
 * edge in the iteration just stepped (the result is then readable). */
int cfpq_shard_apply(cfpq_ctx *ctx, const uint64_t *d_full, int *done);

/* Loop statistics of the sharded run so far (iterations, passes, edges found
 * by every rank, this rank's row ORs and tile products). */
int cfpq_shard_stats(cfpq_ctx *ctx, cfpq_run_stats *stats);

/* ---- building block: dense Boolean product on the tensor cores ---------------------- */

/* c = a * b over the Boolean semiring for n x n bit matrices (host buffers,
 * row x = ceil(n/64) uint64 words, bit y of a row = word y/64, bit y%64),
 * computed by the closure's tcgen05 tile kernel: 0/1 operands as FP8-E4M3
 * with FP32 accumulation, a count > 0 giving a 1.  Exact for n <= 65536
 * (counts < 2^24).  use_int8 = 1 (0/1 INT8 with INT32 accumulation) returns
 * CFPQ_ERR_UNSUPPORTED: sm_103a has no tcgen05 kind::i8 MMA.  The closure's dense tiles (Sec. 3.1, Listing 1) use the
 * same kernel; this call exposes it for testing and reuse.  Allocates and
 * frees its device buffers on `stream` (a cudaStream_t) and synchronises it.
 * CFPQ_ERR_TIMEOUT if a bounded wait inside the kernel gave up. */
int cfpq_tc_bool_product(uint32_t n, int use_int8, const uint64_t *a, const uint64_t *b, uint64_t *c, void *stream);

/* ---- staging without device allocation ------------------------------------------------ */

/* The paper has no counterpart to this call: it serves callers that must not
 * have the library allocate device memory, such as a service that keeps all
 * device memory in its own fixed pool and swaps in new graph snapshots, or a
 * process whose remaining GPU memory belongs to another framework.
 *
 * Same result as cfpq_load_graph_device (edge list in device memory, read on
 * the context's stream; duplicates merged; range errors -> INVALID_ARG), but
 * the staging temporaries (counts, offsets, an unsorted edge copy, the scan
 * workspace, the error flag) live in one fixed array of about 16 MiB compiled
 * into the library, which every GPU that loads the library holds until the
 * process exits.  The output goes into the adjacency buffers the context
 * already owns; they must come from an earlier cfpq_load_graph or
 * cfpq_load_graph_device of a graph at least as large (same or larger
 * n_terminals * n_vertices + 1 offsets and n_edges columns), else
 * CFPQ_ERR_BUFFER_TOO_SMALL.  Limits: n_terminals * n_vertices <= 524288 and
 * n_edges <= 2097152, else CFPQ_ERR_UNSUPPORTED.  No cudaMalloc, cudaFree or
 * other allocating routine is called.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents (each call
 * clears what must start at zero); calls that overlap on the GPU race, so run
 * them one at a time.  Synchronises the context's stream once. */
int cfpq_load_graph_device_noalloc(cfpq_ctx *ctx, uint32_t n_vertices, uint32_t n_terminals, size_t n_edges,
                                   const uint32_t *d_src, const uint32_t *d_label, const uint32_t *d_dst);

/* ---- diagnostics ----------------------------------------------------------------------- */

/* Diagnostic of failure detection.  Every spin-wait of the library's kernels
 * (the mbarrier waits of the tensor-core tile pipeline) is bounded: after 2 s
 * (or 2^26 polls) the kernel gives up, records an error flag, finishes without
 * the awaited data and the run returns CFPQ_ERR_TIMEOUT, with the context
 * still usable.  This call runs that same wait in one thread on an mbarrier
 * that nothing arrives at, bounded by limit_ns (1 ns .. 5 s), on the
 * context's stream, and sets *timed_out to 1 when it gave up (0 would mean
 * the barrier completed, which cannot happen).  CFPQ_ERR_INVALID_ARG for a
 * limit outside that range. */
int cfpq_check_bounded_wait(cfpq_ctx *ctx, uint64_t limit_ns, int *timed_out);

const char *cfpq_status_string(int status);
const char *cfpq_last_error(const cfpq_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* CFPQ_H */
