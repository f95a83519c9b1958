// cfpq_api.cu -- the C ABI of libcfpq (include/cfpq.h).
//
// Every entry point catches C++ exceptions and maps CUDA errors to status
// codes; nothing but plain C types crosses the boundary.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <set>
#include <string>
#include <vector>

#include "cfpq_ctx.cuh"
#include "cfpq_paths_host.h"

using namespace cfpq;

namespace cfpq {
// The tile kernel and cost-model ratio of a query run with options o on a
// graph of n vertices: the autotuner's choice for AUTO with the default tile
// format (its probe runs first when such a query may use tiles, n >= 2048),
// else the format asked for.
void set_tiles(QueryDev &q, const cfpq_options &o, cudaStream_t st, uint32_t n) {
    const bool want = o.closure_mode == CFPQ_CLOSURE_AUTO && o.tile_format == CFPQ_TILES_DEFAULT &&
                      n >= kAutoTilesMinN;
    const Tuning t = o.no_autotune ? Tuning{} : device_tuning(o, st, want, false);
    q.tile_kind = tile_kind_of(o.closure_mode, o.tile_format, t);
    q.tile_fp4 = tile_kind_fp4(q.tile_kind);
    q.tile_ratio = o.tile_ratio ? o.tile_ratio : tile_ratio_of(q.tile_kind, t, n);
}
}  // namespace cfpq

namespace {

constexpr uint32_t kDefaultPassCap = 1u << 20;

int fail(cfpq_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

#define API_TRY try {
#define API_CATCH(ctx)                                                   \
    }                                                                    \
    catch (const std::bad_alloc &) {                                     \
        return fail(ctx, CFPQ_ERR_OUT_OF_MEMORY, "host allocation failed"); \
    }                                                                    \
    catch (const std::exception &e) {                                    \
        return fail(ctx, CFPQ_ERR_CUDA, e.what());                       \
    }                                                                    \
    catch (...) {                                                        \
        return fail(ctx, CFPQ_ERR_CUDA, "unknown exception");            \
    }

#define CK(ctx, call)                                                                               \
    do {                                                                                            \
        cudaError_t _e = (call);                                                                    \
        if (_e != cudaSuccess) return fail(ctx, CFPQ_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)

int set_device(cfpq_ctx *ctx) {
    CK(ctx, cudaSetDevice(ctx->opt.device));
    return CFPQ_OK;
}

uint32_t pass_cap(const cfpq_options &o) { return kDefaultPassCap; }

void fill_stats(cfpq_run_stats *s, const QCtl &c, const QueryDev &q, double ms) {
    memset(s, 0, sizeof(*s));
    s->rows_changed = c.rows_changed_total;
    s->row_bytes = (uint64_t)q.W * 8;
    s->iterations = c.iters_done;
    s->rounds = (uint32_t)c.rounds_total;
    s->status = c.status == kStatusOk ? 0 : (uint32_t)(-CFPQ_ERR_TIMEOUT);
    s->edges_added = c.edges_total;
    s->row_ors = c.row_ors;
    s->tile_mmas = c.tile_mmas;
    s->tile_kstages = c.tile_kstages;
    s->tile_operand_bytes = c.tile_operand_bytes;
    s->closure_blocks = q.blocks.size();
    s->device_bytes = q.device_bytes;
    s->ms_total = ms;
}

// Per-kernel closure time of a profiled (host-loop) run.
struct ClosureProfile {
    double ms_closure = 0.0, ms_gather = 0.0, ms_operands = 0.0, ms_products = 0.0;
    uint32_t closure_launches = 0, gather_launches = 0, tile_launches = 0;
};

void put_profile(cfpq_run_stats *s, const ClosureProfile &p) {
    s->ms_closure = p.ms_closure;
    s->closure_launches = p.closure_launches;
    s->ms_gather = p.ms_gather;
    s->ms_tile_operands = p.ms_operands;
    s->ms_tile_products = p.ms_products;
    s->gather_launches = p.gather_launches;
    s->tile_launches = p.tile_launches;
}

int status_of(const QCtl &c) { return c.status == kStatusOk ? CFPQ_OK : CFPQ_ERR_TIMEOUT; }

// Run the executor's queries to their fixpoint.
int run_executor(cfpq_ctx *ctx, Executor &ex, std::vector<QCtl> *ctls, uint32_t *launches,
                 ClosureProfile *prof_out = nullptr) {
    const cudaStream_t st = ctx->stream;
    const uint32_t mi = ctx->opt.max_iterations, mr = ctx->opt.max_rounds, mp = pass_cap(ctx->opt);
    uint32_t n_gather = 0, n_extract = 0;
    for (int v = 0; v < kClasses; ++v) {
        n_gather += ex.n_items[v] ? 1 : 0;
        n_extract += ex.n_xitems[v] ? 1 : 0;
    }
    // tile jobs: new-edge columns, row list, A and B operands, the two product kernels
    const uint32_t per_pass = n_gather + n_extract + (ex.n_tcjobs ? 6 : 0) + (n_extract ? 0 : 1);
    if (ctx->opt.loop_mode == CFPQ_LOOP_HOST) {
        if (ex.enqueue_prologue(st, mi, mr, mp)) return fail(ctx, CFPQ_ERR_CUDA, "prologue launch failed");
        int running = 1;
        uint32_t passes = 0;
        const bool prof = ctx->opt.profile != 0;
        cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
        auto drop_events = [&]() {
            for (auto &e : ev)
                if (e) cudaEventDestroy(e);
        };
        if (prof)
            for (auto &e : ev) CK(ctx, cudaEventCreate(&e));
        ClosureProfile P;
        while (running) {
            if (ex.enqueue_pass(st, 0, 0, ex.running.as<int>(), prof ? ev : nullptr)) {
                drop_events();
                return fail(ctx, CFPQ_ERR_CUDA, "pass launch failed");
            }
            CK(ctx, cudaMemcpyAsync(&running, ex.running.p, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(ctx, cudaStreamSynchronize(st));
            if (prof) {
                float a = 0.f, b = 0.f, c = 0.f;
                CK(ctx, cudaEventElapsedTime(&a, ev[0], ev[1]));
                CK(ctx, cudaEventElapsedTime(&b, ev[1], ev[2]));
                CK(ctx, cudaEventElapsedTime(&c, ev[2], ev[3]));
                P.ms_operands += a;
                P.ms_gather += b;
                P.ms_products += c;
            }
            ++passes;
        }
        if (prof) {
            drop_events();
            P.ms_closure = P.ms_gather + P.ms_operands + P.ms_products;
            P.closure_launches = passes * n_gather;
            P.gather_launches = passes * n_gather;
            P.tile_launches = ex.n_tcjobs ? passes : 0;
            if (prof_out) *prof_out = P;
        }
        if (launches) *launches = passes * per_pass + 2;
    } else {
        if (!ex.exec) {
            std::string e;
            if (ex.build_graph(st, mi, mr, mp, &e)) return fail(ctx, CFPQ_ERR_CUDA, e);
        }
        CK(ctx, cudaGraphLaunch(ex.exec, st));
    }
    int tc_error = 0;
    if (ex.read_ctls(st, ctls, &tc_error)) return fail(ctx, CFPQ_ERR_CUDA, "reading loop state failed");
    if (tc_error)
        return fail(ctx, CFPQ_ERR_TIMEOUT, "a tile-product kernel gave up (bounded wait on its MMAs or on a counter)");
    if (ctx->opt.loop_mode != CFPQ_LOOP_HOST && launches) {
        // the graph's loop body holds kLoopUnroll passes
        uint32_t passes = 0;
        for (const auto &c : *ctls) passes = std::max(passes, c.passes);
        *launches = (passes + kLoopUnroll - 1) / kLoopUnroll * kLoopUnroll * per_pass + 2;
    }
    CK(ctx, cudaGetLastError());
    return CFPQ_OK;
}

int ensure_query(cfpq_ctx *ctx, bool restricted = false) {
    if (!ctx->has_graph) return fail(ctx, CFPQ_ERR_STATE, "no graph loaded");
    if (!ctx->has_rsm) return fail(ctx, CFPQ_ERR_STATE, "no RSM loaded");
    QueryDev &q = ctx->query;
    q.g = &ctx->graph;
    q.closure_mode = ctx->opt.closure_mode;
    {
        const uint32_t kind0 = q.tile_kind, ratio0 = q.tile_ratio;
        set_tiles(q, ctx->opt, ctx->stream, ctx->graph.n);
        if (q.tile_kind != kind0 || q.tile_ratio != ratio0) ctx->exec_dirty = true;
        if (int rc = set_device(ctx)) return rc;  // (a probe may have run)
    }
    q.gather_slices = ctx->opt.gather_slices;
    q.full_kcap = true;
    if (q.restricted != restricted) ctx->exec_dirty = true;  // the work items carry the row masks
    q.restricted = restricted;
    const bool seeded = ctx->has_start;
    if (seeded && (ctx->start_B != q.rsm.B || ctx->start_n != ctx->graph.n))
        return fail(ctx, CFPQ_ERR_INVALID_ARG, "the start answer does not match the graph and RSM");
    if (q.seeded != seeded) ctx->exec_dirty = true;  // the prologue captured in the loop's graph changes
    q.seeded = seeded;
    if (q.prepared && q.graph_generation == ctx->graph.generation && !ctx->exec_dirty) {
        // Same plan and work lists: a graph of the same shape may have been
        // loaded since, so rebuild what was derived from the old edges.
        std::string e;
        bool moved = false;
        if (int rc = q.refresh_graph_caches(&ctx->A, ctx->stream, &e, &moved)) return fail(ctx, rc, e);
        if (moved) ctx->exec_dirty = true;
    }
    if (!q.prepared || q.graph_generation != ctx->graph.generation || ctx->exec_dirty) {
        std::string e;
        int rc = q.prepare(&ctx->A, &e);
        if (rc) return fail(ctx, rc, e);
        if (restricted && !q.reach_mem.ensure(&ctx->A, (size_t)q.Q * q.W * 8, &e))
            return fail(ctx, CFPQ_ERR_OUT_OF_MEMORY, e);
        ctx->exec.qs.assign(1, &q);
        rc = ctx->exec.assemble(&ctx->A, ctx->stream, &e);
        if (rc) return fail(ctx, rc, e);
        q.small_ok = false;
        if (!ctx->opt.no_single_cta && !restricted && !seeded) {
            rc = q.prepare_small(&ctx->A, ctx->stream, ctx->opt.max_iterations, kDefaultPassCap, &e);
            if (rc) return fail(ctx, rc, e);
        }
        ctx->exec_dirty = false;
    }
    return CFPQ_OK;
}

int bits_to_host(cfpq_ctx *ctx, const uint64_t *dev_rows, uint32_t n, uint32_t W, uint64_t *bits) {
    const size_t wn = (n + 63) / 64;
    CK(ctx, cudaMemcpy2DAsync(bits, wn * 8, dev_rows, (size_t)W * 8, wn * 8, n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return CFPQ_OK;
}

}  // namespace

extern "C" {

const char *cfpq_status_string(int status) {
    switch (status) {
        case CFPQ_OK: return "ok";
        case CFPQ_ERR_INVALID_ARG: return "invalid argument";
        case CFPQ_ERR_OUT_OF_MEMORY: return "out of memory";
        case CFPQ_ERR_BUFFER_TOO_SMALL: return "buffer too small";
        case CFPQ_ERR_TIMEOUT: return "iteration or round cap reached";
        case CFPQ_ERR_NOT_READY: return "result not ready";
        case CFPQ_ERR_CUDA: return "CUDA error";
        case CFPQ_ERR_STATE: return "calls out of order";
        case CFPQ_ERR_UNSUPPORTED: return "unsupported size or mode";
        default: return "unknown status";
    }
}

const char *cfpq_last_error(const cfpq_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int cfpq_default_options(cfpq_options *opt) {
    if (!opt) return CFPQ_ERR_INVALID_ARG;
    memset(opt, 0, sizeof(*opt));
    opt->struct_size = sizeof(cfpq_options);
    opt->device = 0;
    opt->closure_mode = CFPQ_CLOSURE_AUTO;
    opt->loop_mode = CFPQ_LOOP_DEVICE;
    return CFPQ_OK;
}

int cfpq_create(cfpq_ctx **out, const cfpq_options *opt, void *stream) {
    if (!out) return CFPQ_ERR_INVALID_ARG;
    *out = nullptr;
    API_TRY
    std::unique_ptr<cfpq_ctx> c(new cfpq_ctx());
    if (opt) {
        if (opt->struct_size != sizeof(cfpq_options)) return CFPQ_ERR_INVALID_ARG;
        c->opt = *opt;
    } else {
        cfpq_default_options(&c->opt);
    }
    if (c->opt.loop_mode > CFPQ_LOOP_HOST || c->opt.closure_mode > CFPQ_CLOSURE_TC_FP4 ||
        c->opt.tile_format > CFPQ_TILES_NVFP4)
        return CFPQ_ERR_INVALID_ARG;
    if (c->opt.closure_mode == CFPQ_CLOSURE_TC_I8) return CFPQ_ERR_UNSUPPORTED;  // no kind::i8 MMA on sm_103a
    if (c->opt.profile && c->opt.loop_mode != CFPQ_LOOP_HOST) return CFPQ_ERR_INVALID_ARG;
    if ((c->opt.alloc == nullptr) != (c->opt.free == nullptr)) return CFPQ_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c->opt.device < 0 || c->opt.device >= ndev) {
        cudaGetLastError();
        return CFPQ_ERR_CUDA;
    }
    if (cudaSetDevice(c->opt.device) != cudaSuccess) return CFPQ_ERR_CUDA;
    c->stream = static_cast<cudaStream_t>(stream);
    c->A.alloc = c->opt.alloc;
    c->A.free = c->opt.free;
    c->A.user = c->opt.alloc_user;
    c->A.stream = c->stream;
    c->A.budget = c->opt.memory_budget;
    *out = c.release();
    return CFPQ_OK;
    API_CATCH(nullptr)
}

int cfpq_destroy(cfpq_ctx *ctx) {
    if (!ctx) return CFPQ_OK;
    API_TRY
    cudaSetDevice(ctx->opt.device);
    cudaStreamSynchronize(ctx->stream);
    delete ctx;
    return CFPQ_OK;
    API_CATCH(nullptr)
}

static int load_graph_impl(cfpq_ctx *ctx, uint32_t n, uint32_t nt, size_t m, const uint32_t *s, const uint32_t *l,
                           const uint32_t *d, bool dev) {
    if (!ctx) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (int rc = set_device(ctx)) return rc;
    ctx->has_result = false;
    ++ctx->result_gen;
    std::string e;
    int rc = stage_graph(&ctx->graph, &ctx->A, ctx->stream, n, nt, m, s, l, d, dev, &e);
    if (rc) {
        ctx->has_graph = false;
        return fail(ctx, rc, e);
    }
    ctx->has_graph = true;
    // an RSM reading more terminals than this graph has is reported by
    // cfpq_run (the caller may be about to load a matching RSM)
    return CFPQ_OK;
    API_CATCH(ctx)
}

int cfpq_load_graph(cfpq_ctx *ctx, uint32_t n_vertices, uint32_t n_terminals, size_t n_edges, const uint32_t *src,
                    const uint32_t *label, const uint32_t *dst) {
    return load_graph_impl(ctx, n_vertices, n_terminals, n_edges, src, label, dst, false);
}

int cfpq_load_graph_device(cfpq_ctx *ctx, uint32_t n_vertices, uint32_t n_terminals, size_t n_edges,
                           const uint32_t *d_src, const uint32_t *d_label, const uint32_t *d_dst) {
    return load_graph_impl(ctx, n_vertices, n_terminals, n_edges, d_src, d_label, d_dst, true);
}

int cfpq_load_rsm(cfpq_ctx *ctx, const cfpq_rsm *rsm) {
    if (!ctx) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    HostRSM h;
    std::string e;
    int rc = copy_rsm(rsm, &h, &e);
    if (rc) return fail(ctx, rc, e);
    if (ctx->has_graph && h.max_terminal_plus1 > ctx->graph.n_term)
        return fail(ctx, CFPQ_ERR_INVALID_ARG, "the RSM reads a terminal >= the graph's n_terminals");
    ctx->query.rsm = std::move(h);
    ctx->has_rsm = true;
    ctx->has_result = false;
    ++ctx->result_gen;
    ctx->exec_dirty = true;
    return CFPQ_OK;
    API_CATCH(ctx)
}

int cfpq_run(cfpq_ctx *ctx, cfpq_run_stats *stats) {
    if (!ctx) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    const auto t0 = std::chrono::steady_clock::now();
    if (int rc = set_device(ctx)) return rc;
    if (int rc = ensure_query(ctx)) return rc;
    if (ctx->has_start) {
        // the start answer, in the device's row layout (padding words zero)
        QueryDev &q = ctx->query;
        std::string e;
        const size_t wn = (q.n + 63) / 64, bytes = (size_t)q.B * q.n * q.W * 8;
        if (!q.seed_mem.ensure(&ctx->A, bytes, &e)) return fail(ctx, CFPQ_ERR_OUT_OF_MEMORY, e);
        CK(ctx, cudaMemsetAsync(q.seed_mem.p, 0, bytes, ctx->stream));
        CK(ctx, cudaMemcpy2DAsync(q.seed_mem.p, (size_t)q.W * 8, ctx->start_bits.data(), wn * 8, wn * 8,
                                  (size_t)q.B * q.n, cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    const auto t1 = std::chrono::steady_clock::now();
    std::vector<QCtl> ctls;
    uint32_t launches = 0;
    ClosureProfile prof;
    if (ctx->query.small_ok && ctx->opt.loop_mode == CFPQ_LOOP_DEVICE) {
        // the whole fixpoint in one CTA (state in shared memory)
        CK(ctx, launch_small_fixpoint(ctx->query.small_desc.p, 1, ctx->query.small_smem, ctx->stream));
        ctls.resize(1);
        CK(ctx, cudaMemcpyAsync(ctls.data(), ctx->query.ctl(), sizeof(QCtl), cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        launches = 1;
    } else if (int rc = run_executor(ctx, ctx->exec, &ctls, &launches, &prof)) {
        return rc;
    }
    ctx->has_result = true;
    ++ctx->result_gen;
    ctx->result_sources.clear();
    const auto t2 = std::chrono::steady_clock::now();
    const double ms = std::chrono::duration<double, std::milli>(t2 - t0).count();
    if (stats) {
        fill_stats(stats, ctls[0], ctx->query, ms);
        stats->gpu_launches = launches;
        put_profile(stats, prof);
        stats->ms_setup = std::chrono::duration<double, std::milli>(t1 - t0).count();
        stats->ms_loop = std::chrono::duration<double, std::milli>(t2 - t1).count();
    }
    const int st = status_of(ctls[0]);
    if (st) return fail(ctx, st, "iteration, round or pass cap reached before the fixpoint");
    return CFPQ_OK;
    API_CATCH(ctx)
}

int cfpq_run_sources(cfpq_ctx *ctx, const uint32_t *sources, uint32_t n_sources, cfpq_run_stats *stats) {
    if (!ctx || (n_sources && !sources)) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (ctx->has_start)
        return fail(ctx, CFPQ_ERR_STATE, "a start answer is set (cfpq_set_start); clear it for multiple-source runs");
    if (!ctx->has_graph) return fail(ctx, CFPQ_ERR_STATE, "no graph loaded");
    if (!ctx->has_rsm) return fail(ctx, CFPQ_ERR_STATE, "no RSM loaded");
    for (uint32_t i = 0; i < n_sources; ++i)
        if (sources[i] >= ctx->graph.n) return fail(ctx, CFPQ_ERR_INVALID_ARG, "source vertex out of range");
    bool reads_nt = false;
    for (const auto &tr : ctx->query.rsm.tr) reads_nt |= tr.kind == 1;
    if (reads_nt) return cfpq_run(ctx, stats);  // M3 grows with M2: every row is computed
    const auto t0 = std::chrono::steady_clock::now();
    if (int rc = set_device(ctx)) return rc;
    if (int rc = ensure_query(ctx, true)) return rc;
    {
        std::string e;
        int rc = ctx->query.compute_reach(&ctx->A, ctx->stream, sources, n_sources, &e);
        if (rc) return fail(ctx, rc, e);
    }
    const auto t1 = std::chrono::steady_clock::now();
    std::vector<QCtl> ctls;
    uint32_t launches = 0;
    ClosureProfile prof;
    if (int rc = run_executor(ctx, ctx->exec, &ctls, &launches, &prof)) return rc;
    ctx->has_result = true;
    ++ctx->result_gen;
    ctx->result_sources.assign(ctx->graph.n, 0);
    for (uint32_t i = 0; i < n_sources; ++i) ctx->result_sources[sources[i]] = 1;
    const auto t2 = std::chrono::steady_clock::now();
    if (stats) {
        fill_stats(stats, ctls[0], ctx->query, std::chrono::duration<double, std::milli>(t2 - t0).count());
        stats->gpu_launches = launches;
        put_profile(stats, prof);
        stats->ms_setup = std::chrono::duration<double, std::milli>(t1 - t0).count();
        stats->ms_loop = std::chrono::duration<double, std::milli>(t2 - t1).count();
    }
    const int st = status_of(ctls[0]);
    if (st) return fail(ctx, st, "iteration, round or pass cap reached before the fixpoint");
    return CFPQ_OK;
    API_CATCH(ctx)
}

int cfpq_set_start(cfpq_ctx *ctx, const uint64_t *bits, uint32_t n_boxes, uint32_t n_vertices) {
    if (!ctx) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (!bits) {
        ctx->has_start = false;
        ctx->start_bits.clear();
        ctx->start_bits.shrink_to_fit();
        return CFPQ_OK;
    }
    if (n_boxes == 0 || n_vertices == 0) return fail(ctx, CFPQ_ERR_INVALID_ARG, "empty start answer");
    const size_t wn = (n_vertices + 63) / 64;
    ctx->start_bits.assign(bits, bits + (size_t)n_boxes * n_vertices * wn);
    // bits past n_vertices in a row's last word are not pairs of the graph
    if (n_vertices % 64)
        for (size_t r = 0; r < (size_t)n_boxes * n_vertices; ++r)
            ctx->start_bits[r * wn + wn - 1] &= (1ull << (n_vertices % 64)) - 1ull;
    ctx->start_B = n_boxes;
    ctx->start_n = n_vertices;
    ctx->has_start = true;
    return CFPQ_OK;
    API_CATCH(ctx)
}

int cfpq_check_bounded_wait(cfpq_ctx *ctx, uint64_t limit_ns, int *timed_out) {
    if (!ctx || !timed_out || limit_ns == 0 || limit_ns > 5000000000ull) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (int rc = set_device(ctx)) return rc;
    std::string e;
    if (!ctx->counter.ensure(&ctx->A, 64, &e)) return fail(ctx, CFPQ_ERR_OUT_OF_MEMORY, e);
    int *d = ctx->counter.as<int>();
    CK(ctx, cudaMemsetAsync(d, 0xff, 4, ctx->stream));
    CK(ctx, launch_wait_selftest(limit_ns, d, ctx->stream));
    int h = -1;
    CK(ctx, cudaMemcpyAsync(&h, d, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (h != 0 && h != 1) return fail(ctx, CFPQ_ERR_CUDA, "wait self-check did not report");
    *timed_out = h;
    return CFPQ_OK;
    API_CATCH(ctx)
}

int cfpq_count_index(cfpq_ctx *ctx, uint64_t *closure_bits, uint64_t *m3_bits) {
    if (!ctx) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (!ctx->has_result) return fail(ctx, CFPQ_ERR_NOT_READY, "no result");
    if (int rc = set_device(ctx)) return rc;
    QueryDev &q = ctx->query;
    std::string e;
    if (!ctx->counter.ensure(&ctx->A, 64, &e)) return fail(ctx, CFPQ_ERR_OUT_OF_MEMORY, e);
    unsigned long long *cnt = ctx->counter.as<unsigned long long>();
    CK(ctx, cudaMemsetAsync(cnt, 0, 64, ctx->stream));
    CK(ctx, launch_popcount(q.blk_mem.as<uint64_t>(), q.blocks.size() * (size_t)q.n * q.W, cnt, ctx->stream));
    for (uint32_t b = 0; b < q.B; ++b)
        CK(ctx, launch_popcount(q.m2_ptr(b), (size_t)q.n * q.W, cnt + 1 + (b < 6 ? b : 6), ctx->stream));
    unsigned long long h[8];
    CK(ctx, cudaMemcpyAsync(h, cnt, 64, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (closure_bits) *closure_bits = h[0];
    if (m3_bits) {
        // nnz(M3) = sum over transitions s -l-> u of nnz(M2^l) (exact when no
        // two transitions join the same pair of states).
        std::vector<uint32_t> off((size_t)ctx->graph.n_term * q.n + 1);
        CK(ctx, cudaMemcpy(off.data(), ctx->graph.csr_off.p, off.size() * 4, cudaMemcpyDeviceToHost));
        std::vector<uint64_t> nnz_nt(q.B, 0);
        if (q.B > 6) {
            for (uint32_t b = 0; b < q.B; ++b) {
                CK(ctx, cudaMemsetAsync(cnt, 0, 8, ctx->stream));
                CK(ctx, launch_popcount(q.m2_ptr(b), (size_t)q.n * q.W, cnt, ctx->stream));
                unsigned long long v = 0;
                CK(ctx, cudaMemcpyAsync(&v, cnt, 8, cudaMemcpyDeviceToHost, ctx->stream));
                CK(ctx, cudaStreamSynchronize(ctx->stream));
                nnz_nt[b] = v;
            }
        } else {
            for (uint32_t b = 0; b < q.B; ++b) nnz_nt[b] = h[1 + b];
        }
        uint64_t s = 0;
        for (const auto &t : q.rsm.tr) {
            if (t.kind == 0) s += off[(size_t)(t.sym + 1) * q.n] - off[(size_t)t.sym * q.n];
            else s += nnz_nt[t.sym];
        }
        *m3_bits = s;
    }
    return CFPQ_OK;
    API_CATCH(ctx)
}

int cfpq_get_reachable_bits(cfpq_ctx *ctx, uint32_t box, uint64_t *bits) {
    if (!ctx || !bits) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (!ctx->has_result) return fail(ctx, CFPQ_ERR_NOT_READY, "no result");
    if (box >= ctx->query.B) return fail(ctx, CFPQ_ERR_INVALID_ARG, "box out of range");
    if (int rc = set_device(ctx)) return rc;
    return bits_to_host(ctx, ctx->query.m2_ptr(box), ctx->query.n, ctx->query.W, bits);
    API_CATCH(ctx)
}

int cfpq_count_reachable(cfpq_ctx *ctx, uint32_t box, uint64_t *count) {
    if (!ctx || !count) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (!ctx->has_result) return fail(ctx, CFPQ_ERR_NOT_READY, "no result");
    if (box >= ctx->query.B) return fail(ctx, CFPQ_ERR_INVALID_ARG, "box out of range");
    if (int rc = set_device(ctx)) return rc;
    std::string e;
    if (!ctx->counter.ensure(&ctx->A, 64, &e)) return fail(ctx, CFPQ_ERR_OUT_OF_MEMORY, e);
    unsigned long long *cnt = ctx->counter.as<unsigned long long>();
    CK(ctx, cudaMemsetAsync(cnt, 0, 8, ctx->stream));
    CK(ctx, launch_popcount(ctx->query.m2_ptr(box), (size_t)ctx->query.n * ctx->query.W, cnt, ctx->stream));
    unsigned long long v = 0;
    CK(ctx, cudaMemcpyAsync(&v, cnt, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    *count = v;
    return CFPQ_OK;
    API_CATCH(ctx)
}

int cfpq_get_reachable(cfpq_ctx *ctx, uint32_t box, uint32_t *src, uint32_t *dst, size_t cap, size_t *count) {
    if (!ctx || !count) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (!ctx->has_result) return fail(ctx, CFPQ_ERR_NOT_READY, "no result");
    if (box >= ctx->query.B) return fail(ctx, CFPQ_ERR_INVALID_ARG, "box out of range");
    const uint32_t n = ctx->query.n;
    const size_t wn = (n + 63) / 64;
    std::vector<uint64_t> bits((size_t)n * wn);
    if (int rc = cfpq_get_reachable_bits(ctx, box, bits.data())) return rc;
    size_t total = 0;
    for (uint64_t w : bits) total += (size_t)__builtin_popcountll(w);
    *count = total;
    if (!src && !dst && cap == 0) return CFPQ_OK;
    if (!src || !dst || cap < total) return fail(ctx, CFPQ_ERR_BUFFER_TOO_SMALL, "pair buffers too small");
    size_t k = 0;
    for (uint32_t x = 0; x < n; ++x)
        for (size_t w = 0; w < wn; ++w) {
            uint64_t b = bits[(size_t)x * wn + w];
            while (b) {
                const uint32_t y = (uint32_t)(w * 64 + (uint64_t)__builtin_ctzll(b));
                b &= b - 1;
                src[k] = x;
                dst[k] = y;
                ++k;
            }
        }
    return CFPQ_OK;
    API_CATCH(ctx)
}

int cfpq_get_closure_rows(cfpq_ctx *ctx, uint32_t n_rows, const uint32_t *row_state, const uint32_t *row_vertex,
                          uint64_t *out) {
    if (!ctx || (n_rows && (!row_state || !row_vertex || !out))) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (!ctx->has_result) return fail(ctx, CFPQ_ERR_NOT_READY, "no result");
    if (int rc = set_device(ctx)) return rc;
    QueryDev &q = ctx->query;
    const uint32_t n = q.n, Q = q.Q, W = q.W;
    const size_t wN = ((size_t)Q * n + 63) / 64;
    for (uint32_t k = 0; k < n_rows; ++k)
        if (row_state[k] >= Q || row_vertex[k] >= n) return fail(ctx, CFPQ_ERR_INVALID_ARG, "row out of range");
    const uint32_t chunk = 4096;
    std::vector<const uint64_t *> ptrs;
    std::vector<uint32_t> rows;
    std::vector<uint64_t> host;
    std::string e;
    for (uint32_t k0 = 0; k0 < n_rows; k0 += chunk / Q + 1) {
        const uint32_t k1 = std::min(n_rows, k0 + chunk / Q + 1);
        ptrs.clear();
        rows.clear();
        for (uint32_t k = k0; k < k1; ++k)
            for (uint32_t t = 0; t < Q; ++t) {
                const int32_t b = q.blk_of[(size_t)row_state[k] * Q + t];
                ptrs.push_back(b >= 0 ? q.blk_ptr((uint32_t)b) : nullptr);
                rows.push_back(row_vertex[k]);
            }
        const uint32_t nj = (uint32_t)ptrs.size();
        if (!ctx->rows_ptrs.ensure(&ctx->A, nj * sizeof(void *), &e) || !ctx->rows_idx.ensure(&ctx->A, nj * 4, &e) ||
            !ctx->rows_out.ensure(&ctx->A, (size_t)nj * W * 8, &e))
            return fail(ctx, CFPQ_ERR_OUT_OF_MEMORY, e);
        CK(ctx, cudaMemcpyAsync(ctx->rows_ptrs.p, ptrs.data(), nj * sizeof(void *), cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, cudaMemcpyAsync(ctx->rows_idx.p, rows.data(), nj * 4, cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, launch_copy_rows(ctx->rows_ptrs.as<const uint64_t *>(), ctx->rows_idx.as<uint32_t>(), nj, W,
                                 ctx->rows_out.as<uint64_t>(), ctx->stream));
        host.resize((size_t)nj * W);
        CK(ctx, cudaMemcpyAsync(host.data(), ctx->rows_out.p, host.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        // Remap block-local columns (t, y) to the paper's index t * n + y.
        for (uint32_t k = k0; k < k1; ++k) {
            uint64_t *o = out + (size_t)k * wN;
            memset(o, 0, wN * 8);
            for (uint32_t t = 0; t < Q; ++t) {
                const uint64_t *src = host.data() + ((size_t)(k - k0) * Q + t) * W;
                for (uint32_t w = 0; w < W; ++w) {
                    uint64_t b = src[w];
                    while (b) {
                        const uint64_t y = w * 64 + (uint64_t)__builtin_ctzll(b);
                        b &= b - 1;
                        const uint64_t col = (uint64_t)t * n + y;
                        o[col >> 6] |= 1ull << (col & 63);
                    }
                }
            }
        }
    }
    return CFPQ_OK;
    API_CATCH(ctx)
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Path extraction (Sec. 3.2, Listing 2): enumeration in cfpq_paths_host.h,
// backward layers on the device (cfpq_paths.cu).
// ---------------------------------------------------------------------------
using PathCtx = cfpq::PathEnum<cfpq::HostRSM>;

extern "C" int cfpq_extract_paths(cfpq_ctx *ctx, uint32_t box, uint32_t vs, uint32_t vf, uint32_t max_len,
                                  size_t max_paths, uint32_t *edge_buf, size_t edge_cap, size_t *path_offsets,
                                  size_t *n_paths, int *truncated) {
    if (!ctx || !n_paths || !path_offsets) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (!ctx->has_result) return fail(ctx, CFPQ_ERR_NOT_READY, "no result");
    QueryDev &q = ctx->query;
    if (box >= q.B || vs >= q.n || vf >= q.n) return fail(ctx, CFPQ_ERR_INVALID_ARG, "box or vertex out of range");
    if (!ctx->result_sources.empty() && !ctx->result_sources[vs])
        return fail(ctx, CFPQ_ERR_INVALID_ARG, "vs was not a source of the last multiple-source run");
    if (int rc = set_device(ctx)) return rc;
    std::string e;
    // The host copies, the device tables and the memo of path sets stay valid
    // until the next result (run, graph or RSM change).
    if (!ctx->penum || ctx->penum_gen != ctx->result_gen) {
        ctx->penum.reset(new PathCtx());
        PathCtx &P = *ctx->penum;
        P.r = &q.rsm;
        P.n = q.n;
        P.wn = (q.n + 63) / 64;
        // host copies: unique terminal edges and M2 of every box
        const GraphDev &g = ctx->graph;
        std::vector<uint32_t> off((size_t)g.n_term * g.n + 1), col(std::max<size_t>(g.m_unique, 1));
        CK(ctx, cudaMemcpy(off.data(), g.csr_off.p, off.size() * 4, cudaMemcpyDeviceToHost));
        if (g.m_unique) CK(ctx, cudaMemcpy(col.data(), g.csr_col.p, g.m_unique * 4, cudaMemcpyDeviceToHost));
        std::vector<std::tuple<uint32_t, uint32_t, uint32_t>> tri;
        for (uint32_t l = 0; l < g.n_term; ++l)
            for (uint32_t x = 0; x < g.n; ++x)
                for (uint32_t k = off[(size_t)l * g.n + x]; k < off[(size_t)l * g.n + x + 1]; ++k)
                    tri.emplace_back(x, l, col[k]);
        std::sort(tri.begin(), tri.end());
        tri.erase(std::unique(tri.begin(), tri.end()), tri.end());
        P.eoff.assign(g.n + 1, 0);
        for (auto &t : tri) {
            P.es.push_back(std::get<0>(t));
            P.el.push_back(std::get<1>(t));
            P.ed.push_back(std::get<2>(t));
            P.eoff[std::get<0>(t) + 1]++;
        }
        for (uint32_t v = 0; v < g.n; ++v) P.eoff[v + 1] += P.eoff[v];
        // reverse terminal CSR over (label, target vertex) for the backward layers
        std::vector<uint32_t> roff((size_t)g.n_term * g.n + 1, 0), rcol(tri.size());
        for (auto &t : tri) ++roff[(size_t)std::get<1>(t) * g.n + std::get<2>(t) + 1];
        for (size_t i = 1; i < roff.size(); ++i) roff[i] += roff[i - 1];
        {
            std::vector<uint32_t> fill(roff.begin(), roff.end() - 1);
            for (auto &t : tri) rcol[fill[(size_t)std::get<1>(t) * g.n + std::get<2>(t)]++] = std::get<0>(t);
        }
        if (int rc = ctx->paths.prepare(&ctx->A, ctx->stream, q, g.n_term, roff, rcol, &e)) {
            ctx->penum.reset();
            return fail(ctx, rc, e);
        }
        P.Qd = q.Q;
        P.Wd = q.W;
        P.m2.resize(q.B);
        for (uint32_t b = 0; b < q.B; ++b) {
            P.m2[b].resize((size_t)q.n * P.wn);
            if (int rc = bits_to_host(ctx, q.m2_ptr(b), q.n, q.W, P.m2[b].data())) {
                ctx->penum.reset();
                return rc;
            }
        }
        ctx->penum_gen = ctx->result_gen;
    }
    PathCtx &P = *ctx->penum;
    // layers of a larger bound contain those of a smaller one
    if (max_len > P.Lmax) {
        P.Lmax = max_len;
        P.lay.clear();
        P.wanted.clear();
        P.fdist.clear();
    }
    if (P.stored > P.cap / 2) {
        P.memo.clear();
        P.readers.clear();
        P.stored = 0;
    }
    P.over = false;
    P.dev_rc = 0;
    const uint32_t L = P.Lmax;
    P.fetch = [ctx, &q, &e, L](const std::vector<PathCtx::Target> &ts, std::vector<std::vector<uint64_t>> *out) {
        return ctx->paths.layers(&ctx->A, ctx->stream, q.rsm, ts, L, out, &e);
    };
    // Paths in order of length, then lexicographic (edge ids follow the triple order).
    std::vector<std::vector<uint32_t>> result;
    bool trunc = false;
    const uint64_t *root = P.m2[box].data() + (size_t)vs * P.wn;
    const bool reachable = (root[vf >> 6] >> (vf & 63)) & 1;
    // until the fixpoints below complete, the cached memo is not reusable
    // (an exception leaves it marked stale)
    ctx->penum_gen = ~0ull;
    if (reachable) {
        for (uint32_t len = 0; len <= max_len && !trunc; ++len) {
            P.get(box, vs, vf, len);
            P.solve();
            if (P.dev_rc || P.over) {
                // an interrupted fixpoint leaves partial sets: drop them
                const int rc = P.dev_rc;
                ctx->penum.reset();
                if (rc) return fail(ctx, rc, "backward layers: " + e);
                return fail(ctx, CFPQ_ERR_UNSUPPORTED, "path enumeration exceeded its work cap");
            }
            const auto &S = P.memo[std::make_tuple(box, vs, vf, len)];
            for (const auto &p : S) {
                if (result.size() == max_paths) { trunc = true; break; }
                result.push_back(p);
            }
        }
    }
    ctx->penum_gen = ctx->result_gen;
    size_t need = 0;
    for (auto &p : result) need += p.size();
    *n_paths = result.size();
    if (truncated) *truncated = trunc ? 1 : 0;
    if (need > edge_cap || (need && !edge_buf)) return fail(ctx, CFPQ_ERR_BUFFER_TOO_SMALL, "edge buffer too small");
    size_t k = 0;
    path_offsets[0] = 0;
    for (size_t i = 0; i < result.size(); ++i) {
        for (uint32_t e : result[i]) {
            edge_buf[3 * k] = P.es[e];
            edge_buf[3 * k + 1] = P.el[e];
            edge_buf[3 * k + 2] = P.ed[e];
            ++k;
        }
        path_offsets[i + 1] = k;
    }
    return CFPQ_OK;
    API_CATCH(ctx)
}

// ---------------------------------------------------------------------------
// Column-sharded index creation (one query over several ranks).
// ---------------------------------------------------------------------------
namespace {

// Passes of the executor driven from the host until no query runs (done or
// paused for the exchange of a sharded iteration).
int host_passes(cfpq_ctx *ctx, Executor &ex) {
    int running = 1;
    while (running) {
        if (ex.enqueue_pass(ctx->stream, 0, 0, ex.running.as<int>(), nullptr))
            return fail(ctx, CFPQ_ERR_CUDA, "pass launch failed");
        CK(ctx, cudaMemcpyAsync(&running, ex.running.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return CFPQ_OK;
}

}  // namespace

extern "C" int cfpq_shard_begin(cfpq_ctx *ctx, uint32_t col0, uint32_t col1) {
    if (!ctx) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (!ctx->has_graph || !ctx->has_rsm) return fail(ctx, CFPQ_ERR_STATE, "load a graph and an RSM first");
    if (ctx->has_start) return fail(ctx, CFPQ_ERR_STATE, "a start answer is set (cfpq_set_start); clear it first");
    const uint32_t n_pad = ctx->graph.n_pad;
    if (col0 > col1 || col1 > n_pad || col0 % 256u != 0u || (col1 % 256u != 0u && col1 != n_pad))
        return fail(ctx, CFPQ_ERR_INVALID_ARG,
                    "columns must satisfy col0 <= col1 <= n_pad (n rounded up to 128), col0 a multiple of 256 and "
                    "col1 a multiple of 256 or n_pad");
    if (int rc = set_device(ctx)) return rc;
    if (int rc = ensure_query(ctx)) return rc;
    QueryDev &q = ctx->query;
    std::string e;
    if (!ctx->shard_cnt.ensure(&ctx->A, (size_t)q.B * 16, &e)) return fail(ctx, CFPQ_ERR_OUT_OF_MEMORY, e);
    ctx->has_result = false;
    ++ctx->result_gen;
    ctx->result_sources.clear();
    if (ctx->exec.enqueue_prologue(ctx->stream, ctx->opt.max_iterations, ctx->opt.max_rounds, kDefaultPassCap))
        return fail(ctx, CFPQ_ERR_CUDA, "prologue launch failed");
    CK(ctx, launch_shard_setup(q.ctl(), col0 / 128u, col1 / 128u, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->shard_on = true;
    ctx->shard_c0 = col0;
    ctx->shard_c1 = col1;
    return CFPQ_OK;
    API_CATCH(ctx)
}

extern "C" int cfpq_shard_step(cfpq_ctx *ctx, uint64_t *d_slice, uint64_t *new_edges) {
    if (!ctx) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (!ctx->shard_on) return fail(ctx, CFPQ_ERR_STATE, "no sharded run (cfpq_shard_begin)");
    const uint32_t wl = (ctx->shard_c1 - ctx->shard_c0) / 64u;
    if (wl && !d_slice) return fail(ctx, CFPQ_ERR_INVALID_ARG, "d_slice is NULL");
    if (int rc = set_device(ctx)) return rc;
    QueryDev &q = ctx->query;
    if (int rc = host_passes(ctx, ctx->exec)) return rc;
    std::vector<QCtl> ctls;
    int tc_error = 0;
    if (ctx->exec.read_ctls(ctx->stream, &ctls, &tc_error)) return fail(ctx, CFPQ_ERR_CUDA, "reading loop state failed");
    if (tc_error)
        return fail(ctx, CFPQ_ERR_TIMEOUT, "a tile-product kernel gave up (bounded wait on its MMAs or on a counter)");
    const QCtl &c = ctls[0];
    if (c.phase == kPhasePause) {
        CK(ctx, launch_shard_export(q.a2_mem.as<uint64_t>(), q.a2it_mem.as<uint32_t>(), q.n, q.W, q.B,
                                    ctx->shard_c0 / 64u, ctx->shard_c1 / 64u, c.iter, d_slice, ctx->stream));
        if (new_edges) *new_edges = c.shard_new;
    } else {
        if (wl) CK(ctx, cudaMemsetAsync(d_slice, 0, (size_t)q.B * q.n * wl * 8, ctx->stream));
        if (new_edges) *new_edges = 0;
    }
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (c.phase == kPhaseDone && c.status != kStatusOk)
        return fail(ctx, CFPQ_ERR_TIMEOUT, "iteration, round or pass cap reached before the fixpoint");
    return CFPQ_OK;
    API_CATCH(ctx)
}

extern "C" int cfpq_shard_apply(cfpq_ctx *ctx, const uint64_t *d_full, int *done) {
    if (!ctx || !d_full || !done) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (!ctx->shard_on) return fail(ctx, CFPQ_ERR_STATE, "no sharded run (cfpq_shard_begin)");
    if (int rc = set_device(ctx)) return rc;
    QueryDev &q = ctx->query;
    std::vector<QCtl> ctls;
    if (ctx->exec.read_ctls(ctx->stream, &ctls, nullptr)) return fail(ctx, CFPQ_ERR_CUDA, "reading loop state failed");
    if (ctls[0].phase == kPhasePause) {
        CK(ctx, launch_shard_apply(d_full, q.m2_mem.as<uint64_t>(), q.a2_mem.as<uint64_t>(),
                                   q.a2it_mem.as<uint32_t>(), q.n, q.W, q.B, ctls[0].iter,
                                   ctx->shard_cnt.as<unsigned long long>(), q.ctl(), q.boxit_mem.as<uint32_t>(),
                                   ctx->stream));
        if (ctx->exec.enqueue_lists(ctx->stream)) return fail(ctx, CFPQ_ERR_CUDA, "list launch failed");
        if (ctx->exec.read_ctls(ctx->stream, &ctls, nullptr))
            return fail(ctx, CFPQ_ERR_CUDA, "reading loop state failed");
    }
    *done = ctls[0].phase != kPhaseRun ? 1 : 0;
    if (*done) {
        ctx->shard_on = false;
        ctx->has_result = true;
        ++ctx->result_gen;
        if (ctls[0].status != kStatusOk)
            return fail(ctx, CFPQ_ERR_TIMEOUT, "iteration, round or pass cap reached before the fixpoint");
    }
    return CFPQ_OK;
    API_CATCH(ctx)
}

extern "C" int cfpq_shard_stats(cfpq_ctx *ctx, cfpq_run_stats *stats) {
    if (!ctx || !stats) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (int rc = set_device(ctx)) return rc;
    std::vector<QCtl> ctls;
    if (!ctx->query.prepared) return fail(ctx, CFPQ_ERR_NOT_READY, "no run");
    if (ctx->exec.read_ctls(ctx->stream, &ctls, nullptr)) return fail(ctx, CFPQ_ERR_CUDA, "reading loop state failed");
    fill_stats(stats, ctls[0], ctx->query, 0.0);
    return CFPQ_OK;
    API_CATCH(ctx)
}

// ---------------------------------------------------------------------------
// Batched index creation.
// ---------------------------------------------------------------------------
extern "C" int cfpq_batch_run(cfpq_ctx *ctx, uint32_t n_queries, const cfpq_query *queries,
                              cfpq_run_stats *per_query_stats, cfpq_run_stats *total_stats) {
    if (!ctx || (n_queries && !queries)) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    const auto t0 = std::chrono::steady_clock::now();
    if (int rc = set_device(ctx)) return rc;
    ctx->has_batch = false;
    ctx->bexec.qs.clear();
    ctx->bexec.drop_graph();
    ctx->bqueries.clear();
    ctx->bgraphs.clear();
    // the graphs and queries of the batch take their buffers from the slab
    // (rewound, its chunks kept from the previous batch)
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    bind_slab(&ctx->bslab, &ctx->A, ctx->stream);
    ctx->bslab.reset();
    std::string e;
    // one tile kernel for the batch: tuned for its largest graph
    uint32_t max_n = 0;
    for (uint32_t i = 0; i < n_queries; ++i) max_n = std::max(max_n, queries[i].n_vertices);
    if (max_n) {
        QueryDev probe_q;
        set_tiles(probe_q, ctx->opt, ctx->stream, max_n);  // (runs the probe first when it may pay)
        if (int rc = set_device(ctx)) return rc;
    }
    for (uint32_t i = 0; i < n_queries; ++i) {
        const cfpq_query &qq = queries[i];
        std::unique_ptr<GraphDev> g(new GraphDev());
        int rc = stage_graph(g.get(), &ctx->bslab.A, ctx->stream, qq.n_vertices, qq.n_terminals, qq.n_edges, qq.src,
                             qq.label, qq.dst, false, &e);
        if (rc) return fail(ctx, rc, "query " + std::to_string(i) + ": " + e);
        std::unique_ptr<QueryDev> q(new QueryDev());
        q->closure_mode = ctx->opt.closure_mode;
        set_tiles(*q, ctx->opt, ctx->stream, max_n);
        q->gather_slices = ctx->opt.gather_slices;
        rc = copy_rsm(qq.rsm, &q->rsm, &e);
        if (rc) return fail(ctx, rc, "query " + std::to_string(i) + ": " + e);
        q->g = g.get();
        rc = q->prepare(&ctx->bslab.A, &e);
        if (rc) return fail(ctx, rc, "query " + std::to_string(i) + ": " + e);
        ctx->bgraphs.push_back(std::move(g));
        ctx->bqueries.push_back(std::move(q));
    }
    for (auto &q : ctx->bqueries) ctx->bexec.qs.push_back(q.get());
    int rc = ctx->bexec.assemble(&ctx->A, ctx->stream, &e);
    if (rc) return fail(ctx, rc, e);
    const auto t1 = std::chrono::steady_clock::now();
    std::vector<QCtl> ctls;
    uint32_t launches = 0;
    ClosureProfile prof;
    if ((rc = run_executor(ctx, ctx->bexec, &ctls, &launches, &prof))) return rc;
    ctx->has_batch = true;
    const auto t2 = std::chrono::steady_clock::now();
    const double ms = std::chrono::duration<double, std::milli>(t2 - t0).count();
    int worst = CFPQ_OK;
    cfpq_run_stats tot;
    memset(&tot, 0, sizeof(tot));
    for (uint32_t i = 0; i < n_queries; ++i) {
        cfpq_run_stats s;
        fill_stats(&s, ctls[i], *ctx->bqueries[i], ms);
        if (per_query_stats) per_query_stats[i] = s;
        tot.iterations = std::max(tot.iterations, s.iterations);
        tot.rounds = std::max(tot.rounds, s.rounds);
        tot.edges_added += s.edges_added;
        tot.row_ors += s.row_ors;
        tot.tile_mmas += s.tile_mmas;
        tot.tile_kstages += s.tile_kstages;
        tot.tile_operand_bytes += s.tile_operand_bytes;
        tot.closure_blocks += s.closure_blocks;
        tot.device_bytes += s.device_bytes;
        if (status_of(ctls[i])) worst = status_of(ctls[i]);
    }
    tot.ms_total = ms;
    tot.ms_closure = prof.ms_closure;  // profile = 1: the batch's closure passes by kernel group
    tot.ms_gather = prof.ms_gather;
    tot.ms_tile_operands = prof.ms_operands;
    tot.ms_tile_products = prof.ms_products;
    tot.closure_launches = prof.closure_launches;
    tot.gather_launches = prof.gather_launches;
    tot.tile_launches = prof.tile_launches;
    tot.ms_setup = std::chrono::duration<double, std::milli>(t1 - t0).count();
    tot.ms_loop = std::chrono::duration<double, std::milli>(t2 - t1).count();
    tot.gpu_launches = launches;
    tot.status = worst ? (uint32_t)(-worst) : 0;
    if (total_stats) *total_stats = tot;
    if (worst) return fail(ctx, worst, "a query reached an iteration, round or pass cap");
    return CFPQ_OK;
    API_CATCH(ctx)
}

extern "C" int cfpq_batch_get_reachable_bits(cfpq_ctx *ctx, uint32_t qi, uint32_t box, uint64_t *bits) {
    if (!ctx || !bits) return CFPQ_ERR_INVALID_ARG;
    API_TRY
    if (!ctx->has_batch) return fail(ctx, CFPQ_ERR_NOT_READY, "no batch result");
    if (qi >= ctx->bqueries.size()) return fail(ctx, CFPQ_ERR_INVALID_ARG, "query index out of range");
    QueryDev &q = *ctx->bqueries[qi];
    if (box >= q.B) return fail(ctx, CFPQ_ERR_INVALID_ARG, "box out of range");
    if (int rc = set_device(ctx)) return rc;
    return bits_to_host(ctx, q.m2_ptr(box), q.n, q.W, bits);
    API_CATCH(ctx)
}
