// cfpq_tune.cu -- autotuner of the closure's tile products.
//
// The closure of Listing 1 (Sec. 3.1) can compute a product of a label
// matrix with closure rows either as bit-packed row ORs (the gather) or as
// 0/1 tensor-core tiles, in one of four tile kernels (FP8 256 x 256, FP8
// 128 x 256, E2M1 256 x 192 with 32-element UE8M0 or 16-element UE4M3
// scales).  Which is faster depends on the device, so this file measures
// it: once per device and process it runs a probe query through the
// library's own API -- Dyck-4 on a seeded graph of 8192 vertices with
// Zipf(2.1) out-degrees (mean about 3), 8 labels -- with the bit-packed
// closure and with every
// tile kernel, in the host-driven loop with per-kernel CUDA events, times
// reads of an L2-sized and an HBM-sized buffer, and keeps
//   - the rate of each tile kernel (0/1 multiply-adds per second over its
//     launches) and of the gather (source-row bytes ORed per second; the
//     probe's 8 MiB closure blocks stay in L2, so for blocks beyond half the
//     L2 the rate is scaled by the ratio of the device's read bandwidth
//     from HBM to that from L2, both measured);
//   - the fastest tile kernel, AUTO's default (the built-in FP4 one unless
//     another is 3% faster);
//   - per kernel and query size, the ratio of the cost model that decides
//     per pass whether an iteration's new edges run as tiles
//     (new_tiles_pay): a new edge costs the gather one row of n/8 bytes, a
//     compacted tile product of M x K 2n multiply-adds per (row, column), so
//     tiles win while M * K < e * tile_rate / (16 * gather_rate).
// Every choice leaves the answer unchanged (the products are exact).
#include <chrono>
#include <cmath>
#include <mutex>
#include <vector>

#include "cfpq_ctx.cuh"

namespace cfpq {

namespace {

std::recursive_mutex g_tune_mu;  // recursive: the probe's own contexts read the table
Tuning g_tune[64];
bool g_tune_tried[64];

uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Dyck-4 as a one-box RSM with 11 states: q0 = 0, p = 1, F = 2, x_i = 3 + i,
// y_i = 7 + i; q0 -S-> p -S-> F, q0 -o_i-> x_i -c_i-> F, x_i -S-> y_i -c_i-> F
// (o_i = terminal i, c_i = terminal 4 + i).
struct ProbeRsm {
    std::vector<uint32_t> box_start{0}, state_box = std::vector<uint32_t>(11, 0), from, kind, sym, to;
    std::vector<uint8_t> fin = std::vector<uint8_t>(11, 0);
    cfpq_rsm r;
    ProbeRsm() {
        fin[2] = 1;
        auto add = [&](uint32_t f, uint32_t k, uint32_t s, uint32_t t) {
            from.push_back(f);
            kind.push_back(k);
            sym.push_back(s);
            to.push_back(t);
        };
        add(0, 1, 0, 1);
        add(1, 1, 0, 2);
        for (uint32_t i = 0; i < 4; ++i) {
            add(0, 0, i, 3 + i);
            add(3 + i, 0, 4 + i, 2);
            add(3 + i, 1, 0, 7 + i);
            add(7 + i, 0, 4 + i, 2);
        }
        r.n_states = 11;
        r.n_boxes = 1;
        r.start_box = 0;
        r.n_trans = (uint32_t)from.size();
        r.box_start = box_start.data();
        r.state_box = state_box.data();
        r.state_final = fin.data();
        r.tr_from = from.data();
        r.tr_kind = kind.data();
        r.tr_sym = sym.data();
        r.tr_to = to.data();
    }
};

constexpr uint32_t kProbeN = 8192, kProbeMaxDeg = 192, kProbeLabels = 8;
constexpr double kTileFlopPerKstage = 2.0 * 128 * 256 * 128;

// One probe run (the second of two: the first pays for set-up and module
// loading); returns a CFPQ status.  profiled: the host-driven loop with
// per-kernel events (the kernel groups' rates); else the device loop, and
// *ms gets the host time of the second run.
int probe_run(const cfpq_options &like, cudaStream_t st, uint32_t mode, uint32_t fmt, uint32_t ratio,
              bool profiled, const ProbeRsm &pr, const std::vector<uint32_t> &src,
              const std::vector<uint32_t> &lbl, const std::vector<uint32_t> &dst, cfpq_run_stats *out,
              double *ms = nullptr) {
    cfpq_options o;
    cfpq_default_options(&o);
    o.device = like.device;
    o.alloc = like.alloc;
    o.free = like.free;
    o.alloc_user = like.alloc_user;
    o.closure_mode = mode;
    o.tile_format = fmt;
    o.tile_ratio = ratio;
    o.loop_mode = profiled ? CFPQ_LOOP_HOST : CFPQ_LOOP_DEVICE;
    o.profile = profiled ? 1u : 0u;
    o.no_single_cta = 1;
    o.no_autotune = 1;
    cfpq_ctx *c = nullptr;
    int rc = cfpq_create(&c, &o, st);
    if (rc) return rc;
    rc = cfpq_load_graph(c, kProbeN, kProbeLabels, src.size(), src.data(), lbl.data(), dst.data());
    if (!rc) rc = cfpq_load_rsm(c, &pr.r);
    if (!rc) rc = cfpq_run(c, out);
    const auto t0 = std::chrono::steady_clock::now();
    if (!rc) rc = cfpq_run(c, out);  // (returns after reading the loop's final state)
    if (ms) *ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    cfpq_destroy(c);
    return rc;
}

// Read bandwidth: every thread XORs 16-byte words of the buffer (L2-cached
// loads, no L1), `reps` passes; the result only decides whether the one
// word it may write is written, so no load is dropped.
__global__ void k_read_bw(const uint4 *__restrict__ p, size_t n16, uint32_t reps, unsigned int *sink) {
    uint32_t acc = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (uint32_t r = 0; r < reps; ++r)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
            const uint4 v = __ldcg(p + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1u);
}

// Device read bandwidth (GB/s) over a buffer of `bytes`, read `reps` times
// per launch, best of 3 launches after an untimed one; 0 on error.
double read_gbs(Allocator &A, cudaStream_t st, int dev, size_t bytes, uint32_t reps) {
    std::string err;
    void *a = A.get(bytes + 256, &err);
    double best = 0;
    int sms = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (a && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0 &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
        cudaMemsetAsync(a, 0, bytes + 256, st) == cudaSuccess) {
        const uint4 *p = static_cast<const uint4 *>(a);
        unsigned int *sink = reinterpret_cast<unsigned int *>(static_cast<char *>(a) + bytes);
        const size_t n16 = bytes / 16;
        k_read_bw<<<(unsigned)sms * 4u, 512, 0, st>>>(p, n16, 1u, sink);
        for (int r = 0; r < 3; ++r) {
            cudaEventRecord(e0, st);
            k_read_bw<<<(unsigned)sms * 4u, 512, 0, st>>>(p, n16, reps, sink);
            cudaEventRecord(e1, st);
            float ms = 0;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) break;
            if (ms > 0) best = std::max(best, (double)bytes * reps / (ms * 1e6));
        }
    }
    cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (a) A.put(a, bytes + 256);
    cudaGetLastError();
    return best;
}

uint32_t ratio_for(double tflops, double gather_gbs) {
    // M * K < e * rate_tile / (16 * rate_gather): TFLOP/s over GB/s is 1e3
    const double r = tflops * 1e3 / (16.0 * gather_gbs);
    return (uint32_t)std::min(4096.0, std::max(8.0, std::floor(r + 0.5)));
}

Tuning run_probe(const cfpq_options &like, cudaStream_t st) {
    Tuning t;
    const auto t0 = std::chrono::steady_clock::now();
    {
        Allocator A;
        A.alloc = like.alloc;
        A.free = like.free;
        A.user = like.alloc_user;
        A.stream = st;
        int l2 = 0;
        if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, like.device) == cudaSuccess && l2 > 0)
            t.l2_bytes = (uint64_t)l2;
        t.read_l2_gbs = read_gbs(A, st, like.device, (size_t)24 << 20, 20);
        t.read_hbm_gbs = read_gbs(A, st, like.device, (size_t)2 << 30, 1);
    }
    ProbeRsm pr;
    std::vector<uint32_t> src, lbl, dst;
    uint64_t seed = 0x2103146880000001ull;
    // out-degree Zipf(2.1) on 1..192 (mean about 3), targets and labels uniform
    double cdf[kProbeMaxDeg], acc = 0;
    for (uint32_t k = 1; k <= kProbeMaxDeg; ++k) cdf[k - 1] = (acc += std::pow((double)k, -2.1));
    for (uint32_t v = 0; v < kProbeN; ++v) {
        const double u = (double)(splitmix64(seed) >> 11) * 0x1.0p-53 * acc;
        uint32_t deg = 1;
        while (deg < kProbeMaxDeg && cdf[deg - 1] < u) ++deg;
        for (uint32_t k = 0; k < deg; ++k) {
            src.push_back(v);
            dst.push_back((uint32_t)(splitmix64(seed) % kProbeN));
            lbl.push_back((uint32_t)(splitmix64(seed) % kProbeLabels));
        }
    }
    cfpq_run_stats s;
    int rc = probe_run(like, st, CFPQ_CLOSURE_BITPACKED, CFPQ_TILES_DEFAULT, 0, true, pr, src, lbl, dst, &s);
    if (!rc && s.ms_gather > 0) t.gather_gbs = (double)s.row_ors * (double)s.row_bytes / (s.ms_gather * 1e6);
    const uint32_t fmts[kTileKinds] = {CFPQ_TILES_FP8, CFPQ_TILES_FP8_128, CFPQ_TILES_FP4, CFPQ_TILES_NVFP4};
    for (uint32_t k = 0; k < kTileKinds && !rc; ++k) {
        const uint32_t mode = tile_kind_fp4(k) ? CFPQ_CLOSURE_TC_FP4 : CFPQ_CLOSURE_TC_FP8;
        rc = probe_run(like, st, mode, fmts[k], 0, true, pr, src, lbl, dst, &s);
        if (!rc && s.ms_tile_products > 0)
            t.tflops[k] = (double)s.tile_kstages * kTileFlopPerKstage / (s.ms_tile_products * 1e9);
    }
    t.probe_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    t.status = rc;
    if (rc || t.gather_gbs <= 0) {  // keep the measurements, not the choices
        t.tuned = false;
        t.kind = kTileFp4Pair;
        t.status = rc ? rc : -1;
        return t;
    }
    // the fastest kernel; the built-in one unless another beats it by 3%
    uint32_t best = kTileFp4Pair;
    for (uint32_t k = 0; k < kTileKinds; ++k)
        if (t.tflops[k] > 1.03 * t.tflops[best]) best = k;
    t.kind = best;
    // The cost model's ratio, searched: the rate formula's value and 1/2,
    // 2, 4, 8 times it, each timed on the whole probe query in AUTO with
    // that kernel (the formula's rates average over all the gather's work,
    // while the rows the new-edge tiles replace are the hub rows it handles
    // worst).  The fastest is kept for L2-resident queries.
    const uint32_t base = ratio_for(t.tflops[best], t.gather_gbs);
    double best_ms = 0;
    for (uint32_t f = 0; f < 5 && !rc; ++f) {
        const uint32_t r = std::min<uint32_t>(4096u, std::max<uint32_t>(8u, f == 0 ? base / 2u : base << (f - 1)));
        double ms = 0;
        rc = probe_run(like, st, CFPQ_CLOSURE_AUTO, fmts[best], r, false, pr, src, lbl, dst, &s, &ms);
        if (!rc && (best_ms == 0 || ms < best_ms)) {
            best_ms = ms;
            t.ratio_l2 = r;
        }
    }
    t.probe_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rc) {
        t.status = rc;
        t.kind = kTileFp4Pair;
        return t;
    }
    t.tuned = true;
    return t;
}


}  // namespace

Tuning device_tuning(const cfpq_options &like, cudaStream_t st, bool run, bool force) {
    const int dev = like.device;
    if (dev < 0 || dev >= 64) return Tuning{};
    std::lock_guard<std::recursive_mutex> lk(g_tune_mu);
    if ((run && !g_tune_tried[dev]) || force) {
        g_tune_tried[dev] = true;  // before the probe: its own contexts never probe
        g_tune[dev] = run_probe(like, st);
        cudaSetDevice(dev);
    }
    return g_tune[dev];
}

uint32_t tile_kind_of(uint32_t mode, uint32_t fmt, const Tuning &t) {
    if (mode == CFPQ_CLOSURE_TC_FP4) return fmt == CFPQ_TILES_NVFP4 ? kTileFp4NvPair : kTileFp4Pair;
    if (fmt == CFPQ_TILES_FP8_128) return kTileFp8Single;
    if (mode == CFPQ_CLOSURE_TC_FP8 || fmt == CFPQ_TILES_FP8) return kTileFp8Pair;
    if (fmt == CFPQ_TILES_FP4) return kTileFp4Pair;
    if (fmt == CFPQ_TILES_NVFP4) return kTileFp4NvPair;
    return t.kind;  // AUTO, the default format: the tuned kernel (built-in: FP4)
}

uint32_t tile_ratio_of(uint32_t kind, const Tuning &t, uint32_t n) {
    const uint64_t block = (uint64_t)n * (((uint64_t)n + 127u) & ~127ull) / 8u;
    if (t.tuned && kind == t.kind && t.ratio_l2) {
        // the searched ratio, for rows from HBM scaled like the gather's rate
        const double r = (double)t.ratio_l2 / t.memory_scale(block);
        return (uint32_t)std::min(4096.0, std::floor(r + 0.5));
    }
    if (t.tuned && kind < kTileKinds && t.tflops[kind] > 0) return ratio_for(t.tflops[kind], t.gather_rate(block));
    return (uint32_t)(tile_kind_fp4(kind) ? kTileEdgeRatioFp4 : kTileEdgeRatio);
}

}  // namespace cfpq

extern "C" int cfpq_tune(cfpq_ctx *ctx, int force, cfpq_tuning *out) {
    using namespace cfpq;
    if (!ctx || !out || out->struct_size != sizeof(cfpq_tuning)) return CFPQ_ERR_INVALID_ARG;
    try {
        if (cudaSetDevice(ctx->opt.device) != cudaSuccess) return CFPQ_ERR_CUDA;
        const Tuning t = device_tuning(ctx->opt, ctx->stream, true, force != 0);
        const uint32_t fmt_of[kTileKinds] = {CFPQ_TILES_FP8, CFPQ_TILES_FP8_128, CFPQ_TILES_FP4, CFPQ_TILES_NVFP4};
        const uint32_t kind = t.kind < kTileKinds ? t.kind : kTileFp4Pair;
        out->tuned = t.tuned ? 1u : 0u;
        out->tile_format = fmt_of[kind];
        out->edge_ratio = tile_ratio_of(kind, t, 8192u);        // 8 MiB blocks: L2-resident
        out->edge_ratio_hbm = tile_ratio_of(kind, t, 65536u);   // 512 MiB blocks
        out->edge_ratio_formula = t.tflops[kind] > 0 && t.gather_gbs > 0 ? ratio_for(t.tflops[kind], t.gather_gbs) : 0u;
        out->probe_status = t.status;
        out->gather_gbs = t.gather_gbs;
        out->gather_gbs_hbm = t.gather_rate(~0ull >> 8);
        out->read_l2_gbs = t.read_l2_gbs;
        out->read_hbm_gbs = t.read_hbm_gbs;
        out->fp8_tflops = t.tflops[kTileFp8Pair];
        out->fp8_128_tflops = t.tflops[kTileFp8Single];
        out->fp4_tflops = t.tflops[kTileFp4Pair];
        out->nvfp4_tflops = t.tflops[kTileFp4NvPair];
        out->probe_ms = t.probe_ms;
        return CFPQ_OK;
    } catch (...) {
        return CFPQ_ERR_OUT_OF_MEMORY;
    }
}
