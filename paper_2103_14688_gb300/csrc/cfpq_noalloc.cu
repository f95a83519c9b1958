// cfpq_noalloc.cu -- graph staging for callers that cannot allocate device memory.
//
// cfpq_load_graph_device builds the per-label adjacency lists of a new graph
// with temporary device buffers (counts, offsets, an unsorted copy of the
// edges, a scan workspace, an error flag) that the context allocates.  Some
// callers cannot let a library allocate at that moment: a service that keeps
// every byte of device memory in its own pre-sized pool and swaps in a new
// graph snapshot of the same size, or a process that has already handed the
// rest of the GPU to another framework.  cfpq_load_graph_device_noalloc does
// the same staging with those temporaries in one fixed array compiled into
// the library, and writes the result into the adjacency buffers the context
// already holds from an earlier cfpq_load_graph / cfpq_load_graph_device call.
//
// The fixed array is __device__ memory of every GPU that loads the library,
// held until the process exits.  Every call shares it and it keeps the last
// call's contents, so the counters are cleared at the start of each call, and
// two calls that run at the same time on the GPU (different streams, devices
// sharing nothing else) race on it: callers serialise them.
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "cfpq_ctx.cuh"

using namespace cfpq;

namespace {

// Limits of the fixed workspace.
constexpr size_t kNaMaxRows = (size_t)1 << 19;   // n_terminals * n_vertices
constexpr size_t kNaMaxEdges = (size_t)1 << 21;  // input edges, duplicates included
constexpr size_t kNaAlign = 64;                  // words (256 bytes)
constexpr size_t rup(size_t x) { return (x + kNaAlign - 1) / kNaAlign * kNaAlign; }
constexpr size_t kNaCnt = 0;
constexpr size_t kNaOff = kNaCnt + rup(kNaMaxRows);
constexpr size_t kNaUcnt = kNaOff + rup(kNaMaxRows + 1);
constexpr size_t kNaCol = kNaUcnt + rup(kNaMaxRows);
constexpr size_t kNaTmp = kNaCol + rup(kNaMaxEdges);
constexpr size_t kNaMap = kNaTmp + rup(kNaMaxRows / 4096 + 2);
constexpr size_t kNaErr = kNaMap + rup(kNaMaxRows);
constexpr size_t kNaWords = kNaErr + kNaAlign;  // 4 * 2^19 + 2^21 words + padding: about 16 MiB

__device__ __align__(256) uint32_t g_na_scratch[kNaWords];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
uint32_t *g_na_ptr[kNaMaxDevices] = {nullptr};

__global__ void k_na_identity(int32_t *map, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) map[i] = (int32_t)i;
}

// Device address of the workspace on the current device.  The first call on a
// device resolves it with cudaGetSymbolAddress (which may load the module, so
// it must not happen inside a stream capture).
int scratch_on_device(int dev, uint32_t **out, std::string *err) {
    if (dev < 0 || dev >= kNaMaxDevices) {
        *err = "device ordinal out of range for the fixed workspace table";
        return CFPQ_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p) {
            *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return CFPQ_ERR_CUDA;
        }
        g_na_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_na_ptr[dev];
    return CFPQ_OK;
}

}  // namespace

extern "C" int cfpq_load_graph_device_noalloc(cfpq_ctx *ctx, uint32_t n, uint32_t n_term, size_t m,
                                              const uint32_t *d_src, const uint32_t *d_label,
                                              const uint32_t *d_dst) {
    if (!ctx) return CFPQ_ERR_INVALID_ARG;
    try {
        auto fail = [&](int code, const std::string &msg) {
            ctx->err = msg;
            return code;
        };
        if (n == 0 || n_term == 0) return fail(CFPQ_ERR_INVALID_ARG, "graph needs n_vertices > 0 and n_terminals > 0");
        if (m && (!d_src || !d_label || !d_dst)) return fail(CFPQ_ERR_INVALID_ARG, "edge arrays are NULL");
        const size_t rows = (size_t)n_term * n;
        if (rows > kNaMaxRows || m > kNaMaxEdges)
            return fail(CFPQ_ERR_UNSUPPORTED, "graph exceeds the fixed staging workspace: n_terminals * n_vertices <= " +
                                                  std::to_string(kNaMaxRows) + " and n_edges <= " +
                                                  std::to_string(kNaMaxEdges) + " are required");
        const uint32_t n_pad = (n + 127u) & ~127u, W = n_pad / 64u;
        if (vpl_for_words(W) == 0) return fail(CFPQ_ERR_UNSUPPORTED, "graphs above 65536 vertices are not supported");
        GraphDev &g = ctx->graph;
        if (!g.csr_off.p || g.csr_off.bytes < (rows + 1) * 4 || g.csr_col.bytes < (m ? m : 1) * 4)
            return fail(CFPQ_ERR_BUFFER_TOO_SMALL,
                        "the context's adjacency buffers are smaller than this graph; load a graph at least this "
                        "large with cfpq_load_graph or cfpq_load_graph_device first");
        if (cudaSetDevice(ctx->opt.device) != cudaSuccess) return fail(CFPQ_ERR_CUDA, "cudaSetDevice failed");
        uint32_t *base = nullptr;
        std::string e;
        if (int rc = scratch_on_device(ctx->opt.device, &base, &e)) return fail(rc, e);
        uint32_t *cnt = base + kNaCnt, *off = base + kNaOff, *ucnt = base + kNaUcnt, *col = base + kNaCol;
        uint32_t *tmp = base + kNaTmp;
        int32_t *map = reinterpret_cast<int32_t *>(base + kNaMap);
        int *errf = reinterpret_cast<int *>(base + kNaErr);
        const cudaStream_t st = ctx->stream;
        ctx->has_result = false;
        ++ctx->result_gen;
        ctx->has_graph = false;
#define NA_CK(call)                                                                                 \
    do {                                                                                            \
        cudaError_t _e = (call);                                                                    \
        if (_e != cudaSuccess) return fail(CFPQ_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)
        k_na_identity<<<(n_term + 255) / 256, 256, 0, st>>>(map, n_term);
        NA_CK(cudaGetLastError());
        NA_CK(cudaMemsetAsync(cnt, 0, rows * 4, st));
        NA_CK(cudaMemsetAsync(errf, 0, 16, st));
        NA_CK(launch_stage_count(d_src, d_label, d_dst, m, n, n_term, map, cnt, errf, st));
        NA_CK(scan_exclusive(cnt, off, rows, tmp, st));
        NA_CK(cudaMemsetAsync(ucnt, 0, rows * 4, st));
        NA_CK(launch_stage_fill(d_src, d_label, d_dst, m, n, n_term, map, off, ucnt, col, st));
        NA_CK(launch_stage_unique(off, col, ucnt, rows, st));
        NA_CK(scan_exclusive(ucnt, g.csr_off.as<uint32_t>(), rows, tmp, st));
        NA_CK(launch_stage_compact(off, col, g.csr_off.as<uint32_t>(), g.csr_col.as<uint32_t>(), rows, st));
        int herr = 0;
        uint32_t total = 0;
        NA_CK(cudaMemcpyAsync(&herr, errf, 4, cudaMemcpyDeviceToHost, st));
        NA_CK(cudaMemcpyAsync(&total, g.csr_off.as<uint32_t>() + rows, 4, cudaMemcpyDeviceToHost, st));
        NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
        if (herr) {
            g.n = 0;
            return fail(CFPQ_ERR_INVALID_ARG, "an edge names a vertex >= n_vertices or a label >= n_terminals");
        }
        if (g.n != n || g.n_term != n_term) g.generation += 1;
        g.content += 1;  // the row bitmaps derived from the old edges are stale
        g.n = n;
        g.n_pad = n_pad;
        g.W = W;
        g.n_term = n_term;
        g.m_in = m;
        g.m_unique = total;
        g.host_valid = false;
        ctx->has_graph = true;
        // an RSM reading more terminals than this graph has is reported by
        // cfpq_run, as after cfpq_load_graph_device
        return CFPQ_OK;
    } catch (...) {
        ctx->err = "unexpected exception";
        return CFPQ_ERR_CUDA;
    }
}
