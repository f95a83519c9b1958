// cfpq_shard.cu -- kernels of column-sharded index creation: one query over
// several ranks (GPUs), each computing the closure of Listing 1 (arXiv
// 2103.14688, Sec. 3.1) on its own range of columns (target vertices).
//
// Row x of a closure block C[s,t] is the OR over the product edges
// (s,x) -> (u,y) of row y of C[u,t] (and bit y when u = t), so a range of
// columns of it needs only that range of the rows it reads: a rank holding
// the whole graph and the whole M2 computes its columns of C3 alone, and its
// extraction yields the new edges in its columns.  After every iteration the
// ranks exchange those edges (an all-gather of A2 column slices, done by the
// caller) and install them; these kernels export a rank's slice and install
// the gathered rows.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cfpq_dev.cuh"

namespace cfpq {

// Mark the query as sharded with output columns [v0, v1) (128-bit vectors).
__global__ void k_shard_setup(QCtl *ctl, uint32_t v0, uint32_t v1) {
    ctl->shard = 1u;
    ctl->col_v0 = v0;
    ctl->col_v1 = v1;
    ctl->shard_new = 0ull;
}

// out[b][x][w - w0] = A2^b[x][w] for the words [w0, w1) of rows new in
// iteration `iter` (a2_it), else 0.  One thread per output word.
__global__ void k_shard_export(const uint64_t *__restrict__ a2, const uint32_t *__restrict__ a2_it,
                               uint32_t n, uint32_t W, uint32_t B, uint32_t w0, uint32_t w1, uint32_t iter,
                               uint64_t *__restrict__ out) {
    const uint32_t wl = w1 - w0;
    const size_t total = (size_t)B * n * wl;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / wl;  // b * n + x
        const uint32_t w = (uint32_t)(i % wl) + w0;
        out[i] = a2_it[row] == iter ? a2[row * W + w] : 0ull;
    }
}

// Install the gathered new edges full[b][x][0..W) (every rank's columns):
// per row with any, A2 := full row, a2_it := iter, M2 |= full row; per box,
// cnt[2b] += new edges, cnt[2b + 1] += those this rank had not found (not
// yet in M2).  One warp per row.
__global__ void k_shard_apply(const uint64_t *__restrict__ full, uint64_t *m2, uint64_t *a2, uint32_t *a2_it,
                              uint32_t n, uint32_t W, uint32_t B, uint32_t iter, unsigned long long *cnt) {
    const int lane = threadIdx.x & 31;
    const size_t rows = (size_t)B * n;
    const size_t warp0 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    for (size_t row = warp0; row < rows; row += nwarps) {
        const uint64_t *f = full + row * W;
        uint64_t *m = m2 + row * W, *a = a2 + row * W;
        unsigned long long all = 0ull, foreign = 0ull;
        for (uint32_t w = (uint32_t)lane; w < W; w += 32u) {
            const uint64_t v = f[w];
            all += (unsigned long long)__popcll(v);
            if (v) {
                const uint64_t old = m[w];
                foreign += (unsigned long long)__popcll(v & ~old);
                m[w] = old | v;
            }
        }
        all = __reduce_add_sync(0xffffffffu, (uint32_t)all);
        foreign = __reduce_add_sync(0xffffffffu, (uint32_t)foreign);
        if (all) {
            for (uint32_t w = (uint32_t)lane; w < W; w += 32u) a[w] = f[w];
            if (lane == 0) {
                a2_it[row] = iter;
                const uint32_t b = (uint32_t)(row / n);
                atomicAdd(cnt + 2u * b, all);
                if (foreign) atomicAdd(cnt + 2u * b + 1u, foreign);
            }
        }
    }
}

// After k_shard_apply: per box with new edges box_new_it := iter, box edge
// counts += the edges new to this rank, then the loop's next state: done when
// no rank found an edge (that iteration was the last, as in the unsharded
// loop), or when no transition reads a box that gained edges (the next
// iteration would add none: counted without passes), or at the iteration
// cap; else run the next iteration.  One thread.
__global__ void k_shard_finish(QCtl *ctl, const unsigned long long *cnt, uint32_t *box_new_it, uint32_t B) {
    QCtl &c = *ctl;
    if (c.phase != kPhasePause) return;
    unsigned long long all = 0ull, foreign = 0ull;
    bool read_new = false;
    for (uint32_t b = 0; b < B; ++b) {
        all += cnt[2u * b];
        foreign += cnt[2u * b + 1u];
        if (cnt[2u * b]) {
            box_new_it[b] = c.iter;
            if (c.box_edges) c.box_edges[b] += cnt[2u * b + 1u];
            if (b >= 63u || ((c.nt_read_mask >> b) & 1ull) || ((c.nt_read_mask >> 63) & 1ull)) read_new = true;
        }
    }
    c.edges_total += foreign;
    if (c.box_edges) {
        const unsigned long long dense_at = (unsigned long long)c.n * c.n / kDenseDiv;
        uint32_t m = 0;
        for (uint32_t b = 0; b < c.n_boxes && b < 32u; ++b)
            if (c.box_edges[b] >= dense_at && dense_at > 0ull) m |= 1u << b;
        c.dense_mask = m;
    }
    if (all == 0ull) {
        c.phase = kPhaseDone;  // iters_done already counts this iteration
    } else if (c.max_iter && c.iter - 1u >= c.max_iter) {
        c.status = kStatusIterCap;
        c.phase = kPhaseDone;
    } else if (!read_new) {
        c.iters_done = c.iter;
        c.phase = kPhaseDone;
    } else {
        c.phase = kPhaseRun;
    }
}

cudaError_t launch_shard_setup(QCtl *ctl, uint32_t v0, uint32_t v1, cudaStream_t st) {
    k_shard_setup<<<1, 1, 0, st>>>(ctl, v0, v1);
    return cudaGetLastError();
}

cudaError_t launch_shard_export(const uint64_t *a2, const uint32_t *a2_it, uint32_t n, uint32_t W, uint32_t B,
                                uint32_t w0, uint32_t w1, uint32_t iter, uint64_t *out, cudaStream_t st) {
    if (w1 <= w0) return cudaSuccess;
    k_shard_export<<<1024, 256, 0, st>>>(a2, a2_it, n, W, B, w0, w1, iter, out);
    return cudaGetLastError();
}

cudaError_t launch_shard_apply(const uint64_t *full, uint64_t *m2, uint64_t *a2, uint32_t *a2_it, uint32_t n,
                               uint32_t W, uint32_t B, uint32_t iter, unsigned long long *cnt, QCtl *ctl,
                               uint32_t *box_new_it, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)B * 16, st);
    if (e != cudaSuccess) return e;
    k_shard_apply<<<1024, 256, 0, st>>>(full, m2, a2, a2_it, n, W, B, iter, cnt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_shard_finish<<<1, 1, 0, st>>>(ctl, cnt, box_new_it, B);
    return cudaGetLastError();
}

}  // namespace cfpq
