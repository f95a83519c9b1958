// cfpq_resume.cu -- resuming index creation from a checkpointed answer.
//
// Listing 1's fixpoint is monotone in M2: starting it from pairs of the
// answer (an earlier answer on a subset of the edges, or the answer itself)
// ends at the same least fixpoint.  The prologue of a run applies such a
// start after the epsilon rows.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cfpq_dev.cuh"

namespace cfpq {

namespace {
constexpr unsigned FULLMASK = 0xffffffffu;
}  // namespace

// Resume (the fixpoint is monotone): OR a given M2 into every box after the
// epsilon rows, and make each row it touches an A2 row of iteration 1 (A2 :=
// M2 on that row), so the first iteration's passes read all given pairs as
// new edges.  One warp per row of n_boxes x n rows of W words; seed and m2
// share that layout.
__global__ void k_seed_apply(const uint64_t *__restrict__ seed, uint64_t *m2, uint64_t *a2, uint32_t *a2_it,
                             uint32_t *box_new_it, QCtl *ctl, unsigned long long *box_edges, uint32_t n,
                             uint32_t W, uint32_t n_boxes) {
    const uint32_t lane = threadIdx.x & 31u;
    const size_t warps = (size_t)gridDim.x * (blockDim.x >> 5);
    const size_t rows = (size_t)n_boxes * n;
    for (size_t r = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
        const uint64_t *s = seed + r * W;
        bool any = false;
        for (uint32_t k = lane; k < W; k += 32u) any |= s[k] != 0ull;
        if (!__any_sync(FULLMASK, any)) continue;
        uint64_t *m = m2 + r * W, *a = a2 + r * W;
        unsigned long long added = 0;
        for (uint32_t k = lane; k < W; k += 32u) {
            const uint64_t old = m[k], nw = old | s[k];
            m[k] = nw;
            a[k] = nw;
            added += (unsigned long long)__popcll(nw & ~old);
        }
        for (int o = 16; o > 0; o >>= 1) added += __shfl_down_sync(FULLMASK, added, o);
        if (lane == 0) {
            const uint32_t b = (uint32_t)(r / n);
            a2_it[r] = 1u;
            box_new_it[b] = 1u;
            if (added) {
                atomicAdd(&ctl->edges_total, added);
                atomicAdd(&box_edges[b], added);
            }
        }
    }
}

cudaError_t launch_seed_apply(const uint64_t *seed, uint64_t *m2, uint64_t *a2, uint32_t *a2_it, uint32_t *box_new_it,
                              QCtl *ctl, unsigned long long *box_edges, uint32_t n, uint32_t W, uint32_t n_boxes,
                              cudaStream_t st) {
    const size_t rows = (size_t)n_boxes * n, want = (rows + 7) / 8;  // 8 warps (rows) per CTA
    const uint32_t grid = want == 0 ? 1u : (want > 4096 ? 4096u : (uint32_t)want);
    k_seed_apply<<<grid, 256, 0, st>>>(seed, m2, a2, a2_it, box_new_it, ctl, box_edges, n, W, n_boxes);
    return cudaGetLastError();
}

}  // namespace cfpq
