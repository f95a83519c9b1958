// cfpq_small.cu -- whole fixpoint of a small query in one CTA.
//
// When a query's device state (closure blocks, M2, A2, stamps) fits in the
// shared memory of one SM, the index-creation loop of Listing 1 (arXiv
// 2103.14688, Sec. 3.1) runs inside a single CTA: the same level schedule,
// edge channels and dirty stamps as the multi-kernel path (cfpq_kernels.cu),
// with __syncthreads between passes instead of kernel launches.  Rows are at
// most 512 bits wide (W <= 8 words), so each thread owns one output row per
// step and keeps it in registers.  At the end the closure blocks and M2 are
// copied to the query's global buffers, where every result call reads them.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "cfpq_dev.cuh"

namespace cfpq {

constexpr uint32_t kSmallMaxW = 8;
constexpr int kSmallThreads = 512;

struct SmallSrc {
    uint32_t kind, label, ident, same_level;
    int32_t rblk;
    uint32_t pad;
};

struct SmallDesc {
    uint32_t n, W, B, nblk, n_levels, max_iter, max_passes, pad;
    unsigned long long cyclic_mask;
    const uint32_t *blk_level, *blk_src0, *blk_nsrc;
    const SmallSrc *srcs;
    const uint32_t *box_f0, *box_nf, *fblocks, *box_nullable;
    const uint32_t *csr_off;  // label l, vertex x: csr_off[l * n + x] .. csr_off[l * n + x + 1]
    const uint32_t *csr_col;
    uint64_t *blk_out;        // nblk * n * W
    uint64_t *m2_out;         // B * n * W
    QCtl *ctl;                // statistics written at the end
};

__global__ void __launch_bounds__(kSmallThreads) k_small_fixpoint(const SmallDesc *__restrict__ descs) {
    const SmallDesc D = descs[blockIdx.x];
    const uint32_t n = D.n, W = D.W, B = D.B, nblk = D.nblk;
    extern __shared__ uint64_t sm[];
    uint64_t *C = sm;
    uint64_t *M2 = C + (size_t)nblk * n * W;
    uint64_t *A2 = M2 + (size_t)B * n * W;
    uint32_t *stamp = reinterpret_cast<uint32_t *>(A2 + (size_t)B * n * W);
    uint32_t *last = stamp + (size_t)nblk * n;
    uint32_t *a2it = last + nblk;
    uint32_t *boxit = a2it + (size_t)B * n;
    __shared__ uint32_t s_changed;
    __shared__ unsigned long long s_new, s_ors, s_rows;
    const uint32_t tid = threadIdx.x, T = blockDim.x;

    const size_t words64 = (size_t)(nblk + 2 * B) * n * W;
    for (size_t i = tid; i < words64; i += T) sm[i] = 0ull;
    const size_t words32 = (size_t)nblk * n + nblk + (size_t)B * n + B;
    for (size_t i = tid; i < words32; i += T) stamp[i] = 0u;
    if (tid == 0) { s_ors = 0; s_rows = 0; }
    __syncthreads();
    unsigned long long edges_total = 0;
    // epsilon rows: M2^b[i,i] = A2^b[i,i] = 1 for boxes whose start state is final
    for (uint32_t b = 0; b < B; ++b) {
        if (!D.box_nullable[b]) continue;
        for (uint32_t x = tid; x < n; x += T) {
            M2[((size_t)b * n + x) * W + (x >> 6)] |= 1ull << (x & 63);
            A2[((size_t)b * n + x) * W + (x >> 6)] = 1ull << (x & 63);
            a2it[(size_t)b * n + x] = 1;
        }
        if (tid == 0) boxit[b] = 1;
        edges_total += n;
    }
    __syncthreads();

    uint32_t g = 2, iter = 1, passes = 0, iters_done = 0, status = kStatusOk;
    bool done = false;
    while (!done) {
        const uint32_t g0 = g;
        for (uint32_t L = 0; L < D.n_levels && !done; ++L) {
            uint32_t mode = kModeNew;
            while (true) {
                if (tid == 0) s_changed = 0;
                __syncthreads();
                uint32_t my_ors = 0, my_rows = 0;
                for (uint32_t item = tid; item < nblk * n; item += T) {
                    const uint32_t b = item / n, x = item - b * n;
                    if (D.blk_level[b] != L) continue;
                    uint64_t acc[kSmallMaxW];
#pragma unroll
                    for (uint32_t w = 0; w < kSmallMaxW; ++w) acc[w] = 0ull;
                    for (uint32_t k = 0; k < D.blk_nsrc[b]; ++k) {
                        const SmallSrc s = D.srcs[D.blk_src0[b] + k];
                        uint32_t chans = 0;
                        if (mode == kModeNew) {
                            const bool term1 = s.kind == 0 && iter == 1;
                            if (term1 || (s.kind == 1 && boxit[s.label] == iter)) chans |= 1u;
                            if (s.rblk >= 0 && !s.same_level && !term1 && last[s.rblk] >= g0) chans |= 2u;
                        } else if (s.rblk >= 0 && s.same_level && last[s.rblk] + 1u >= g) {
                            chans |= 4u;
                        }
                        for (uint32_t cb = 1u; cb <= 4u; cb <<= 1) {
                            if (!(chans & cb)) continue;
                            const bool new_edges = cb == 1u;
                            const bool ident = new_edges && s.ident;
                            if (!ident && s.rblk < 0) continue;
                            const uint32_t thr = new_edges ? 0u : (cb == 2u ? g0 : g - 1u);
                            auto take = [&](uint32_t y) {
                                if (ident) {
#pragma unroll
                                    for (uint32_t w = 0; w < kSmallMaxW; ++w)
                                        if (w == (y >> 6)) acc[w] |= 1ull << (y & 63);
                                }
                                if (s.rblk >= 0 && (thr == 0u || stamp[(size_t)s.rblk * n + y] >= thr)) {
                                    const uint64_t *r = C + ((size_t)s.rblk * n + y) * W;
#pragma unroll
                                    for (uint32_t w = 0; w < kSmallMaxW; ++w)
                                        if (w < W) acc[w] |= r[w];
                                    ++my_ors;
                                }
                            };
                            if (s.kind == 0) {
                                const uint32_t *off = D.csr_off + (size_t)s.label * n;
                                for (uint32_t e = off[x]; e < off[x + 1]; ++e) take(D.csr_col[e]);
                            } else {
                                const uint64_t *adj;
                                if (new_edges) {
                                    if (a2it[(size_t)s.label * n + x] != iter) continue;
                                    adj = A2 + ((size_t)s.label * n + x) * W;
                                } else {
                                    adj = M2 + ((size_t)s.label * n + x) * W;
                                }
                                for (uint32_t w = 0; w < W; ++w) {
                                    uint64_t bits = adj[w];
                                    while (bits) {
                                        const uint32_t y = w * 64u + (uint32_t)__ffsll((long long)bits) - 1u;
                                        bits &= bits - 1;
                                        take(y);
                                    }
                                }
                            }
                        }
                    }
                    uint64_t *o = C + ((size_t)b * n + x) * W;
                    bool ch = false;
#pragma unroll
                    for (uint32_t w = 0; w < kSmallMaxW; ++w) {
                        if (w < W && (acc[w] & ~o[w])) {
                            o[w] |= acc[w];
                            ch = true;
                        }
                    }
                    if (ch) {
                        stamp[(size_t)b * n + x] = g;
                        last[b] = g;
                        s_changed = 1;
                        ++my_rows;
                    }
                }
                if (my_ors) atomicAdd(&s_ors, (unsigned long long)my_ors);
                if (my_rows) atomicAdd(&s_rows, (unsigned long long)my_rows);
                __syncthreads();
                const bool changed = s_changed != 0;
                __syncthreads();  // every thread has read the flag before it is reset
                ++passes;
                g += 1;
                if (passes >= D.max_passes) {
                    status = kStatusPassCap;
                    done = true;
                    break;
                }
                if (((D.cyclic_mask >> L) & 1ull) && changed) {
                    mode = kModeProp;
                    continue;
                }
                break;
            }
        }
        if (done) break;
        // extraction: new = OR_f C[q0, f] & ~M2 on rows changed this iteration
        if (tid == 0) s_new = 0;
        __syncthreads();
        unsigned long long my_new = 0;
        for (uint32_t item = tid; item < B * n; item += T) {
            const uint32_t b = item / n, x = item - b * n;
            if (D.box_nf[b] == 0) continue;
            uint64_t cand[kSmallMaxW];
#pragma unroll
            for (uint32_t w = 0; w < kSmallMaxW; ++w) cand[w] = 0ull;
            bool any = false;
            for (uint32_t f = 0; f < D.box_nf[b]; ++f) {
                const uint32_t fb = D.fblocks[D.box_f0[b] + f];
                if (stamp[(size_t)fb * n + x] < g0) continue;
                any = true;
                const uint64_t *r = C + ((size_t)fb * n + x) * W;
#pragma unroll
                for (uint32_t w = 0; w < kSmallMaxW; ++w)
                    if (w < W) cand[w] |= r[w];
            }
            if (!any) continue;
            uint64_t *m = M2 + ((size_t)b * n + x) * W;
            uint64_t *a = A2 + ((size_t)b * n + x) * W;
            bool has = false;
#pragma unroll
            for (uint32_t w = 0; w < kSmallMaxW; ++w) {
                if (w < W) {
                    cand[w] &= ~m[w];
                    has |= cand[w] != 0ull;
                }
            }
            if (!has) continue;
#pragma unroll
            for (uint32_t w = 0; w < kSmallMaxW; ++w) {
                if (w < W) {
                    a[w] = cand[w];
                    m[w] |= cand[w];
                    my_new += (unsigned long long)__popcll(cand[w]);
                }
            }
            a2it[(size_t)b * n + x] = iter + 1;
            boxit[b] = iter + 1;
        }
        if (my_new) atomicAdd(&s_new, my_new);
        __syncthreads();
        const unsigned long long added = s_new;
        __syncthreads();
        iters_done = iter;
        edges_total += added;
        if (added == 0ull) break;
        if (D.max_iter && iter >= D.max_iter) {
            status = kStatusIterCap;
            break;
        }
        ++iter;
        __syncthreads();
    }
    __syncthreads();
    for (size_t i = tid; i < (size_t)nblk * n * W; i += T) D.blk_out[i] = C[i];
    for (size_t i = tid; i < (size_t)B * n * W; i += T) D.m2_out[i] = M2[i];
    if (tid == 0) {
        QCtl c;
        memset(&c, 0, sizeof(c));
        c.g = g;
        c.iter = iter;
        c.phase = kPhaseDone;
        c.status = status;
        c.iters_done = iters_done;
        c.passes = passes;
        c.edges_total = edges_total;
        c.row_ors = s_ors;
        c.rounds_total = passes;
        c.rows_changed_total = s_rows;
        c.n_levels = D.n_levels;
        c.cyclic_mask = D.cyclic_mask;
        *D.ctl = c;
    }
}

size_t small_smem_bytes(uint32_t n, uint32_t W, uint32_t B, uint32_t nblk) {
    return (size_t)(nblk + 2 * B) * n * W * 8 + ((size_t)nblk * n + nblk + (size_t)B * n + B) * 4;
}

size_t small_desc_size() { return sizeof(SmallDesc); }
size_t small_src_size() { return sizeof(SmallSrc); }

// Largest dynamic shared memory a CTA may use on the current device.
size_t small_smem_limit() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return (size_t)v > 2048 ? (size_t)v - 2048 : 0;  // room for the static shared variables
}

cudaError_t launch_small_fixpoint(const void *descs, uint32_t count, size_t smem, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_small_fixpoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_small_fixpoint<<<count, kSmallThreads, smem, st>>>(static_cast<const SmallDesc *>(descs));
    return cudaGetLastError();
}

// Host-side packing of one query's plan for the kernel: `blob` receives the
// arrays, `desc` the descriptor with device addresses inside `dev_blob`.
void build_small_desc(void *desc_out, uint32_t n, uint32_t W, uint32_t B, uint32_t nblk,
                      uint32_t n_levels, unsigned long long cyclic_mask, uint32_t max_iter,
                      uint32_t max_passes, const uint32_t *dev_arrays, const SmallSrc *dev_srcs,
                      size_t off_level, size_t off_src0, size_t off_nsrc, size_t off_f0, size_t off_nf, size_t off_fb,
                      size_t off_null, const uint32_t *csr_off, const uint32_t *csr_col, uint64_t *blk_out,
                      uint64_t *m2_out, QCtl *ctl) {
    SmallDesc d;
    memset(&d, 0, sizeof(d));
    d.n = n;
    d.W = W;
    d.B = B;
    d.nblk = nblk;
    d.n_levels = n_levels;
    d.max_iter = max_iter;
    d.max_passes = max_passes;
    d.cyclic_mask = cyclic_mask;
    d.blk_level = dev_arrays + off_level;
    d.blk_src0 = dev_arrays + off_src0;
    d.blk_nsrc = dev_arrays + off_nsrc;
    d.srcs = dev_srcs;
    d.box_f0 = dev_arrays + off_f0;
    d.box_nf = dev_arrays + off_nf;
    d.fblocks = dev_arrays + off_fb;
    d.box_nullable = dev_arrays + off_null;
    d.csr_off = csr_off;
    d.csr_col = csr_col;
    d.blk_out = blk_out;
    d.m2_out = m2_out;
    d.ctl = ctl;
    memcpy(desc_out, &d, sizeof(d));
}

void fill_small_src(void *dst, uint32_t kind, uint32_t label, uint32_t ident, uint32_t same_level, int32_t rblk) {
    SmallSrc s{kind, label, ident, same_level, rblk, 0u};
    memcpy(dst, &s, sizeof(s));
}

}  // namespace cfpq
