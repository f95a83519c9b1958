// cfpq_tc.cu -- dense Boolean matrix products on the 5th-generation tensor
// cores (tcgen05, sm_103a) for the closure of Listing 1 (arXiv 2103.14688,
// Sec. 3.1): out[x, z] |= OR_y A[x, y] AND B[y, z] for 0/1 matrices held as
// bit rows.
//
// The Boolean product is computed exactly as an integer count: operands are
// 0/1 FP8-E4M3 (1.0 = 0x38) with FP32 accumulation, or 0/1 unsigned INT8 with
// INT32 accumulation, and a count > 0 sets the output bit.  Counts never
// exceed the inner dimension (<= 65536 < 2^24), so FP32 represents them
// exactly and the result equals the bit-packed product bit for bit.
//
// Tile: 128 output rows x 256 output columns per CTA, K in stages of 128.
// Per stage the CTA loads the A bits (128 rows x 128 bits) and B bits (128
// rows x 256 bits, rows filtered by a dirty stamp), expands them to bytes in
// shared memory in the canonical no-swizzle K-major layout (8-row x 16-byte
// core matrices), B through a 32 x 32 bit transpose done with warp shuffles,
// and one thread issues four 128x256x32 MMAs into a TMEM accumulator (256
// columns of FP32/INT32).  Two shared-memory buffers alternate; an mbarrier
// signalled by tcgen05.commit says when the tensor core has finished reading
// a buffer.  Stages whose A or B tile is all zero are skipped (dirty tiles).
// The epilogue reads the accumulator with tcgen05.ld, thresholds it, ORs the
// bits into the output rows and stamps the rows that changed.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "cfpq_dev.cuh"

namespace cfpq {

namespace tc {

constexpr int kBM = 128, kBN = 256, kBK = 128;       // tile (K in bytes = elements)
constexpr int kKG = kBK / 16;                         // 16-byte core-matrix columns per stage
constexpr int kStageA = kBM * kBK;                    // bytes
constexpr int kStageB = kBN * kBK;
constexpr int kStageBytes = kStageA + kStageB;        // 48 KiB
constexpr int kThreads = 256;
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kWaitLimit = 1u << 26;             // bounded spin on mbarriers: polls ...
constexpr uint64_t kWaitNs = 2000000000ull;           // ... and nanoseconds of %globaltimer

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K) and
// stride (M/N) byte offsets between core matrices, descriptor version 1,
// no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor: D format (1 = F32, 2 = S32), A/B format 0 (E4M3 for
// kind::f8f6f4, unsigned 8-bit for kind::i8), both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t dfmt, uint32_t M, uint32_t N) {
    return (dfmt << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma(bool int8, uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                    uint32_t accum) {
    // kind::i8 is not available on sm_103a (ptxas: "Feature '.kind::i8' not
    // supported on .target 'sm_103a'"); the 0/1 operands use FP8-E4M3.
    (void)int8;
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
}

// Instruction descriptor of the block-scaled FP4 MMAs (kind::mxf4 and
// kind::mxf4nvf4): A and B E2M1 (format 1), both K-major, N >> 3, scale
// factors UE8M0 (bit 23 set: mxf4) or UE4M3 (clear: mxf4nvf4 with 16-element
// blocks), M >> 4, scale-factor data ids 0.  D is always FP32.
__host__ __device__ constexpr uint32_t make_idesc_fp4(uint32_t M, uint32_t N, bool ue8m0) {
    return (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((ue8m0 ? 1u : 0u) << 23) | ((M >> 4) << 24);
}

// 128 x N x 64 MMA of packed 0/1 E2M1 operands (two per byte, 1.0 = 0x2) with
// block scale factors read from TMEM at sfa / sfb: per 32 elements in UE8M0
// (NV false, kind::mxf4) or per 16 elements in UE4M3 (NV true,
// kind::mxf4nvf4).  Every scale there is 1.0, so D accumulates the plain count.
template <bool NV>
__device__ __forceinline__ void mma_fp4(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t sfa,
                                        uint32_t sfb, uint32_t accum) {
    if constexpr (NV)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::mxf4nvf4.block_scale.scale_vec::4X [%0], %1, %2, %3, [%4], [%5], "
            "p;\n\t}\n" ::"r"(dtmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accum));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], "
            "p;\n\t}\n" ::"r"(dtmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accum));
}

// Store v into 32 consecutive TMEM columns of the warp's 32 lanes.
__device__ __forceinline__ void tmem_fill32(uint32_t taddr, uint32_t v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
        "r"(v)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0u;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: false once limit_ns of %globaltimer or kWaitLimit polls have
// passed (the callers then record an error status and finish their work
// without the awaited data).
__device__ __forceinline__ bool mbar_wait(uint64_t *m, uint32_t parity, uint64_t limit_ns = kWaitNs) {
    if (mbar_try_wait(m, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        if (mbar_try_wait(m, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// Self-check of the bounded wait: one thread waits on an mbarrier that no
// thread ever arrives at, so the wait must give up after limit_ns.
__global__ void k_wait_selftest(uint64_t limit_ns, int *timed_out) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *timed_out = mbar_wait(&bar, 0u, limit_ns) ? 0 : 1;
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 TMEM lanes x 32 consecutive 32-bit columns; lane i of the warp gets its
// lane's 32 values.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// As tmem_ld32, without waiting: the registers are valid after tmem_wait_ld.
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 4 bits -> 4 bytes of 0/1 (bit i -> byte i).
__device__ __forceinline__ uint32_t spread4(uint32_t b) { return ((b & 0xFu) * 0x00204081u) & 0x01010101u; }

// 16 bits -> 16 bytes, each 0 or `one`.
__device__ __forceinline__ uint4 expand16(uint32_t b, uint32_t one) {
    return make_uint4(spread4(b) * one, spread4(b >> 4) * one, spread4(b >> 8) * one, spread4(b >> 12) * one);
}

// 8 bits -> 8 nibbles of a word (bit i -> nibble i, the low nibble of byte
// i/2 for even i), each 0 or 0x2 (E2M1 1.0).
__device__ __forceinline__ uint32_t nib8(uint32_t b) {
    uint32_t x = b & 0xFFu;
    x = (x | (x << 12)) & 0x000F000Fu;
    x = (x | (x << 6)) & 0x03030303u;
    x = (x | (x << 3)) & 0x11111111u;
    return x << 1;
}

// 32 bits -> 32 E2M1 nibbles (16 bytes).
__device__ __forceinline__ uint4 expand32_e2m1(uint32_t b) {
    return make_uint4(nib8(b), nib8(b >> 8), nib8(b >> 16), nib8(b >> 24));
}

// Byte offset of element (row r, k byte) in a K-major no-swizzle tile whose
// rows are grouped by 8 and whose K is split into kKG 16-byte columns.
__device__ __forceinline__ uint32_t core_off(uint32_t r, uint32_t kg) {
    return ((r >> 3) * kKG + kg) * 128u + (r & 7u) * 16u;
}

// Transpose a 32 x 32 bit block across a warp: lane i holds row i on entry,
// column i (bit j = row j) on exit.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
    const uint32_t masks[5] = {0xFFFF0000u, 0xFF00FF00u, 0xF0F0F0F0u, 0xCCCCCCCCu, 0xAAAAAAAAu};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int s = 16 >> i;
        const uint32_t M = masks[i];
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, s);
        x = (lane & s) ? ((x & M) | ((y & M) >> s)) : ((x & ~M) | ((y & ~M) << s));
    }
    return x;
}

}  // namespace tc

// The inner dimension of a job in this pass: compacted (the dirty rows listed
// by k_tc_rows, operands expanded by k_tc_a8/k_tc_b8, multiplied by
// k_tc_product_tma) when the job has buffers and the list fits them, else all
// n rows with a stamp filter (k_tc_product).
struct KDim {
    uint32_t kdim;  // rows of the inner dimension
    bool compact;
};

// Output columns [*c0, *c1) the job may write (column sharding; else all).
__device__ __forceinline__ void job_window(const TcJob &J, uint32_t *c0, uint32_t *c1) {
    *c0 = 0u;
    *c1 = 0xFFFFFFFFu;
    if (J.ctl) {
        *c0 = J.ctl->col_v0 * 128u;
        *c1 = J.ctl->col_v1 >= 0x01000000u ? 0xFFFFFFFFu : J.ctl->col_v1 * 128u;
    }
}

// A channel-1 job (covers_new) is always compacted, and runs (kdim > 0)
// only when new_tiles_pay: otherwise the row gather ORs the new edges' rows.
__device__ __forceinline__ KDim job_kdim(const TcJob &J, uint32_t g) {
    KDim k{J.B ? J.n : 0u, false};
    if (J.ys && J.kcount) {
        const unsigned long long kc = *reinterpret_cast<volatile unsigned long long *>(J.kcount);
        const uint32_t d = ((uint32_t)(kc >> 32) == g) ? (uint32_t)kc : 0u;
        if (J.covers_new) return KDim{new_tiles_pay(d, J.kcap, *J.mcount, *J.ecount, J.tile_ratio) ? d : 0u, true};
        if (d <= J.kcap) k = KDim{d, true};
    }
    return k;
}

// Operand bits of one K stage held in registers: A, 64 bits of row m0 + tid/2;
// B, 4 x 32 bits of one row (see the layout below).
struct TcStage {
    uint64_t a;
    uint32_t b[4];
};

__global__ void __launch_bounds__(tc::kThreads, 2)
    k_tc_product(const TcJob *__restrict__ jobs, ExecTables T, int *err_flag) {
    constexpr bool INT8 = false;
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ uint32_t s_changed_rows;
    __shared__ uint8_t s_row_changed[kBM];
    __shared__ uint32_t s_flags[2][kThreads / 32];

    const uint32_t total = *T.t_total;
    if (blockIdx.x >= total) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t one = INT8 ? 0x01u : 0x38u;
    unsigned char *stage[2] = {smem_raw, smem_raw + kStageBytes};
    if (warp == 0) tmem_alloc(&tmem_base, kTmemCols);
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = INT8 ? make_idesc(2, kBM, kBN) : make_idesc(1, kBM, kBN);
    uint32_t parity[2] = {0u, 0u};
    bool inflight[2] = {false, false};
    int buf = 0;
    bool timed_out = false;
    // A: thread = (row ar, half ah) of the 128 x 128-bit stage.  B: 32 blocks
    // of 32 rows x 32 columns; warp w loads rows 32 * (w / 2) + lane of the
    // stage, columns n0 + 128 * (w % 2) + 32 * b.
    const uint32_t ar = (uint32_t)tid >> 1, ah = (uint32_t)tid & 1u;

    for (uint32_t li = blockIdx.x; li < total; li += gridDim.x) {
        // live tile li -> query -> job (tile0 is relative to the query's level group)
        const uint32_t q = find_owner(T.t_pre, T.nq, li);
        const uint32_t ti = li - T.t_pre[q];
        uint32_t lo = T.t_job_beg[q], hi = T.t_job_end[q];
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (jobs[mid].tile0 <= ti) lo = mid;
            else hi = mid;
        }
        const TcJob &J = jobs[lo];
        uint32_t thr, iter, g;
        const uint32_t t = ti - J.tile0;
        const bool act = tc_job_active(J, &thr, &iter, &g) && t < J.tiles_m * J.tiles_n;
        const KDim K = act ? job_kdim(J, g) : KDim{0u, false};
        // compacted jobs run in k_tc_product_tma
        if (!act || K.compact || (K.kdim == 0u && !J.ident)) {
            // skip the rest of this job's tiles in this CTA's stride
            const uint32_t left = J.tiles_m * J.tiles_n > t ? J.tiles_m * J.tiles_n - t : 1u;
            li += ((left - 1u) / gridDim.x) * gridDim.x;
            continue;
        }
        const uint32_t m0 = (t / J.tiles_n) * kBM, n0 = (t % J.tiles_n) * kBN;
        uint32_t wc0, wc1;
        job_window(J, &wc0, &wc1);
        if (n0 < wc0 || n0 >= wc1) continue;  // another rank's columns (uniform over the CTA)
        const uint32_t n = J.n, W = J.W;
        const uint32_t kwords = (K.kdim + 63u) >> 6;
        if (tid < kBM) s_row_changed[tid] = 0;
        if (tid == 0) s_changed_rows = 0;
        bool started = false;
        uint32_t stages_run = 0;
        const uint32_t ksteps = (K.kdim + kBK - 1) / kBK;
        const uint32_t xa = m0 + ar;
        const bool xa_ok = xa < n && (!J.a_it || J.a_it[xa] == iter);

        auto load = [&](uint32_t ks, TcStage &st) {
            const uint32_t k0 = ks * kBK;
            const uint32_t w = (k0 >> 6) + ah;
            st.a = (xa_ok && w < kwords) ? J.A[(size_t)xa * W + w] : 0ull;
            const uint32_t kk = k0 + 32u * ((uint32_t)warp >> 1) + (uint32_t)lane;
            const uint32_t y = kk;
            const bool rok = kk < n && (!J.b_stamp || thr == 0u || J.b_stamp[kk] >= thr);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t zc = n0 + 128u * ((uint32_t)warp & 1u) + 32u * (uint32_t)b;
                uint32_t v = 0;
                if (rok && zc < (W << 6)) v = (uint32_t)(J.B[(size_t)y * W + (zc >> 6)] >> (zc & 63u));
                st.b[b] = v;
            }
        };
        // per-warp flags of a stage: bit 0 some A bit, bit 1 some B bit, bit 2 a wait timed out
        auto flags_of = [&](const TcStage &st) -> uint32_t {
            const bool fa = __any_sync(0xffffffffu, st.a != 0ull);
            const bool fb = __any_sync(0xffffffffu, (st.b[0] | st.b[1] | st.b[2] | st.b[3]) != 0u);
            return (fa ? 1u : 0u) | (fb ? 2u : 0u);
        };

        TcStage s0{0ull, {0u, 0u, 0u, 0u}}, s1{0ull, {0u, 0u, 0u, 0u}}, s2{0ull, {0u, 0u, 0u, 0u}};
        if (ksteps > 0) load(0, s0);
        if (ksteps > 1) load(1, s1);
        {
            const uint32_t f = ksteps > 0 ? flags_of(s0) : 0u;
            if (lane == 0) s_flags[0][warp] = f;
        }
        __syncthreads();
        for (uint32_t ks = 0; ks < ksteps; ++ks) {
            // flags of stage ks were published before the last barrier
            uint32_t fa = 0u, fb = 0u, fx = 0u;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) {
                const uint32_t f = s_flags[ks & 1u][w];
                fa |= f & 1u;
                fb |= f & 2u;
                fx |= f & 4u;
            }
            if (fx) {
                timed_out = true;
                break;
            }
            if (ks + 2 < ksteps) load(ks + 2, s2);  // two stages in flight
            const bool run = fa && fb;              // dirty-tile skip: a stage with no A or no B bit adds nothing
            bool my_to = false;
            if (run) {
                if (inflight[buf]) {  // the buffer must be free: wait for the MMAs that read it
                    if (!mbar_wait(&mbar[buf], parity[buf])) my_to = true;
                    parity[buf] ^= 1u;
                    inflight[buf] = false;
                }
                unsigned char *sa = stage[buf], *sb = stage[buf] + kStageA;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    const uint32_t kg = ah * 4u + (uint32_t)qq;
                    *reinterpret_cast<uint4 *>(sa + core_off(ar, kg)) =
                        expand16((uint32_t)(s0.a >> (16 * qq)) & 0xFFFFu, one);
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const uint32_t col = transpose32(s0.b[b], lane);  // bit i = row 32 * (warp/2) + i
                    const uint32_t z = 128u * ((uint32_t)warp & 1u) + 32u * (uint32_t)b + (uint32_t)lane;
                    const uint32_t kg = 2u * ((uint32_t)warp >> 1);
                    *reinterpret_cast<uint4 *>(sb + core_off(z, kg)) = expand16(col & 0xFFFFu, one);
                    *reinterpret_cast<uint4 *>(sb + core_off(z, kg + 1u)) = expand16(col >> 16, one);
                }
                fence_async_smem();
            }
            {
                uint32_t f = ks + 1 < ksteps ? flags_of(s1) : 0u;
                if (__any_sync(0xffffffffu, my_to)) f |= 4u;
                if (lane == 0) s_flags[(ks + 1) & 1u][warp] = f;
            }
            tc_before();
            __syncthreads();
            tc_after();
            if (run) {
                if (tid == 0) {
                    const uint32_t abase = smem_u32(stage[buf]), bbase = smem_u32(stage[buf] + kStageA);
#pragma unroll
                    for (int kk = 0; kk < kBK / 32; ++kk) {
                        const uint64_t ad = make_desc(abase + (uint32_t)kk * 256u, 128u, kKG * 128u);
                        const uint64_t bd = make_desc(bbase + (uint32_t)kk * 256u, 128u, kKG * 128u);
                        tc::mma(INT8, tmem, ad, bd, idesc, (started || kk > 0) ? 1u : 0u);
                    }
                    mma_commit(&mbar[buf]);
                }
                started = true;
                ++stages_run;
                inflight[buf] = true;
                buf ^= 1;
            }
            s0 = s1;
            s1 = s2;
        }
        for (int b = 0; b < 2; ++b) {  // drain
            if (inflight[b]) {
                if (!mbar_wait(&mbar[b], parity[b])) timed_out = true;
                parity[b] ^= 1u;
                inflight[b] = false;
            }
        }
        tc_before();
        __syncthreads();
        tc_after();
        if (__syncthreads_or(timed_out)) {
            timed_out = true;
            break;
        }
        // epilogue: warps 0-3 columns [0,128), warps 4-7 columns [128,256)
        if (started || J.ident) {
            const uint32_t quarter = (uint32_t)warp & 3u, half = (uint32_t)warp >> 2;
            const uint32_t r = quarter * 32u + (uint32_t)lane;  // tile row = TMEM lane
            const uint32_t x = m0 + r;
            uint32_t mask[4] = {0u, 0u, 0u, 0u};
            if (started) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    uint32_t v[32];
                    const uint32_t col = half * 128u + 32u * (uint32_t)c;
                    tc::tmem_ld32(tmem + ((quarter * 32u) << 16) + col, v);
                    uint32_t mbits = 0u;
#pragma unroll
                    for (int i = 0; i < 32; ++i) mbits |= (v[i] != 0u ? 1u : 0u) << i;
                    mask[c] = mbits;
                }
            }
            if (x < n) {
                const uint32_t w0 = (n0 + half * 128u) >> 6;
                bool ch = false;
#pragma unroll
                for (int wq = 0; wq < 2; ++wq) {
                    const uint32_t w = w0 + (uint32_t)wq;
                    if (w >= W) continue;
                    uint64_t add = (uint64_t)mask[2 * wq] | ((uint64_t)mask[2 * wq + 1] << 32);
                    if (J.ident && (!J.a_it || J.a_it[x] == iter)) add |= J.A[(size_t)x * W + w];
                    if (!add) continue;
                    // several jobs (sources) of one output block may share a launch
                    const uint64_t old = atomicOr(reinterpret_cast<unsigned long long *>(J.out + (size_t)x * W + w),
                                                  (unsigned long long)add);
                    if (add & ~old) ch = true;
                }
                if (ch) s_row_changed[r] = 1;
            }
        }
        tc_before();
        __syncthreads();
        tc_after();
        if (tid < kBM && s_row_changed[tid]) {
            if (J.out_stamp) J.out_stamp[m0 + tid] = g;
            atomicAdd(&s_changed_rows, 1u);
        }
        __syncthreads();
        if (tid == 0) {
            if (s_changed_rows) {
                if (J.out_last) *J.out_last = g;
                if (J.ctl) atomicAdd(&J.ctl->changed_rows, (unsigned long long)s_changed_rows);
            }
            if (J.ctl && started) {
                atomicAdd(&J.ctl->tile_mmas, 1ull);
                atomicAdd(&J.ctl->tile_kstages, (unsigned long long)stages_run);
            }
        }
        __syncthreads();
    }
    if (timed_out && tid == 0) atomicOr(err_flag, 1);
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// Dirty-row compaction of the product jobs (channels 2 and 4).
// ---------------------------------------------------------------------------
constexpr uint32_t kRowChunk = 2048;  // k_tc_rows: rows per unit
constexpr uint32_t kColRows = 8;      // k_tc_cols: rows per unit (one per warp)
constexpr uint32_t kColMaxW = 1024;   // largest row in words (n <= 65536)
constexpr uint32_t kCasLimit = 1u << 20;

// Reserve `cnt` entries of the job's list for pass g; the count word carries
// the pass stamp, so the first reservation of a pass starts from 0.
__device__ __forceinline__ uint32_t reserve_rows(unsigned long long *kc, uint32_t g, uint32_t cnt, int *err_flag) {
    unsigned long long old = *reinterpret_cast<volatile unsigned long long *>(kc);
    for (uint32_t i = 0; i < kCasLimit; ++i) {
        const uint32_t cur = ((uint32_t)(old >> 32) == g) ? (uint32_t)old : 0u;
        const unsigned long long nw = ((unsigned long long)g << 32) | (unsigned long long)(cur + cnt);
        const unsigned long long prev = atomicCAS(kc, old, nw);
        if (prev == old) return cur;
        old = prev;
    }
    atomicOr(err_flag, 2);
    return 0xFFFFFFFFu;
}

// Units (job, chunk) of the pass's active jobs (the control kernel's list)
// are numbered in list order; the CTA takes those congruent to its index.
// `body(J, c)` runs for each.
template <typename F>
__device__ __forceinline__ void for_job_chunks(const TcJob *jobs, const ExecTables &T, uint32_t rows_per_chunk,
                                               F body) {
    uint32_t u0 = 0;
    const uint32_t na = *T.aj_n;
    for (uint32_t a = 0; a < na; ++a) {
        const TcJob &J = jobs[T.aj[a]];
        const uint32_t chunks = (J.n + rows_per_chunk - 1) / rows_per_chunk;
        const uint32_t first = (blockIdx.x + gridDim.x - (u0 % gridDim.x)) % gridDim.x;
        u0 += chunks;
        if (first >= chunks || !J.ys) continue;
        for (uint32_t c = first; c < chunks; c += gridDim.x) body(J, c);
    }
}

// Channel-1 jobs (TcJob::covers_new), before their row lists: for the A2
// rows x new in the iteration, newcols (zeroed before the pass) |= row x,
// x is appended to xs, and *ecount += the row's edges.  Unit: 512 rows;
// thread t ORs words t, t + 256, ... of those rows in registers and merges
// them with one atomicOr per word.
constexpr uint32_t kNewColRows = 512;
__global__ void __launch_bounds__(256) k_tc_newcols(const TcJob *__restrict__ jobs, ExecTables T) {
    __shared__ unsigned long long s_edges;
    for_job_chunks(jobs, T, kNewColRows, [&](const TcJob &J, uint32_t c) {
        uint32_t thr, iter, g;
        if (!J.covers_new || !tc_job_active(J, &thr, &iter, &g)) return;
        const uint32_t W = J.W, x_end = min(J.n, (c + 1u) * kNewColRows);
        constexpr int kWordsPerThread = (int)(kColMaxW / 256u);
        uint64_t acc[kWordsPerThread];
#pragma unroll
        for (int i = 0; i < kWordsPerThread; ++i) acc[i] = 0ull;
        unsigned long long edges = 0ull;
        for (uint32_t x = c * kNewColRows; x < x_end; ++x) {
            if (J.a_it[x] != iter) continue;
            if (threadIdx.x == 0) J.xs[atomicAdd(J.mcount, 1ull)] = x;
            const uint64_t *row = J.A + (size_t)x * W;
#pragma unroll
            for (int i = 0; i < kWordsPerThread; ++i) {
                const uint32_t w = threadIdx.x + 256u * (uint32_t)i;
                if (w < W) {
                    const uint64_t v = row[w];
                    acc[i] |= v;
                    edges += (unsigned long long)__popcll(v);
                }
            }
        }
        if (threadIdx.x == 0) s_edges = 0ull;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kWordsPerThread; ++i) {
            const uint32_t w = threadIdx.x + 256u * (uint32_t)i;
            if (w < W && acc[i]) atomicOr(reinterpret_cast<unsigned long long *>(J.newcols + w), acc[i]);
        }
        edges = __reduce_add_sync(0xffffffffu, (uint32_t)edges);
        if ((threadIdx.x & 31) == 0 && edges) atomicAdd(&s_edges, edges);
        __syncthreads();
        if (threadIdx.x == 0 && s_edges) atomicAdd(J.ecount, s_edges);
        __syncthreads();
    });
}

// List the rows y of B with stamp >= thr; for a channel-1 job the columns
// of its newcols (order irrelevant: the product sums over them).
__global__ void __launch_bounds__(256) k_tc_rows(const TcJob *__restrict__ jobs, ExecTables T, int *err_flag) {
    // a unit's listed rows are counted over the CTA first, so that the unit
    // reserves its part of the list with one atomic (one per warp step kept
    // thousands of atomics queued on the count word of a pass)
    constexpr uint32_t kPer = kRowChunk / 256u;  // rows per thread
    static_assert(kRowChunk % 256u == 0u && kPer <= 32u, "k_tc_rows: 256 threads, a bit per row");
    __shared__ uint32_t s_warp[8], s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for_job_chunks(jobs, T, kRowChunk, [&](const TcJob &J, uint32_t c) {
        uint32_t thr, iter, g;
        if (!tc_job_active(J, &thr, &iter, &g) || (!J.b_stamp && !J.covers_new)) return;
        const uint32_t y_beg = c * kRowChunk, y_end = min(J.n, y_beg + kRowChunk);
        uint32_t mask = 0u;
#pragma unroll
        for (uint32_t i = 0; i < kPer; ++i) {
            const uint32_t y = y_beg + threadIdx.x + 256u * i;
            const bool dirty = y < y_end && (J.covers_new ? ((J.newcols[y >> 6] >> (y & 63u)) & 1ull) != 0ull
                                                          : J.b_stamp[y] >= thr);
            if (dirty) mask |= 1u << i;
        }
        // exclusive prefix of the threads' counts over the CTA
        const uint32_t cnt = (uint32_t)__popc(mask);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t run = 0u;
            for (int w = 0; w < 8; ++w) {
                const uint32_t t = s_warp[w];
                s_warp[w] = run;
                run += t;
            }
            s_base = run ? reserve_rows(J.kcount, g, run, err_flag) : 0u;
        }
        __syncthreads();
        const uint32_t base = s_base;
        if (base != 0xFFFFFFFFu) {
            uint32_t pos = base + s_warp[warp] + incl - cnt;
            for (uint32_t m = mask; m; m &= m - 1u) J.ys[pos++] = y_beg + threadIdx.x + 256u * (uint32_t)(__ffs(m) - 1);
        }
        __syncthreads();  // s_warp and s_base are reused by the next unit
    });
}

// a8[x][k] = A[x][ys[k]] as a 0/1 FP8 byte for k < D, 0 up to the next
// multiple of 128; one warp per row x, the row staged in shared memory, each
// lane writing 4 consecutive bytes of a coalesced 128-byte step.  FP4 jobs
// get E2M1 nibbles instead (see below).
__global__ void __launch_bounds__(256) k_tc_a8(const TcJob *__restrict__ jobs, ExecTables T, uint32_t max_w) {
    extern __shared__ uint64_t s_rowbuf[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *row = s_rowbuf + (size_t)warp * max_w;
    for_job_chunks(jobs, T, kColRows, [&](const TcJob &J, uint32_t c) {
        uint32_t thr, iter, g;
        if (!tc_job_active(J, &thr, &iter, &g)) return;
        const KDim K = job_kdim(J, g);
        if (!K.compact || K.kdim == 0u) return;
        // row m of a8: A's row m, or for a channel-1 job A2's row xs[m]
        const uint32_t m = c * kColRows + (uint32_t)warp;
        if (m >= (J.covers_new ? (uint32_t)*J.mcount : J.n)) return;
        const uint32_t x = J.covers_new ? J.xs[m] : m;
        const uint32_t W = J.W, D = K.kdim, dpad = (D + 127u) & ~127u;
        const uint4 *src = reinterpret_cast<const uint4 *>(J.A + (size_t)x * W);
        bool nz = false;
        for (uint32_t v = (uint32_t)lane; v < W / 2u; v += 32u) {
            const uint4 t4 = src[v];
            reinterpret_cast<uint4 *>(row)[v] = t4;
            nz |= (t4.x | t4.y | t4.z | t4.w) != 0u;
        }
        nz = __any_sync(0xffffffffu, nz);
        __syncwarp();
        uint32_t *dst = reinterpret_cast<uint32_t *>(J.a8 + (size_t)m * J.kstride);
        if (J.fp4) {
            // E2M1 nibbles: 8 elements (4 bytes) per lane and 256-element step,
            // zero up to the next multiple of 256 (a whole K stage) within kcap
            const uint32_t kend = min((D + 255u) & ~255u, J.kcap);
            for (uint32_t k0 = 0; k0 < kend; k0 += 256u) {
                const uint32_t kb = k0 + 8u * (uint32_t)lane;
                if (kb >= kend) continue;
                uint32_t word = 0u;
                if (nz && kb < D) {
                    const uint4 y0 = *reinterpret_cast<const uint4 *>(J.ys + kb);
                    const uint4 y1 = *reinterpret_cast<const uint4 *>(J.ys + kb + 4u);
                    const uint32_t yv[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (kb + (uint32_t)i < D && ((row[yv[i] >> 6] >> (yv[i] & 63u)) & 1ull))
                            word |= 0x2u << (4 * i);
                }
                dst[kb >> 3] = word;
            }
            __syncwarp();
            return;
        }
        for (uint32_t k0 = 0; k0 < dpad; k0 += 128u) {
            const uint32_t kb = k0 + 4u * (uint32_t)lane;
            uint32_t word = 0u;
            if (nz && kb < D) {
                const uint4 y4 = *reinterpret_cast<const uint4 *>(J.ys + kb);
                const uint32_t yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (kb + (uint32_t)i < D && ((row[yv[i] >> 6] >> (yv[i] & 63u)) & 1ull)) word |= 0x38u << (8 * i);
            }
            dst[kb >> 2] = word;
        }
        __syncwarp();  // the next row reuses the staging buffer
    });
}

// b8[z][k] = B[ys[k]][z] as a 0/1 FP8 byte (B's listed rows transposed), for
// the columns z of the rank's window below n_pad and k below the next
// multiple of 128 of D (FP4 jobs: E2M1 nibbles, k below the next multiple of
// 256 within kcap).  Unit of a warp: 64 listed rows x 256 columns (128 at
// the end of a row).  Lane l loads 32 bytes of rows ys[k0 + l] and
// ys[k0 + 32 + l] at those columns (whole 32-byte sectors); every 32 x 32
// bit block is transposed across the warp with shuffles (lane c then holds
// column z0 + c over the 32 rows), and every lane writes its column's 64
// elements: 32 bytes of E2M1 nibbles (a whole sector) or 64 FP8 bytes.
__global__ void __launch_bounds__(256) k_tc_b8(const TcJob *__restrict__ jobs, ExecTables T) {
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    uint32_t u0 = 0;
    const uint32_t na = *T.aj_n;
    for (uint32_t a = 0; a < na; ++a) {
        const TcJob &J = jobs[T.aj[a]];
        if (!J.ys) continue;
        uint32_t thr, iter, g;
        if (!tc_job_active(J, &thr, &iter, &g)) continue;
        const KDim K = job_kdim(J, g);
        if (!K.compact || K.kdim == 0u) continue;
        uint32_t wc0, wc1;
        job_window(J, &wc0, &wc1);
        const uint32_t D = K.kdim, W = J.W, zend = min(W * 64u, wc1), zbeg = min(wc0, zend);
        // (the window and n_pad are multiples of 128 columns; an FP4 job's
        // K stage is 256 elements, zero-padded within kcap)
        const uint32_t kpad = J.fp4 ? min((D + 255u) & ~255u, J.kcap) : (D + 127u) & ~127u;
        const uint32_t kchunks = kpad / 64u, zchunks = (zend - zbeg + 255u) / 256u;
        const uint32_t units = kchunks * zchunks;
        const uint32_t first = (gw + nw - (u0 % nw)) % nw;
        u0 += units;
        if (first == 0u && lane == 0 && units && J.ctl) {
            // operand bytes of the job in this pass: B's (this kernel) and A's (k_tc_a8)
            const uint32_t ka = J.fp4 ? min((D + 255u) & ~255u, J.kcap) / 2u : (D + 127u) & ~127u;
            const unsigned long long rows_a = J.covers_new ? *J.mcount : (unsigned long long)J.n;
            atomicAdd(&J.ctl->tile_operand_bytes,
                      (unsigned long long)(zend - zbeg) * (J.fp4 ? kpad / 2u : kpad) + rows_a * ka);
        }
        for (uint32_t u = first; u < units; u += nw) {
            const uint32_t k0 = (u / zchunks) * 64u, z0 = zbeg + (u % zchunks) * 256u;
            const uint32_t halves = min(2u, (zend - z0) / 128u);  // 128-column halves in the row
            // rows k0 + lane (h = 0) and k0 + 32 + lane (h = 1), columns z0 .. z0 + 255
            uint4 row[2][2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t k = k0 + 32u * (uint32_t)h + (uint32_t)lane;
                const uint4 *src = k < D ? reinterpret_cast<const uint4 *>(J.B + (size_t)J.ys[k] * W + (z0 >> 6))
                                         : nullptr;
#pragma unroll
                for (int c = 0; c < 2; ++c)
                    row[h][c] = (src && (uint32_t)c < halves) ? src[c] : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if ((uint32_t)c >= halves) continue;  // (uniform over the warp)
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const uint32_t zc = z0 + 128u * (uint32_t)c + 32u * (uint32_t)p;
                    uint32_t mine[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t bits = p == 0 ? row[h][c].x : p == 1 ? row[h][c].y : p == 2 ? row[h][c].z
                                                                                                     : row[h][c].w;
                        // lane l holds columns zc .. zc + 31 of row ys[k0 + 32 h + l]; after
                        // the shuffle transpose lane c holds column zc + c (bit i: row i)
                        mine[h] = tc::transpose32(bits, lane);
                    }
                    unsigned char *rowp = J.b8 + (size_t)(zc + (uint32_t)lane) * J.kstride;
                    if (J.fp4) {
                        uint4 *dst = reinterpret_cast<uint4 *>(rowp + k0 / 2u);
                        dst[0] = tc::expand32_e2m1(mine[0]);
                        dst[1] = tc::expand32_e2m1(mine[1]);
                    } else {
                        uint4 *dst = reinterpret_cast<uint4 *>(rowp + k0);
                        dst[0] = tc::expand16(mine[0] & 0xFFFFu, 0x38u);
                        dst[1] = tc::expand16(mine[0] >> 16, 0x38u);
                        dst[2] = tc::expand16(mine[1] & 0xFFFFu, 0x38u);
                        dst[3] = tc::expand16(mine[1] >> 16, 0x38u);
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// TMA-fed product of the compacted jobs.  Warp 0 (one lane) streams the FP8
// operand tiles of every K stage into a ring of shared-memory stages with
// cp.async.bulk.tensor (128-byte swizzle); warp 1 (one lane) issues the
// tcgen05 MMAs into TMEM and commits each stage back to the producer; warps
// 2-9 read a finished accumulator (each its TMEM lane quarter and column
// half), threshold it and OR the bits into the output block.
// ---------------------------------------------------------------------------
namespace tc2 {
constexpr int kRing = 4;
constexpr uint32_t kABytes = 128u * 128u, kBBytes = 256u * 128u, kStage = kABytes + kBBytes;  // 48 KiB
constexpr int kThreads = 320;      // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr uint32_t kEpiWarps = 8;
constexpr uint32_t kTmemCols = 512;  // two 256-column accumulators

// K-major operand tile written by TMA with the 128-byte swizzle: 128-byte
// rows, 8-row groups 1024 bytes apart; layout type 2 (SWIZZLE_128B).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void arrive_expect_tx(uint64_t *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(m)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void arrive(uint64_t *m) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(m)) : "memory");
}

__device__ __forceinline__ void tma_load(void *dst, const void *map, int32_t c0, int32_t c1, uint64_t *m) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(tc::smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(tc::smem_u32(m))
        : "memory");
}

// The next live tile of a compacted job at or after li (same walk in every
// role): job, tile origin, K stages and pass stamp.  The job of the last tile
// is cached with its range of live-tile indices, so the tables are read once
// per job rather than once per tile.
struct Tile {
    const TcJob *J;
    uint32_t m0, n0, ks, g;
    uint32_t mlim;  // rows of a8 (a channel-1 job's row count; else n)
};
struct JobCache {
    const TcJob *J = nullptr;
    uint32_t li0 = 1u, li1 = 0u;  // live-tile indices of the job: [li0, li1)
    uint32_t ks = 0, g = 0, mlim = 0;
    uint32_t c0 = 0, c1 = 0;      // output columns of this rank (column sharding)
    uint32_t ntn = 0;             // column tiles of the job
    bool ok = false;
};

constexpr uint32_t kGroupCols = 8;  // column tiles per group of the tile walk

// ROWS: output rows per tile, 128, or 256 (two accumulators, PAIR).  COLS:
// output columns per tile, 256 (FP8), or 192 (FP4: the two accumulators
// leave TMEM columns for the scale factors).  KSTAGE: elements of K per
// 128-byte stage row (128 FP8 bytes or 256 E2M1 nibbles).  The live-tile
// indices of a job cover tiles_m x tiles_n tiles of 128 x 256, at least as
// many as ceil(n / ROWS) x ceil(n / COLS) for both shapes.
template <uint32_t ROWS, uint32_t COLS = 256u, uint32_t KSTAGE = 128u>
__device__ __forceinline__ bool next_tile(const TcJob *jobs, const ExecTables &T, uint32_t total, uint32_t &li,
                                          Tile &tl, JobCache &jc) {
    for (; li < total; li += gridDim.x) {
        if (li >= jc.li0 && li < jc.li1) {
            if (!jc.ok) {  // skip the rest of the cached job's tiles
                li += ((jc.li1 - 1u - li) / gridDim.x) * gridDim.x;
                continue;
            }
            // Grouped tile order: the column tiles form groups of
            // kGroupCols; a group is walked row tile by row tile, its
            // columns inner.  CTAs running side by side then share each A
            // tile (ROWS rows x K) kGroupCols times and each B tile (COLS
            // columns x K) about gridDim / kGroupCols times, and A is read
            // once per group instead of once per column tile (a plain
            // column-major walk re-read A -- n x K operand bytes, beyond L2
            // at n = 65536 -- for every column tile).  A channel-1 job walks
            // only the tile rows its row list fills.
            const uint32_t t = li - jc.li0, mt = (jc.mlim + ROWS - 1u) / ROWS;
            if (t >= mt * jc.ntn) {  // past the job's row tiles: the rest of the job too
                li += ((jc.li1 - 1u - li) / gridDim.x) * gridDim.x;
                continue;
            }
            const uint32_t gsz = mt * kGroupCols, grp = t / gsz, within = t - grp * gsz;
            const uint32_t gcols = min(kGroupCols, jc.ntn - grp * kGroupCols);
            tl.m0 = (within / gcols) * ROWS;
            tl.n0 = (grp * kGroupCols + within % gcols) * COLS;
            // another rank's columns (rank windows are multiples of 256
            // columns; a 192-column tile may straddle one and is masked)
            if (tl.n0 + COLS <= jc.c0 || tl.n0 >= jc.c1) continue;
            tl.J = jc.J;
            tl.ks = jc.ks;
            tl.g = jc.g;
            tl.mlim = jc.mlim;
            return true;
        }
        const uint32_t q = find_owner(T.t_pre, T.nq, li);
        const uint32_t ti = li - T.t_pre[q];
        uint32_t lo = T.t_job_beg[q], hi = T.t_job_end[q];
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (jobs[mid].tile0 <= ti) lo = mid;
            else hi = mid;
        }
        const TcJob &J = jobs[lo];
        const uint32_t t = ti - J.tile0, tiles = J.tiles_m * J.tiles_n;
        if (t >= tiles) continue;  // past the jobs of this query's level
        uint32_t thr, iter, g = 0;
        bool ok = J.ys != nullptr && tc_job_active(J, &thr, &iter, &g);
        KDim K{0u, false};
        if (ok) {
            K = job_kdim(J, g);
            ok = K.compact && K.kdim > 0u;
        }
        jc.J = &J;
        jc.li0 = li - t;
        jc.li1 = li - t + tiles;
        jc.ok = ok;
        jc.ks = (K.kdim + KSTAGE - 1u) / KSTAGE;
        jc.g = g;
        jc.mlim = ok && J.covers_new ? (uint32_t)*J.mcount : J.n;
        jc.ntn = COLS == 256u ? J.tiles_n : (J.n + COLS - 1u) / COLS;
        job_window(J, &jc.c0, &jc.c1);
        li -= gridDim.x;  // re-enter through the cache
    }
    return false;
}
}  // namespace tc2

// PAIR: each CTA computes 256 output rows (two 128-row A tiles against one
// B tile per K stage, two TMEM accumulators, so no second buffer): 64 KiB of
// operands per stage feed twice the multiply-adds of the 48 KiB stage of the
// single tile, and three stages in flight hold as much work as six of those.
//
// FP4 (with PAIR): the operands are packed 0/1 E2M1 nibbles, 256 elements of
// K per 128-byte stage row, multiplied by the block-scaled kind::mxf4 MMA
// (NV: kind::mxf4nvf4; M = 128, N = 192, K = 64) whose scale factors are all
// 1.0.  The two
// 192-column accumulators sit at TMEM columns 0 and 256; the columns between
// (192-255 and 448-511) hold the scale factors, every byte 1.0 (UE8M0 0x7F,
// UE4M3 0x38), so any scale the MMA reads there is 1.0 and the accumulator
// holds the plain count.
// A stage is 2 x 16 KiB of A and 24 KiB of B; four stages are in flight.
template <bool PAIR, bool FP4, bool NV = false>
__global__ void __launch_bounds__(tc2::kThreads, 1)
    k_tc_product_tma(const TcJob *__restrict__ jobs, const unsigned char *__restrict__ maps, ExecTables T,
                     int *err_flag) {
    using namespace tc;
    using namespace tc2;
    static_assert(PAIR || !FP4, "FP4 tiles run paired");
    constexpr uint32_t kRows = PAIR ? 256u : 128u;
    constexpr uint32_t kCols = FP4 ? 192u : 256u;        // output columns per tile (MMA N)
    constexpr uint32_t kKStage = FP4 ? 256u : 128u;      // K elements per 128-byte stage row
    constexpr uint32_t kBBytesN = kCols * 128u;
    constexpr int kRingN = FP4 ? 4 : (PAIR ? 3 : kRing);
    constexpr uint32_t kStageN = (PAIR ? 2u : 1u) * kABytes + kBBytesN;
    constexpr uint32_t kBufs = PAIR ? 1u : 2u;  // accumulator buffers (each 256 columns per 128 rows)
    static_assert(kRingN * kStageN + 1024u <= 227u * 1024u, "stages exceed the shared memory of an SM");
    extern __shared__ __align__(1024) unsigned char smem_raw2[];
    __shared__ uint64_t full[kRingN], empty[kRingN], tfull[2], tempty[2];
    __shared__ uint32_t tmem_base;
    const uint32_t total = *T.t_total;
    if (blockIdx.x >= total) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // stage buffers start 1024-byte aligned (the swizzle pattern repeats every 1024 bytes)
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw2) + 1023u) & ~static_cast<uintptr_t>(1023u));
    if (warp == 0) tmem_alloc(&tmem_base, tc2::kTmemCols);
    if (tid == 0) {
        for (int i = 0; i < kRingN; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], kEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t kSfa = 192u, kSfb = 224u;  // FP4: scale-factor columns of A and B
    if constexpr (FP4) {
        // every TMEM column outside the two accumulators holds UE8M0 1.0
        // (warps 2-5 cover the four lane quarters of columns 192-255, warps
        // 6-9 those of columns 448-511)
        if (warp >= 2) {
            const uint32_t quarter = (uint32_t)warp & 3u, col = warp < 6 ? 192u : 448u;
            // 1.0: UE8M0 0x7F (2^(127-127)); UE4M3 0x38 (2^(7-7) x 1.0)
            constexpr uint32_t one4 = NV ? 0x38383838u : 0x7F7F7F7Fu;
            tmem_fill32(tmem + ((quarter * 32u) << 16) + col, one4);
            tmem_fill32(tmem + ((quarter * 32u) << 16) + col + 32u, one4);
            tmem_wait_st();
        }
        tc_before();
        __syncthreads();
        tc_after();
    }
    constexpr uint32_t idesc = FP4 ? make_idesc_fp4(128, kCols, !NV) : make_idesc(1, 128, 256);
    bool to = false;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            uint32_t stage = 0, ph = 0, li = blockIdx.x;
            Tile tl;
            JobCache jc;
            while (!to && next_tile<kRows, kCols, kKStage>(jobs, T, total, li, tl, jc)) {
                const unsigned char *ma = maps + (size_t)tl.J->map * 2u * 128u, *mb = ma + 128;
                for (uint32_t k = 0; k < tl.ks; ++k) {
                    if (!mbar_wait(&empty[stage], ph ^ 1u)) { to = true; break; }
                    unsigned char *sa = base + (size_t)stage * kStageN, *sb = sa + (PAIR ? 2u : 1u) * kABytes;
                    arrive_expect_tx(&full[stage], kStageN);
                    tma_load(sa, ma, (int32_t)(k * 128u), (int32_t)tl.m0, &full[stage]);
                    if (PAIR) tma_load(sa + kABytes, ma, (int32_t)(k * 128u), (int32_t)(tl.m0 + 128u), &full[stage]);
                    tma_load(sb, mb, (int32_t)(k * 128u), (int32_t)tl.n0, &full[stage]);
                    if (++stage == (uint32_t)kRingN) { stage = 0; ph ^= 1u; }
                }
                li += gridDim.x;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            uint32_t stage = 0, ph = 0, acc = 0, aph = 0, li = blockIdx.x;
            Tile tl;
            JobCache jc;
            while (!to && next_tile<kRows, kCols, kKStage>(jobs, T, total, li, tl, jc)) {
                if (!mbar_wait(&tempty[acc], aph ^ 1u)) { to = true; break; }
                tc_after();
                const uint32_t d = tmem + acc * 256u;
                for (uint32_t k = 0; k < tl.ks; ++k) {
                    if (!mbar_wait(&full[stage], ph)) { to = true; break; }
                    tc_after();
                    const uint32_t sa = smem_u32(base + (size_t)stage * kStageN);
                    const uint32_t sb = sa + (PAIR ? 2u : 1u) * kABytes;
#pragma unroll
                    for (uint32_t kk = 0; kk < 4; ++kk) {
                        // 32 bytes of each operand row per MMA: K = 32 FP8 or 64 E2M1
                        const uint32_t accum = (k > 0 || kk > 0) ? 1u : 0u;
                        if constexpr (FP4) {
                            tc::mma_fp4<NV>(d, desc_sw128(sa + kk * 32u), desc_sw128(sb + kk * 32u), idesc, tmem + kSfa,
                                        tmem + kSfb, accum);
                            tc::mma_fp4<NV>(d + 256u, desc_sw128(sa + kABytes + kk * 32u), desc_sw128(sb + kk * 32u),
                                        idesc, tmem + kSfa, tmem + kSfb, accum);
                        } else {
                            tc::mma(false, d, desc_sw128(sa + kk * 32u), desc_sw128(sb + kk * 32u), idesc, accum);
                            if (PAIR)  // rows m0 + 128 .. into the second accumulator
                                tc::mma(false, d + 256u, desc_sw128(sa + kABytes + kk * 32u),
                                        desc_sw128(sb + kk * 32u), idesc, accum);
                        }
                    }
                    mma_commit(&empty[stage]);  // the stage is free once these MMAs have read it
                    if (++stage == (uint32_t)kRingN) { stage = 0; ph ^= 1u; }
                }
                if (to) break;
                mma_commit(&tfull[acc]);
                QCtl *cw = tl.J->ctl;
                if (cw) {
                    // counted in 128 x 256 tiles and 128 x 256 x 128 stages (an
                    // FP4 pair stage, 2 x 128 x 192 x 256, is three of those)
                    atomicAdd(&cw->tile_mmas, PAIR ? 2ull : 1ull);
                    atomicAdd(&cw->tile_kstages, (unsigned long long)tl.ks * (FP4 ? 3ull : PAIR ? 2ull : 1ull));
                }
                if (++acc == kBufs) { acc = 0; aph ^= 1u; }
                li += gridDim.x;
            }
        }
    } else if constexpr (FP4) {
        // epilogue: warps 2-5 read accumulator 0 (tile rows 0-127), warps 6-9
        // accumulator 1 (rows 128-255), each its TMEM lane quarter and all 192
        // columns (three output words per row)
        const uint32_t quarter = (uint32_t)warp & 3u, hh = (uint32_t)(warp - 2) >> 2;
        uint32_t aph = 0, li = blockIdx.x;
        Tile tl;
        JobCache jc;
        while (!to && next_tile<kRows, kCols, kKStage>(jobs, T, total, li, tl, jc)) {
            if (!mbar_wait(&tfull[0], aph)) { to = true; }
            if (__any_sync(0xffffffffu, to)) { to = true; break; }
            tc_after();
            const TcJob &J = *tl.J;
            // three 32-column loads in flight per wait: two waits per tile
            uint32_t mask[6];
#pragma unroll 1
            for (int c3 = 0; c3 < 6; c3 += 3) {
                uint32_t v[3][32];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    tmem_ld32_nowait(tmem + hh * 256u + 32u * (uint32_t)(c3 + c) + ((quarter * 32u) << 16), v[c]);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    uint32_t mb = 0u;
#pragma unroll
                    for (int i = 0; i < 32; ++i) mb |= (v[c][i] != 0u ? 1u : 0u) << i;
#pragma unroll
                    for (int cc = 0; cc < 6; ++cc)  // (constant indices keep mask in registers)
                        if (cc == c3 + c) mask[cc] = mb;
                }
            }
            tc_before();
            __syncwarp();
            if (lane == 0) arrive(&tempty[0]);  // the accumulators may be overwritten
            const uint32_t r = quarter * 32u + (uint32_t)lane, mr = tl.m0 + 128u * hh + r;
            const uint32_t x = mr >= tl.mlim ? J.n : (J.covers_new ? J.xs[mr] : mr);
            bool ch = false;
            if (x < J.n) {
                // read the three output words first and OR only those that
                // gain a bit (the bits of a block are only ever set, so a
                // stale read costs at most a redundant atomic): after the
                // first passes most products add nothing new
                uint64_t add[3], cur[3];
#pragma unroll
                for (int w = 0; w < 3; ++w) {
                    const uint32_t ww = (tl.n0 >> 6) + (uint32_t)w, z = ww * 64u;
                    add[w] = (uint64_t)mask[2 * w] | ((uint64_t)mask[2 * w + 1] << 32);
                    if (z < jc.c0 || z >= jc.c1 || ww >= J.W) add[w] = 0ull;  // another rank's columns; past the row
                    cur[w] = add[w] ? __ldcg(reinterpret_cast<const unsigned long long *>(J.out + (size_t)x * J.W + ww))
                                    : 0ull;
                }
#pragma unroll
                for (int w = 0; w < 3; ++w) {
                    if (!(add[w] & ~cur[w])) continue;
                    const uint32_t ww = (tl.n0 >> 6) + (uint32_t)w;
                    const uint64_t old = atomicOr(
                        reinterpret_cast<unsigned long long *>(J.out + (size_t)x * J.W + ww), (unsigned long long)add[w]);
                    if (add[w] & ~old) ch = true;
                }
            }
            if (ch && J.out_stamp) J.out_stamp[x] = tl.g;
            const unsigned chb = __ballot_sync(0xffffffffu, ch);
            if (lane == 0 && chb) {
                if (J.out_last) *J.out_last = tl.g;
                if (J.ctl) atomicAdd(&J.ctl->changed_rows, (unsigned long long)__popc(chb));
            }
            aph ^= 1u;
            li += gridDim.x;
        }
    } else {  // epilogue: warps 2-9; TMEM lanes 32 * (warp % 4) ..., columns half * 128 ...
        const uint32_t quarter = (uint32_t)warp & 3u, half = (uint32_t)(warp - 2) >> 2;
        constexpr int kHalves = PAIR ? 2 : 1;  // 128-row halves of the tile
        uint32_t acc = 0, aph = 0, li = blockIdx.x;
        Tile tl;
        JobCache jc;
        while (!to && next_tile<kRows>(jobs, T, total, li, tl, jc)) {
            if (!mbar_wait(&tfull[acc], aph)) { to = true; }
            if (__any_sync(0xffffffffu, to)) { to = true; break; }
            tc_after();
            const TcJob &J = *tl.J;
            uint32_t mask[kHalves][4];
#pragma unroll
            for (int hh = 0; hh < kHalves; ++hh) {
#pragma unroll 1
                for (int c = 0; c < 4; ++c) {
                    uint32_t v[32];
                    tmem_ld32(tmem + acc * 256u + (uint32_t)hh * 256u + half * 128u + 32u * (uint32_t)c +
                                  ((quarter * 32u) << 16),
                              v);
                    uint32_t mb = 0u;
#pragma unroll
                    for (int i = 0; i < 32; ++i) mb |= (v[i] != 0u ? 1u : 0u) << i;
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc)
                        if (cc == c) mask[hh][cc] = mb;
                }
            }
            tc_before();
            __syncwarp();
            if (lane == 0) arrive(&tempty[acc]);  // the accumulators may be overwritten
#pragma unroll
            for (int hh = 0; hh < kHalves; ++hh) {
                // output row: tile row m0 + 128 hh + r, through xs for a channel-1 job
                const uint32_t r = quarter * 32u + (uint32_t)lane, mr = tl.m0 + 128u * (uint32_t)hh + r;
                const uint32_t x = mr >= tl.mlim ? J.n : (J.covers_new ? J.xs[mr] : mr);
                bool ch = false;
                if (x < J.n) {
                    const uint32_t w0 = (tl.n0 >> 6) + half * 2u;
                    // (read first, OR only the words that gain a bit: as in the E2M1 epilogue)
                    uint64_t add[2], cur[2];
#pragma unroll
                    for (int w = 0; w < 2; ++w) {
                        const uint32_t ww = w0 + (uint32_t)w;
                        add[w] = ww < J.W ? ((uint64_t)mask[hh][2 * w] | ((uint64_t)mask[hh][2 * w + 1] << 32)) : 0ull;
                        cur[w] = add[w] ? __ldcg(reinterpret_cast<const unsigned long long *>(J.out + (size_t)x * J.W + ww))
                                        : 0ull;
                    }
#pragma unroll
                    for (int w = 0; w < 2; ++w) {
                        if (!(add[w] & ~cur[w])) continue;
                        const uint64_t old = atomicOr(
                            reinterpret_cast<unsigned long long *>(J.out + (size_t)x * J.W + w0 + (uint32_t)w),
                            (unsigned long long)add[w]);
                        if (add[w] & ~old) ch = true;
                    }
                }
                if (ch && J.out_stamp) J.out_stamp[x] = tl.g;  // both column halves may stamp: same value
                const unsigned chb = __ballot_sync(0xffffffffu, ch);
                if (lane == 0 && chb) {
                    if (J.out_last) *J.out_last = tl.g;
                    if (J.ctl) atomicAdd(&J.ctl->changed_rows, (unsigned long long)__popc(chb));
                }
            }
            if (++acc == kBufs) { acc = 0; aph ^= 1u; }
            li += gridDim.x;
        }
    }
    if (to) atomicOr(err_flag, 1);
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0) tmem_dealloc(tmem, tc2::kTmemCols);
}

// 256-row tiles (two accumulators) in the TMA-fed FP8 products: Dyck-4
// n = 65536 tile products 852 -> 762 ms, the query 1.49 -> 1.41 s (128-row
// tiles with double-buffered accumulators: the kernel with PAIR = false,
// tile kind kTileFp8Single).  The autotuner times all three kernels.

// Dynamic shared memory of k_tc_product_tma<PAIR, FP4>: its stage ring and
// 1024 bytes of alignment.
constexpr uint32_t tma_smem_bytes(bool pair, bool fp4) {
    return (fp4 ? 4u * (2u * tc2::kABytes + 192u * 128u)
                : pair ? 3u * (2u * tc2::kABytes + tc2::kBBytes) : (uint32_t)tc2::kRing * tc2::kStage) +
           1024u;
}

static int g_tc_sms[64];

int tc_smem_bytes() { return 2 * tc::kStageBytes; }

// Persistent launch: at most two CTAs per SM (96 KiB of shared memory and 256
// TMEM columns each), walking the live tiles of the pass.


// Set the kernel's shared-memory limit and record the SM count (call outside
// any stream capture).
cudaError_t prepare_tc_launch() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (g_tc_sms[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(k_tc_product, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem_bytes());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tc_a8, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kColMaxW * 8u * (256u / 32u)));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tc_product_tma<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tma_smem_bytes(true, false));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tc_product_tma<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tma_smem_bytes(false, false));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tc_product_tma<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tma_smem_bytes(true, true));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tc_product_tma<true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tma_smem_bytes(true, true));
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_tc_sms[dev] = sms;
    return cudaSuccess;
}

cudaError_t launch_tc_product(bool int8, const TcJob *jobs, uint32_t max_tiles, const ExecTables &T, int *err_flag,
                              cudaStream_t st) {
    if (max_tiles == 0) return cudaSuccess;
    if (int8) return cudaErrorNotSupported;
    const int smem = tc_smem_bytes();
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = (dev >= 0 && dev < 64 && g_tc_sms[dev]) ? g_tc_sms[dev] : 0;
    if (!sms) return cudaErrorNotReady;  // prepare_tc_launch was not called
    uint32_t grid = (uint32_t)sms * 2u;
    if (max_tiles < grid) grid = max_tiles;
    k_tc_product<<<grid, tc::kThreads, smem, st>>>(jobs, T, err_flag);
    return cudaGetLastError();
}

cudaError_t launch_tc_compact(const TcJob *jobs, const ExecTables &T, uint32_t max_w, int *err_flag, cudaStream_t st) {
    if (max_w == 0) return cudaSuccess;
    if (max_w > kColMaxW) return cudaErrorInvalidValue;
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = (dev >= 0 && dev < 64 && g_tc_sms[dev]) ? g_tc_sms[dev] : 0;
    if (!sms) return cudaErrorNotReady;  // prepare_tc_launch was not called
    k_tc_newcols<<<(unsigned)sms * 2u, 256, 0, st>>>(jobs, T);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tc_rows<<<(unsigned)sms * 4u, 256, 0, st>>>(jobs, T, err_flag);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tc_a8<<<(unsigned)sms * 4u, 256, (size_t)max_w * 8u * 8u, st>>>(jobs, T, max_w);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tc_b8<<<(unsigned)sms * 8u, 256, 0, st>>>(jobs, T);
    return cudaGetLastError();
}

cudaError_t launch_tc_product_tma(const TcJob *jobs, const void *maps, uint32_t max_tiles, const ExecTables &T,
                                  int *err_flag, cudaStream_t st, uint32_t tile_kind) {
    if (max_tiles == 0 || maps == nullptr) return cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = (dev >= 0 && dev < 64 && g_tc_sms[dev]) ? g_tc_sms[dev] : 0;
    if (!sms) return cudaErrorNotReady;  // prepare_tc_launch was not called
    uint32_t grid = (uint32_t)sms;  // one CTA per SM: the ring and both accumulators fill it
    if (max_tiles < grid) grid = max_tiles;
    const unsigned char *mp = static_cast<const unsigned char *>(maps);
    if (tile_kind == kTileFp4Pair)
        k_tc_product_tma<true, true><<<grid, tc2::kThreads, tma_smem_bytes(true, true), st>>>(jobs, mp, T, err_flag);
    else if (tile_kind == kTileFp4NvPair)
        k_tc_product_tma<true, true, true><<<grid, tc2::kThreads, tma_smem_bytes(true, true), st>>>(jobs, mp, T,
                                                                                                    err_flag);
    else if (tile_kind == kTileFp8Single)
        k_tc_product_tma<false, false><<<grid, tc2::kThreads, tma_smem_bytes(false, false), st>>>(jobs, mp, T,
                                                                                                  err_flag);
    else
        k_tc_product_tma<true, false><<<grid, tc2::kThreads, tma_smem_bytes(true, false), st>>>(jobs, mp, T, err_flag);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(uint64_t limit_ns, int *timed_out, cudaStream_t st) {
    tc::k_wait_selftest<<<1, 32, 0, st>>>(limit_ns, timed_out);
    return cudaGetLastError();
}

static_assert(sizeof(CUtensorMap) == 128, "the product kernel indexes tensor maps in 128-byte steps");
size_t tc_map_bytes() { return sizeof(CUtensorMap); }

// a8: kstride x n bytes, box 128 x 128; b8: kstride x n_pad bytes, box 128 x
// 256 (FP4 jobs: 128 x 192, the tile's columns); both UINT8 with the
// 128-byte swizzle (the K-major layout the MMA reads; an E2M1 byte holds two
// elements).
cudaError_t tc_encode_maps(const TcJob *jobs, uint32_t n_jobs, void *out) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult qr;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
        if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    CUtensorMap *m = static_cast<CUtensorMap *>(out);
    for (uint32_t j = 0; j < n_jobs; ++j) {
        const TcJob &J = jobs[j];
        if (!J.ys) continue;
        const cuuint64_t dims_a[2] = {J.kstride, J.n}, dims_b[2] = {J.kstride, (cuuint64_t)J.W * 64u};
        const cuuint64_t stride[1] = {J.kstride};
        const cuuint32_t box_a[2] = {128u, 128u}, box_b[2] = {128u, J.fp4 ? 192u : 256u}, es[2] = {1u, 1u};
        CUresult r = encode(&m[2 * J.map], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, J.a8, dims_a, stride, box_a, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        r = encode(&m[2 * J.map + 1], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, J.b8, dims_b, stride, box_b, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

size_t tc_job_size() { return sizeof(TcJob); }

}  // namespace cfpq

// ---------------------------------------------------------------------------
// Standalone product (building block, testable on its own).
// ---------------------------------------------------------------------------
#include "../../include/cfpq.h"

extern "C" int cfpq_tc_bool_product(uint32_t n, int use_int8, const uint64_t *a, const uint64_t *b, uint64_t *c,
                                    void *stream) {
    using namespace cfpq;
    if (n == 0 || !a || !b || !c || n > 65536) return CFPQ_ERR_INVALID_ARG;
    if (use_int8) return CFPQ_ERR_UNSUPPORTED;  // no kind::i8 tensor-core MMA on sm_103a
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t n_pad = (n + 127u) & ~127u, W = n_pad / 64u;
    const size_t wn = (n + 63) / 64, bytes = (size_t)n * W * 8;
    uint64_t *dA = nullptr, *dB = nullptr, *dC = nullptr;
    TcJob *dJ = nullptr;
    int *dErr = nullptr;
    uint32_t *dTab = nullptr;
    int rc = CFPQ_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == CFPQ_OK) rc = CFPQ_ERR_CUDA;
        return e == cudaSuccess;
    };
    if (ck(cudaMallocAsync((void **)&dA, bytes, st)) && ck(cudaMallocAsync((void **)&dB, bytes, st)) &&
        ck(cudaMallocAsync((void **)&dC, bytes, st)) && ck(cudaMallocAsync((void **)&dJ, sizeof(TcJob), st)) &&
        ck(cudaMallocAsync((void **)&dErr, sizeof(int), st)) && ck(cudaMallocAsync((void **)&dTab, 16, st))) {
        ck(cudaMemsetAsync(dA, 0, bytes, st));
        ck(cudaMemsetAsync(dB, 0, bytes, st));
        ck(cudaMemsetAsync(dC, 0, bytes, st));
        ck(cudaMemsetAsync(dErr, 0, sizeof(int), st));
        ck(cudaMemcpy2DAsync(dA, W * 8, a, wn * 8, wn * 8, n, cudaMemcpyHostToDevice, st));
        ck(cudaMemcpy2DAsync(dB, W * 8, b, wn * 8, wn * 8, n, cudaMemcpyHostToDevice, st));
        TcJob j;
        memset(&j, 0, sizeof(j));
        j.out = dC;
        j.A = dA;
        j.B = dB;
        j.n = n;
        j.W = W;
        j.tiles_m = (n + 127) / 128;
        j.tiles_n = (n_pad + 255) / 256;
        j.tile0 = 0;
        ck(cudaMemcpyAsync(dJ, &j, sizeof(j), cudaMemcpyHostToDevice, st));
        // one query, one live job: t_total, t_pre, t_job_beg, t_job_end
        const uint32_t tab[4] = {j.tiles_m * j.tiles_n, 0u, 0u, 1u};
        ck(cudaMemcpyAsync(dTab, tab, sizeof(tab), cudaMemcpyHostToDevice, st));
        ExecTables T;
        memset(&T, 0, sizeof(T));
        T.nq = 1;
        T.t_total = dTab;
        T.t_pre = dTab + 1;
        T.t_job_beg = dTab + 2;
        T.t_job_end = dTab + 3;
        ck(prepare_tc_launch());
        ck(launch_tc_product(use_int8 != 0, dJ, tab[0], T, dErr, st));
        int herr = 0;
        ck(cudaMemcpyAsync(&herr, dErr, sizeof(int), cudaMemcpyDeviceToHost, st));
        ck(cudaMemcpy2DAsync(c, wn * 8, dC, W * 8, wn * 8, n, cudaMemcpyDeviceToHost, st));
        ck(cudaStreamSynchronize(st));
        if (rc == CFPQ_OK && herr) rc = CFPQ_ERR_TIMEOUT;
    }
    if (dA) cudaFreeAsync(dA, st);
    if (dB) cudaFreeAsync(dB, st);
    if (dC) cudaFreeAsync(dC, st);
    if (dJ) cudaFreeAsync(dJ, st);
    if (dErr) cudaFreeAsync(dErr, st);
    if (dTab) cudaFreeAsync(dTab, st);
    cudaStreamSynchronize(st);
    return rc;
}
