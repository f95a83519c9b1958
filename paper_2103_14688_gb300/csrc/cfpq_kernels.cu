// cfpq_kernels.cu -- CUDA kernels of libcfpq for sm_103a.
//
// The index-creation loop of Listing 1 (arXiv 2103.14688, Sec. 3.1) runs as
// passes of three kernels, all driven by per-query control words in device
// memory (QCtl):
//   k_gather   one closure pass.  For every output block C[s,t] and row x it
//              ORs, over the product edges (s,x) -> (u,y) generated on the fly
//              from the RSM transitions s -l-> u and the graph edges (x,y) of
//              M2^l (the Kronecker product M1 (x) M2, never materialised), the
//              row (I + C)[u,t][y].  The first pass of an iteration uses only
//              the new edges A2 (left-distributivity, Sec. 3.1.1) with whole
//              source rows; later passes use all edges but only source rows
//              whose dirty stamp says they changed in the previous pass (the
//              incremental closure of Sec. 3.1.1 recomputes only what the new
//              edges reach).
//   k_extract  after a pass that changed nothing: for every box b and final f
//              of b, new = C[q0_b, f] & ~M2^b on the rows changed in this
//              iteration; M2^b |= new; A2^b = new (Listing 1, extraction via
//              getStates/getCoordinates).
//   k_control  advances each query's loop state and sets the CUDA-graph
//              conditional (Listing 1: "while M2 is changing").
#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>

#include "cfpq_dev.cuh"

namespace cfpq {

#define FULLMASK 0xffffffffu

__device__ __forceinline__ bool nz4(const uint4 &v) { return (v.x | v.y | v.z | v.w) != 0u; }
__device__ __forceinline__ void or4(uint4 &a, const uint4 &b) {
    a.x |= b.x; a.y |= b.y; a.z |= b.z; a.w |= b.w;
}
__device__ __forceinline__ uint4 andnot4(const uint4 &a, const uint4 &b) {
    return make_uint4(a.x & ~b.x, a.y & ~b.y, a.z & ~b.z, a.w & ~b.w);
}
__device__ __forceinline__ int popc4(const uint4 &v) {
    return __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
}

// Set bit `pos` (0..127) of a 128-bit vector.
__device__ __forceinline__ void setbit4(uint4 &v, uint32_t pos) {
    const uint32_t m = 1u << (pos & 31);
    switch ((pos >> 5) & 3) {
        case 0: v.x |= m; break;
        case 1: v.y |= m; break;
        case 2: v.z |= m; break;
        default: v.w |= m; break;
    }
}

// Set bit z of a row held by a group of lpr lanes (lane gl holds the 128-bit
// vectors gl, gl + lpr, ...).
template <int VPL>
__device__ __forceinline__ void set_row_bit(uint4 (&acc)[VPL], uint32_t z, int lpr, int gl) {
    const uint32_t v = z >> 7;
    if ((int)(v % (uint32_t)lpr) == gl) {
        const int j = (int)(v / (uint32_t)lpr);
#pragma unroll
        for (int jj = 0; jj < VPL; ++jj)
            if (jj == j) setbit4(acc[jj], z & 127u);
    }
}

// OR rows of a pure-terminal block (see SrcDesc::pure_n) into the group's
// row: every lane with keep_l expands its own source row y_l (the columns of
// y_l's CSR rows under the block's labels, all lanes' loads in flight at
// once), and each column found is passed by shuffle to the lane that holds
// its bit.  Called by all lanes of the warp.
template <int VPL>
__device__ __forceinline__ void or_pure_rows(uint4 (&acc)[VPL], const SrcDesc &d, uint32_t y_l, bool keep_l,
                                             int lpr, int gl, int grp, unsigned gmask) {
    uint32_t e0 = 0, e1 = 0, f0 = 0, f1 = 0;
    if (keep_l) {
        e0 = d.pure_off[0][y_l];
        e1 = d.pure_off[0][y_l + 1];
        if (d.pure_n > 1) {
            f0 = d.pure_off[1][y_l];
            f1 = d.pure_off[1][y_l + 1];
        }
    }
    while (true) {
        bool has = false;
        uint32_t z = 0;
        if (e0 < e1) {
            z = d.pure_col[e0++];
            has = true;
        } else if (f0 < f1) {
            z = d.pure_col[f0++];
            has = true;
        }
        const unsigned bal = __ballot_sync(FULLMASK, has);
        if (!bal) break;
        unsigned mine = (bal & gmask) >> (grp * lpr);
        while (__any_sync(FULLMASK, mine != 0u)) {
            const bool h = mine != 0u;
            const int src = h ? __ffs(mine) - 1 : 0;
            if (h) mine &= mine - 1u;
            const uint32_t zz = __shfl_sync(FULLMASK, z, src, lpr);
            if (h) set_row_bit<VPL>(acc, zz, lpr, gl);
        }
    }
}

// Asynchronous 16-byte global -> shared copy (zero-filled when !valid); the
// copies of a thread form groups it can wait for.
__device__ __forceinline__ void cp_async16(uint4 *dst, const void *src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Source rows a warp of the general gather keeps in flight (shared-memory
// ring), for rows of 4+ vectors per lane where registers allow only one row
// load at a time; narrower rows batch their loads in registers.
template <int VPL>
struct GatherRing {
    static constexpr bool on = VPL >= 4;
    static constexpr int depth = VPL <= 8 ? 4 : 3;
    // narrower rows keep one row-sized slot per warp: the bitmap of
    // pure-terminal reads (pure_bitmap_*)
    static constexpr int slots = on ? depth : 1;
    static constexpr size_t bytes = (size_t)8 * slots * 32 * VPL * 16;  // 8 warps
};

// The same for a warp that owns one row (lpr = 32, rows of 4+ vectors per
// lane), with a row-sized shared-memory bitmap `bm` (uint4-aligned, the
// vectors in row order): the bitmap is cleared once per row and source, every
// lane sets the columns it finds with a shared atomic -- no broadcast -- for
// every candidate of the enumeration, and the bitmap is ORed into the
// accumulators once at the end.
template <int VPL>
__device__ __forceinline__ void pure_bitmap_clear(uint32_t nvec, int lane, uint4 *bm) {
#pragma unroll
    for (int j = 0; j < VPL; ++j) {
        const uint32_t v = (uint32_t)lane + 32u * (uint32_t)j;
        if (v < nvec) bm[v] = make_uint4(0, 0, 0, 0);
    }
    __syncwarp();
}

__device__ __forceinline__ void pure_bitmap_set(const SrcDesc &d, uint32_t y_l, bool keep_l, uint4 *bm) {
    if (!keep_l) return;
    unsigned int *w = reinterpret_cast<unsigned int *>(bm);
    for (uint32_t p = 0; p < d.pure_n; ++p) {
        const uint32_t *off = d.pure_off[p];
        const uint32_t e1 = off[y_l + 1];
        for (uint32_t e = off[y_l]; e < e1; ++e) {
            const uint32_t z = d.pure_col[e];
            atomicOr(w + (z >> 5), 1u << (z & 31u));
        }
    }
}

template <int VPL>
__device__ __forceinline__ void pure_bitmap_or(uint4 (&acc)[VPL], uint32_t nvec, int lane, const uint4 *bm) {
    __syncwarp();
#pragma unroll
    for (int j = 0; j < VPL; ++j) {
        const uint32_t v = (uint32_t)lane + 32u * (uint32_t)j;
        if (v < nvec) or4(acc[j], bm[v]);
    }
    __syncwarp();  // the bitmap (a ring slot) is reused afterwards
}

// Lowest set bit of a 128-bit vector, -1 if none; clears it when `clear`.
__device__ __forceinline__ int lowbit4(uint4 &v, bool clear) {
    if (v.x) { int b = __ffs(v.x) - 1; if (clear) v.x &= v.x - 1; return b; }
    if (v.y) { int b = __ffs(v.y) - 1; if (clear) v.y &= v.y - 1; return 32 + b; }
    if (v.z) { int b = __ffs(v.z) - 1; if (clear) v.z &= v.z - 1; return 64 + b; }
    if (v.w) { int b = __ffs(v.w) - 1; if (clear) v.w &= v.w - 1; return 96 + b; }
    return -1;
}

// Which edges of a source take part in this pass (bit mask):
//   1  new edges of the iteration, whole source rows (FIRST pass): terminal
//      edges in iteration 1, A2 rows afterwards (left-distributivity);
//   2  all edges, source rows of a lower level changed in this iteration
//      (FIRST pass; those levels are final for the iteration);
//   4  all edges, source rows of this level changed in the previous pass
//      (REPEAT pass of a cyclic level).
// Channels 2 and 4 of a tensor-core source (and of a switchable source while
// its box is dense) run as tile products over the dirty rows instead.  When
// the source's channel-1 tile job (SrcDesc::tile_new) runs in this pass,
// channel 1's row ORs go to the tiles too: the result keeps channel 1 only
// for the product edges themselves (ident), flagged by bit 8 (read no
// closure rows).
template <bool NT>
__device__ __forceinline__ uint32_t src_channels(const SrcDesc &d, uint32_t mode, uint32_t iter, uint32_t g,
                                                 uint32_t g0, uint32_t dense_mask) {
    const bool tiles = d.dense || (d.box_switch && d.csr_off == nullptr && d.label_box < 32u &&
                                   ((dense_mask >> d.label_box) & 1u));
    uint32_t ch = 0u;
    if (mode == kModeNew) {
        const bool term1 = d.csr_off != nullptr && iter == 1;
        if (term1 || (d.csr_off == nullptr && *d.box_new_it == iter)) ch |= 1u;
        if (d.rblk && !d.same_level && !term1 && *d.rlast >= g0) ch |= 2u;
    } else {
        if (d.rblk && d.same_level && *d.rlast + 1u >= g) ch |= 4u;
    }
    if (!tiles) return ch;
    ch &= 1u;
    if (NT && ch && d.tile_new && d.tc_kcount) {
        const unsigned long long kc = *reinterpret_cast<const volatile unsigned long long *>(d.tc_kcount);
        const uint32_t listed = ((uint32_t)(kc >> 32) == g) ? (uint32_t)kc : 0u;
        if (new_tiles_pay(listed, d.tc_kcap, *d.tc_mcount, *d.tc_ecount, d.tc_ratio)) ch = d.ident ? 9u : 0u;
    }
    return ch;
}

// --------------------------------------------------------------------------
// Closure pass (bit-packed rows).  One CTA of 8 warps per work item; a row is
// handled by a group of `lpr` lanes, each lane holding VPL 128-bit vectors
// (words 2v, 2v+1 for v = lane_in_group + j * lpr).  NT selects the general
// variant (nonterminal adjacency rows, pure-terminal blocks); without it the
// kernel holds only the CSR paths, which keeps its registers for the rows.
// --------------------------------------------------------------------------
// Occupancy target per row width: narrow rows keep 4 CTAs (32 warps) per SM.
template <int VPL>
struct GatherOcc {
    static constexpr int value = VPL <= 2 ? 4 : (VPL == 4 ? 2 : 1);
};

// Scheduling.  Narrow rows: one CTA per live item (the grid covers every
// item of the class; CTAs past the live count exit at once).  Wide rows of
// the general variant (one warp per row, VPL >= 4, at most one or two CTAs
// per SM for the shared-memory ring): the grid is persistent and each warp
// takes units of kGatherParts row ranges of a live item from a counter of the
// pass (ExecTables::g_next, zeroed by the loop control), so that a warp held
// by a row with thousands of new edges leaves the other warps of its CTA free
// to take more work instead of waiting for it at a barrier.
template <int VPL, bool NT>
struct GatherDyn {
    static constexpr bool on = NT && VPL >= 4;
};
// Units per item: measured on Dyck-4 (AUTO / bit-packed, ms) at n = 65536:
// 4: 1545 / 2707, 8: 1543 / 2589, 16: 1560 / 2564, 32: 1585 / 2531; at
// n = 16384: 4: 58 / 84, 8: 50 / 71, 32: 50 / 62.  (Leaving rows with more
// than 256-4096 bits to enumerate to a second launch split over 16 warps
// gained 1-2% in AUTO and cost 10-20% bit-packed: not kept.)
constexpr uint32_t kGatherParts = 8;
constexpr uint32_t kStrideWaves = 8;  // launch_gather / launch_extract: waves of resident CTAs at most

template <int VPL, bool NT>
__global__ void __launch_bounds__(256, GatherOcc<VPL>::value)
    k_gather(const GItem *__restrict__ items, const SrcDesc *__restrict__ srcs, ExecTables T, int cls) {
    constexpr bool kDyn = GatherDyn<VPL, NT>::on;
    __shared__ unsigned long long s_changed, s_ors;
    // rows of the item to compute (multiple-source runs; else all): the item's
    // rows start at a multiple of 64 and number at most 1024, so its 16 mask
    // words have distinct indices modulo 16
    __shared__ unsigned long long s_rmask[16];
    // general variant: per-warp ring of source rows loaded with cp.async
    extern __shared__ uint4 s_ring[];
    constexpr int P = GatherRing<VPL>::depth;
    uint4 *ring = s_ring + (size_t)(threadIdx.x >> 5) * GatherRing<VPL>::slots * 32 * VPL;
    const uint32_t total = T.g_total[cls];
    uint32_t li = blockIdx.x;
    if (kDyn) li = 0u;
    for (bool first = true;; first = false) {
    uint32_t part = 0u;
    if constexpr (kDyn) {
        uint32_t u = 0u;
        if ((threadIdx.x & 31) == 0) u = atomicAdd(T.g_next + cls, 1u);
        u = __shfl_sync(FULLMASK, u, 0);
        if (u >= total * kGatherParts) break;
        li = u / kGatherParts;
        part = u % kGatherParts;
    } else {
        if (!first) li += gridDim.x;
        if (li >= total) break;
    }
    const uint32_t q = find_owner(T.g_pre[cls], T.nq, li);
    const GItem it = items[T.g_beg[cls][q] + (li - T.g_pre[cls][q])];
    const QCtl *c = it.ctl;
    if (c->phase != kPhaseRun || c->level != it.level) continue;
    const uint32_t g = c->g, iter = c->iter, mode = c->mode, g0 = c->g_iter_start, dmask = c->dense_mask;

    if constexpr (kDyn) {
        bool act = false;
        for (uint32_t k = threadIdx.x & 31; k < it.nsrc; k += 32u)
            act |= src_channels<NT>(srcs[it.src0 + k], mode, iter, g, g0, dmask) != 0u;
        if (!__any_sync(FULLMASK, act)) continue;
    } else {
        int act = 0;
        for (uint32_t k = threadIdx.x; k < it.nsrc; k += blockDim.x)
            act |= src_channels<NT>(srcs[it.src0 + k], mode, iter, g, g0, dmask) != 0u;
        if (!__syncthreads_or(act)) continue;

        if (threadIdx.x == 0) { s_changed = 0; s_ors = 0; }
        if (threadIdx.x < 16u) {
            const uint32_t wrow = it.row0 + threadIdx.x * 64u;
            s_rmask[(wrow >> 6) & 15u] = (it.rmask && wrow < it.row1) ? it.rmask[wrow >> 6] : ~0ull;
        }
        __syncthreads();
    }

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lpr = (int)it.lpr, grp = lane / lpr, gl = lane % lpr, rpw = 32 / lpr;
    const unsigned gmask = (lpr == 32 ? FULLMASK : ((1u << lpr) - 1u)) << (grp * lpr);
    const uint32_t W = it.W, nvec = W / 2;
    // the columns of the output this rank computes (column sharding; else
    // all): closure rows are read and written only there
    // (bit j of winmask: the lane's vector j lies in [col_v0, col_v1) and in the row)
    uint32_t winmask = 0u;
    {
        const uint32_t cv0 = c->col_v0, cv1 = min(c->col_v1, nvec);
#pragma unroll
        for (int j = 0; j < VPL; ++j) {
            const uint32_t v = (uint32_t)gl + (uint32_t)j * lpr;
            if (v >= cv0 && v < cv1) winmask |= 1u << j;
        }
    }
    // column slice of the nonterminal adjacency (general variant, rows of 2+
    // vectors per lane: the engine slices only rows of 8192+ bits)
    constexpr bool kSlices = NT && VPL >= 2;
    const bool slices_on = kSlices && (dmask & it.nt_boxes) != 0u;  // a box the block reads is dense
    uint32_t sv0 = kSlices ? (it.slice & 0xFFFFu) : 0u, sv1 = kSlices ? (it.slice >> 16) : nvec;
    if (kSlices && !slices_on) {
        if (sv0 != 0u) continue;  // the first slice covers every column
        sv1 = nvec;
    }
    const bool sliced = slices_on && (sv0 != 0u || sv1 < nvec);
    uint32_t my_changed = 0, my_ors = 0;
    // channels of the item's first 16 sources in this pass (4 bits each): the
    // same for every row of the unit
    unsigned long long chpack = 0ull;
    if constexpr (NT)
        for (uint32_t k = 0; k < it.nsrc && k < 16u; ++k)
            chpack |= (unsigned long long)src_channels<NT>(srcs[it.src0 + k], mode, iter, g, g0, dmask) << (4u * k);

    // rows of this warp: the unit's range of rpw-row steps (dynamic), or
    // every eighth step of the item (one CTA per item)
    uint32_t r_first = it.row0 + (uint32_t)(warp * rpw), r_end = it.row1, r_step = 8u * rpw;
    if constexpr (kDyn) {
        const uint32_t steps = (it.row1 - it.row0 + (uint32_t)rpw - 1u) / (uint32_t)rpw;
        const uint32_t per = (steps + kGatherParts - 1u) / kGatherParts;
        r_first = it.row0 + part * per * (uint32_t)rpw;
        r_end = min(it.row1, r_first + per * (uint32_t)rpw);
        r_step = (uint32_t)rpw;
    }
    // Rows with nothing to do: when every source taking part in the pass
    // reads only the iteration's new edges of a nonterminal (channel 1; the
    // late passes of Dyck-4's x_i and p levels), a row has work only if one
    // of those boxes has a new edge in it (its A2 stamp is this iteration),
    // so a warp that owns whole rows (dynamic units) jumps from one such row
    // to the next, 32 stamps per coalesced load, instead of visiting every
    // row and source.
    const uint32_t *skip_it[2] = {nullptr, nullptr};
    bool skip_rows = false;
    if constexpr (kDyn) {
        skip_rows = it.nsrc <= 16u;
        uint32_t ns = 0;
        for (uint32_t k = 0; k < it.nsrc && skip_rows; ++k) {
            const uint32_t chans = (uint32_t)(chpack >> (4u * k)) & 15u;
            if (!chans) continue;
            const SrcDesc &d = srcs[it.src0 + k];
            if ((chans & ~9u) != 0u || d.csr_off != nullptr || d.nt_new_it == nullptr) {
                skip_rows = false;
                break;
            }
            if (ns < 2u && (ns == 0u || skip_it[0] != d.nt_new_it)) skip_it[ns++] = d.nt_new_it;
            else if (skip_it[0] != d.nt_new_it && skip_it[1] != d.nt_new_it) skip_rows = false;
        }
        skip_rows = skip_rows && ns > 0u && lpr == 32;
    }
    for (uint32_t rbase = r_first; rbase < r_end; rbase += r_step) {
        if constexpr (kDyn) {
            if (skip_rows) {
                // the next row at or after rbase with a new edge in one of the boxes
                bool found = false;
                while (rbase < r_end) {
                    const uint32_t b32 = rbase & ~31u, r = b32 + (uint32_t)lane;
                    const bool w = r >= rbase && r < r_end &&
                                   (skip_it[0][r] == iter || (skip_it[1] != nullptr && skip_it[1][r] == iter));
                    const unsigned m = __ballot_sync(FULLMASK, w);
                    if (m) {
                        rbase = b32 + (uint32_t)(__ffs(m) - 1);
                        found = true;
                        break;
                    }
                    rbase = b32 + 32u;
                }
                if (!found) break;
            }
        }
        const uint32_t row = rbase + grp;
        bool valid = row < r_end;
        if constexpr (kDyn) valid = valid && (!it.rmask || ((it.rmask[row >> 6] >> (row & 63u)) & 1ull));
        else valid = valid && ((s_rmask[(row >> 6) & 15u] >> (row & 63u)) & 1ull);
        uint4 acc[VPL];
#pragma unroll
        for (int j = 0; j < VPL; ++j) acc[j] = make_uint4(0, 0, 0, 0);

        for (uint32_t k = 0; k < it.nsrc; ++k) {
            uint32_t chans;
            if constexpr (NT)
                chans = k < 16u ? (uint32_t)(chpack >> (4u * k)) & 15u
                                : src_channels<NT>(srcs[it.src0 + k], mode, iter, g, g0, dmask);
            else
                chans = src_channels<NT>(srcs[it.src0 + k], mode, iter, g, g0, dmask);
            if (!chans) continue;  // the source takes no part in this pass
            const SrcDesc d = srcs[it.src0 + k];
            // closure rows read by this source (none when the tiles OR them:
            // only the product edges themselves are left here)
            const uint64_t *const rblk = (NT && (chans & 8u)) ? nullptr : d.rblk;
            for (uint32_t cbit = 1u; cbit <= 4u; cbit <<= 1) {
                if (!(chans & cbit)) continue;
                const bool new_edges = cbit == 1u;
                const bool use_ident = new_edges && d.ident;
                if (!use_ident && rblk == nullptr) continue;
                // a source row takes part when its stamp is >= thr
                const uint32_t thr = new_edges ? 0u : (cbit == 2u ? g0 : g - 1u);

                // Every lane proposes one candidate edge (x, y) of its group's
                // row (y_l, has_l).  The group keeps those whose source row is
                // dirty, then ORs their rows U at a time: all U rows are loaded
                // before any is combined, so several 128-bit loads per lane are
                // in flight.
                constexpr int U = VPL >= 4 ? 1 : 4 / VPL;
                auto take_batch = [&](uint32_t y_l, bool has_l) {
                    const bool keep = has_l && (rblk == nullptr || thr == 0u || d.rstamp[y_l] >= thr);
                    if constexpr (NT) {
                        if (d.pure_n && !use_ident) {
                            if (lpr == 32) {  // one row per warp: the bitmap in the warp's first slot
                                pure_bitmap_set(d, y_l, keep, ring);
                                return;
                            }
                            or_pure_rows<VPL>(acc, d, y_l, keep, lpr, gl, grp, gmask);
                            return;
                        }
                        if (GatherRing<VPL>::on && rblk && !d.pure_n) {
                            // Rows through the warp's shared-memory ring, P in
                            // flight: row i is copied into slot i % P by
                            // cp.async (each lane its own 16-byte pieces, so a
                            // lane reads back only what it copied) and ORed
                            // once P - 1 later rows have been issued.
                            const unsigned bal = __ballot_sync(FULLMASK, keep);
                            unsigned mine = (bal & gmask) >> (grp * lpr);
                            uint32_t issued = 0, done = 0, vmask = 0;
                            auto or_slot = [&](uint32_t sidx) {
                                const uint4 *sl = ring + sidx * 32u * VPL;
#pragma unroll
                                for (int j = 0; j < VPL; ++j) or4(acc[j], sl[j * 32 + lane]);
                            };
                            while (__any_sync(FULLMASK, mine != 0u)) {
                                const bool h = mine != 0u;
                                const int pl = h ? __ffs(mine) - 1 : 0;
                                if (h) mine &= mine - 1u;
                                const uint32_t y = __shfl_sync(FULLMASK, y_l, pl, lpr);
                                if (use_ident && h) set_row_bit<VPL>(acc, y, lpr, gl);
                                const uint32_t sidx = issued % (uint32_t)P;
                                if (h) {
                                    uint4 *sl = ring + sidx * 32u * VPL;
                                    const uint4 *r = reinterpret_cast<const uint4 *>(rblk + (size_t)y * W);
#pragma unroll
                                    for (int j = 0; j < VPL; ++j) {
                                        const uint32_t v = (uint32_t)gl + (uint32_t)j * lpr;
                                        cp_async16(&sl[j * 32 + lane], r + (((winmask >> j) & 1u) ? v : 0u), ((winmask >> j) & 1u));
                                    }
                                    if (gl == 0) ++my_ors;
                                    vmask |= 1u << sidx;
                                } else {
                                    vmask &= ~(1u << sidx);
                                }
                                cp_async_commit();
                                ++issued;
                                if (issued - done == (uint32_t)P) {
                                    cp_async_wait<P - 1>();
                                    const uint32_t ds = done % (uint32_t)P;
                                    if ((vmask >> ds) & 1u) or_slot(ds);
                                    ++done;
                                }
                            }
                            cp_async_wait<0>();
                            for (; done < issued; ++done) {
                                const uint32_t ds = done % (uint32_t)P;
                                if ((vmask >> ds) & 1u) or_slot(ds);
                            }
                            return;
                        }
                    }
                    const unsigned bal = __ballot_sync(FULLMASK, keep);
                    unsigned mine = (bal & gmask) >> (grp * lpr);
                    while (__any_sync(FULLMASK, mine != 0u)) {
                        uint32_t ys[U];
                        bool hs[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            hs[u] = mine != 0u;
                            const int p = hs[u] ? __ffs(mine) - 1 : 0;
                            if (hs[u]) mine &= mine - 1u;
                            ys[u] = __shfl_sync(FULLMASK, y_l, p, lpr);
                        }
                        if (use_ident) {
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                if (!hs[u]) continue;
                                const uint32_t v = ys[u] >> 7;
                                if ((int)(v % lpr) == gl) {
                                    const int j = (int)(v / lpr);
#pragma unroll
                                    for (int jj = 0; jj < VPL; ++jj)
                                        if (jj == j) setbit4(acc[jj], ys[u] & 127u);
                                }
                            }
                        }
                        if (rblk && (!NT || !d.pure_n)) {
                            uint4 rv[U][VPL];
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                const uint4 *r = reinterpret_cast<const uint4 *>(rblk + (size_t)ys[u] * W);
#pragma unroll
                                for (int j = 0; j < VPL; ++j) {
                                    const uint32_t v = (uint32_t)gl + (uint32_t)j * lpr;
                                    rv[u][j] = (hs[u] && ((winmask >> j) & 1u)) ? r[v] : make_uint4(0, 0, 0, 0);
                                }
                            }
#pragma unroll
                            for (int u = 0; u < U; ++u) {
#pragma unroll
                                for (int j = 0; j < VPL; ++j) or4(acc[j], rv[u][j]);
                                if (gl == 0 && hs[u]) ++my_ors;
                            }
                        }
                    }
                };

                if (d.csr_off) {
                    if (sv0 != 0u) continue;  // CSR sources belong to the first slice
                    const uint32_t e0 = valid ? d.csr_off[row] : 0u, e1 = valid ? d.csr_off[row + 1] : 0u;
                    const uint32_t cnt = e1 - e0;
                    const uint32_t maxcnt = __reduce_max_sync(FULLMASK, cnt);
                    if (maxcnt <= 8u && (!NT || !d.pure_n)) {
                        // short adjacency rows (the common case on sparse
                        // graphs): no ballot; edges two at a time so that the
                        // column, stamp and row loads of both are in flight
                        auto ident_bit = [&](uint32_t y) {
                            const uint32_t v = y >> 7;
                            if ((int)(v % lpr) == gl) {
                                const int j = (int)(v / lpr);
#pragma unroll
                                for (int jj = 0; jj < VPL; ++jj)
                                    if (jj == j) setbit4(acc[jj], y & 127u);
                            }
                        };
                        for (uint32_t e = e0; e < e1; e += 2) {
                            const bool two = e + 1 < e1;
                            const uint32_t y0 = d.csr_col[e], y1 = two ? d.csr_col[e + 1] : 0u;
                            if (use_ident) {
                                ident_bit(y0);
                                if (two) ident_bit(y1);
                            }
                            if (rblk) {
                                const bool k0 = !thr || d.rstamp[y0] >= thr;
                                const bool k1 = two && (!thr || d.rstamp[y1] >= thr);
                                const uint4 *r0 = reinterpret_cast<const uint4 *>(rblk + (size_t)y0 * W);
                                const uint4 *r1 = reinterpret_cast<const uint4 *>(rblk + (size_t)y1 * W);
                                uint4 a0[VPL], a1[VPL];
#pragma unroll
                                for (int j = 0; j < VPL; ++j) {
                                    const uint32_t v = (uint32_t)gl + (uint32_t)j * lpr;
                                    a0[j] = (k0 && ((winmask >> j) & 1u)) ? r0[v] : make_uint4(0, 0, 0, 0);
                                    a1[j] = (k1 && ((winmask >> j) & 1u)) ? r1[v] : make_uint4(0, 0, 0, 0);
                                }
#pragma unroll
                                for (int j = 0; j < VPL; ++j) {
                                    or4(acc[j], a0[j]);
                                    or4(acc[j], a1[j]);
                                }
                                if (gl == 0) my_ors += (k0 ? 1u : 0u) + (k1 ? 1u : 0u);
                            }
                        }
                    } else {
                        for (uint32_t base = 0; base < maxcnt; base += (uint32_t)lpr) {
                            const uint32_t k2 = base + (uint32_t)gl;
                            const bool has = k2 < cnt;
                            const uint32_t y = has ? d.csr_col[e0 + k2] : 0u;
                            take_batch(y, has);
                        }
                    }
                } else if constexpr (NT) {
                    const uint64_t *adj;
                    bool rowok;
                    if (new_edges) { adj = d.nt_new; rowok = valid && d.nt_new_it[row] == iter; }
                    else { adj = d.nt_all; rowok = valid; }
                    // no row of the warp has edges of this channel: nothing to enumerate
                    if (!__any_sync(FULLMASK, rowok)) continue;
                    uint4 a[VPL];
#pragma unroll
                    for (int j = 0; j < VPL; ++j) {
                        const uint32_t v = (uint32_t)gl + (uint32_t)j * lpr;
                        a[j] = (rowok && v >= sv0 && v < sv1 && v < nvec)
                                   ? reinterpret_cast<const uint4 *>(adj + (size_t)row * W)[v]
                                   : make_uint4(0, 0, 0, 0);
                    }
                    if (d.pure_n) {
                        // a row y of a pure-terminal block is empty unless y
                        // has an edge of one of its labels
#pragma unroll
                        for (int j = 0; j < VPL; ++j) {
                            const uint32_t v = (uint32_t)gl + (uint32_t)j * lpr;
                            if (v >= nvec) continue;
                            uint4 m = reinterpret_cast<const uint4 *>(d.pure_mask[0])[v];
                            if (d.pure_n > 1) or4(m, reinterpret_cast<const uint4 *>(d.pure_mask[1])[v]);
                            a[j] = make_uint4(a[j].x & m.x, a[j].y & m.y, a[j].z & m.z, a[j].w & m.w);
                        }
                    }
                    if (use_ident) {
                        // product edges into t itself: bit y of the adjacency
                        // row is bit y of the output row, and the lane that
                        // holds an adjacency vector holds the same vector of
                        // the output row -- no enumeration
#pragma unroll
                        for (int j = 0; j < VPL; ++j) or4(acc[j], a[j]);
                        if (rblk == nullptr) continue;
                    }
                    // a pure-terminal block read by a warp-owned row: the
                    // columns found go to the row's shared-memory bitmap
                    const bool pure_bm = d.pure_n && !use_ident && lpr == 32;
                    if (pure_bm) pure_bitmap_clear<VPL>(nvec, lane, ring);
                    // Each lane proposes the lowest set bit of its part of the
                    // adjacency row per step (ballot/ffs enumeration).
                    while (true) {
                        bool has = false;
                        uint32_t y = 0u;
#pragma unroll
                        for (int j = 0; j < VPL; ++j) {
                            if (!has && nz4(a[j])) {
                                const int bit = lowbit4(a[j], true);
                                y = ((uint32_t)gl + (uint32_t)j * lpr) * 128u + (uint32_t)bit;
                                has = true;
                            }
                        }
                        if (!__any_sync(FULLMASK, has)) break;
                        take_batch(y, has);
                    }
                    if (pure_bm) pure_bitmap_or<VPL>(acc, nvec, lane, ring);
                }
            }
        }

        bool ch = false;
        if (valid && sliced) {
            // other slices write the same rows: merge with atomics
            unsigned long long *o = reinterpret_cast<unsigned long long *>(it.out + (size_t)row * W);
#pragma unroll
            for (int j = 0; j < VPL; ++j) {
                const uint32_t v = (uint32_t)gl + (uint32_t)j * lpr;
                if (((winmask >> j) & 1u) && nz4(acc[j])) {
                    const unsigned long long lo = ((unsigned long long)acc[j].y << 32) | acc[j].x;
                    const unsigned long long hi = ((unsigned long long)acc[j].w << 32) | acc[j].z;
                    if (lo && (lo & ~atomicOr(o + 2u * v, lo))) ch = true;
                    if (hi && (hi & ~atomicOr(o + 2u * v + 1u, hi))) ch = true;
                }
            }
        } else if (valid) {
            uint4 *o = reinterpret_cast<uint4 *>(it.out + (size_t)row * W);
#pragma unroll
            for (int j = 0; j < VPL; ++j) {
                const uint32_t v = (uint32_t)gl + (uint32_t)j * lpr;
                if (((winmask >> j) & 1u) && nz4(acc[j])) {
                    const uint4 old = o[v];
                    const uint4 nw = andnot4(acc[j], old);
                    if (nz4(nw)) {
                        uint4 m = old;
                        or4(m, nw);
                        o[v] = m;
                        ch = true;
                    }
                }
            }
        }
        const unsigned chb = __ballot_sync(FULLMASK, ch);
        if ((chb & gmask) && gl == 0) {
            it.out_stamp[row] = g;
            ++my_changed;
        }
    }
    if constexpr (kDyn) {
        const uint32_t wc = __reduce_add_sync(FULLMASK, my_changed), wo = __reduce_add_sync(FULLMASK, my_ors);
        if (lane == 0) {
            QCtl *cw = it.ctl;
            if (wc) {
                *it.out_last = g;
                atomicAdd(&cw->changed_rows, (unsigned long long)wc);
            }
            if (wo) atomicAdd(&cw->row_ors, (unsigned long long)wo);
        }
    } else {
        if (my_changed) atomicAdd(&s_changed, (unsigned long long)my_changed);
        if (my_ors) atomicAdd(&s_ors, (unsigned long long)my_ors);
        __syncthreads();
        if (threadIdx.x == 0) {
            QCtl *cw = it.ctl;
            if (s_changed) {
                *it.out_last = g;
                atomicAdd(&cw->changed_rows, s_changed);
            }
            if (s_ors) atomicAdd(&cw->row_ors, s_ors);
        }
        __syncthreads();
    }
    }
}

// --------------------------------------------------------------------------
// Extraction: runs for a query only after a pass that changed no row.
// --------------------------------------------------------------------------
__device__ void control_body(QCtl *const *ctls, uint32_t nq, QCtl *mirror, cudaGraphConditionalHandle handle,
                             int use_handle, int *running_out, const ExecTables &T, int advance);

// Control fused into the last extraction launch of a pass: the CTA that
// finishes last (counted with an atomic after a fence) runs control_body.
struct FusedControl {
    QCtl *const *ctls;
    QCtl *mirror;
    int *running_out;
    unsigned int *done_counter;
    cudaGraphConditionalHandle handle;
    uint32_t nq;
    int use_handle;
    int enabled;
};

template <int VPL>
__global__ void __launch_bounds__(256) k_extract(const XItem *__restrict__ items, const FDesc *__restrict__ fds,
                                                 ExecTables T, int cls, FusedControl FC) {
    __shared__ unsigned long long s_new;
    __shared__ int s_last;
    const uint32_t total = T.x_total[cls];
    for (uint32_t li = blockIdx.x; li < total; li += gridDim.x) {
    const uint32_t q = find_owner(T.x_pre[cls], T.nq, li);
    const XItem it = items[T.x_beg[cls][q] + (li - T.x_pre[cls][q])];
    const QCtl *c = it.ctl;
    if (c->phase != kPhaseRun) continue;
    // Extraction follows the last level's final pass: its FIRST pass when the
    // level is acyclic, else the first pass that changed no row.
    const bool cyc = (c->cyclic_mask >> c->level) & 1ull;
    if (c->level + 1 != c->n_levels || (cyc && c->changed_rows != 0ull)) continue;
    const uint32_t g0 = c->g_iter_start, iter = c->iter;
    if (threadIdx.x == 0) s_new = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lpr = (int)it.lpr, grp = lane / lpr, gl = lane % lpr, rpw = 32 / lpr;
    const unsigned gmask = (lpr == 32 ? FULLMASK : ((1u << lpr) - 1u)) << (grp * lpr);
    const uint32_t W = it.W, nvec = W / 2;
    const uint32_t cv0 = c->col_v0, cv1 = min(c->col_v1, nvec);  // this rank's columns (all unless sharded)
    uint32_t my_new = 0;
    for (uint32_t rbase = it.row0 + (uint32_t)(warp * rpw); rbase < it.row1; rbase += 8u * rpw) {
        const uint32_t row = rbase + grp;
        const bool valid = row < it.row1;
        uint4 acc[VPL];
#pragma unroll
        for (int j = 0; j < VPL; ++j) acc[j] = make_uint4(0, 0, 0, 0);
        bool any = false;
        for (uint32_t f = 0; f < it.nf; ++f) {
            const FDesc fd = fds[it.f0 + f];
            if (!valid || fd.stamp[row] < g0) continue;
            any = true;
            const uint4 *r = reinterpret_cast<const uint4 *>(fd.blk + (size_t)row * W);
#pragma unroll
            for (int j = 0; j < VPL; ++j) {
                const uint32_t v = (uint32_t)gl + (uint32_t)j * lpr;
                if (v >= cv0 && v < cv1) or4(acc[j], r[v]);
            }
        }
        bool has = false;
        if (any) {
            const uint4 *m = reinterpret_cast<const uint4 *>(it.m2 + (size_t)row * W);
#pragma unroll
            for (int j = 0; j < VPL; ++j) {
                const uint32_t v = (uint32_t)gl + (uint32_t)j * lpr;
                if (v >= cv0 && v < cv1) {
                    acc[j] = andnot4(acc[j], m[v]);
                    if (nz4(acc[j])) has = true;
                }
            }
        }
        const unsigned hb = __ballot_sync(FULLMASK, has);
        if (hb & gmask) {
            uint4 *m = reinterpret_cast<uint4 *>(it.m2 + (size_t)row * W);
            uint4 *a = reinterpret_cast<uint4 *>(it.a2 + (size_t)row * W);
#pragma unroll
            for (int j = 0; j < VPL; ++j) {
                const uint32_t v = (uint32_t)gl + (uint32_t)j * lpr;
                if (v >= cv0 && v < cv1) {
                    a[v] = acc[j];
                    if (nz4(acc[j])) {
                        uint4 mm = m[v];
                        or4(mm, acc[j]);
                        m[v] = mm;
                        my_new += (uint32_t)popc4(acc[j]);
                    }
                }
            }
            if (gl == 0) it.a2_it[row] = iter + 1;
        }
    }
    if (my_new) atomicAdd(&s_new, (unsigned long long)my_new);
    __syncthreads();
    if (threadIdx.x == 0 && s_new) {
        *it.box_new_it = iter + 1;
        atomicAdd(&it.ctl->new_edges, s_new);
        if (it.box_edges) atomicAdd(it.box_edges, s_new);
    }
    __syncthreads();
    }
    if (FC.enabled) {
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned int prev = atomicAdd(FC.done_counter, 1u);
            s_last = (prev == gridDim.x - 1) ? 1 : 0;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            if (threadIdx.x == 0) *FC.done_counter = 0u;
            control_body(FC.ctls, FC.nq, FC.mirror, FC.handle, FC.use_handle, FC.running_out, T, 1);
        }
    }
}

// --------------------------------------------------------------------------
// Loop control: one CTA for all queries.
// --------------------------------------------------------------------------
// Loop control for every query of the executor, run by one whole CTA (any
// size up to 1024 threads): advance each running query's state machine
// (unless `advance` is 0), then build the live lists of the next pass.
__device__ void control_body(QCtl *const *ctls, uint32_t nq, QCtl *mirror, cudaGraphConditionalHandle handle,
                             int use_handle, int *running_out, const ExecTables &T, int advance) {
    int running = 0;
    for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x) {
        QCtl &c = *ctls[q];
        if (c.phase != kPhaseRun || !advance) {
            running |= (c.phase == kPhaseRun);
            mirror[q] = c;
            continue;
        }
        c.passes += 1;
        c.rounds_total += 1;
        c.rows_changed_total += c.changed_rows;
        c.rounds_in_iter += 1;
        const bool cyc = (c.cyclic_mask >> c.level) & 1ull;
        if (cyc && c.changed_rows != 0ull) {
            // a cyclic level repeats until a pass changes nothing
            c.g += 1;
            c.mode = kModeProp;
            if (c.max_rounds && c.rounds_in_iter >= c.max_rounds) {
                c.status = kStatusRoundCap;
                c.phase = kPhaseDone;
            }
        } else if (c.level + 1 < c.n_levels) {
            c.level += 1;
            c.g += 1;
            c.mode = kModeNew;
        } else {
            // extraction ran in this pass: the iteration is complete
            c.iters_done = c.iter;
            c.edges_total += c.new_edges;
            if (c.box_edges) {
                const unsigned long long dense_at = (unsigned long long)c.n * c.n / kDenseDiv;
                uint32_t m = 0;
                for (uint32_t b = 0; b < c.n_boxes && b < 32u; ++b)
                    if (c.box_edges[b] >= dense_at && dense_at > 0ull) m |= 1u << b;
                c.dense_mask = m;
            }
            bool read_new = true;  // does some transition read a box that gained edges?
            if (c.box_new_it && c.n_boxes <= 63u && !((c.nt_read_mask >> 63) & 1ull)) {
                read_new = false;
                for (uint32_t b = 0; b < c.n_boxes; ++b)
                    if (((c.nt_read_mask >> b) & 1ull) && c.box_new_it[b] == c.iter + 1u) read_new = true;
            }
            if (c.shard) {
                // column sharding: whether the loop goes on depends on every
                // rank's new edges; pause at the next iteration's start until
                // they are installed (k_shard_apply, k_shard_finish)
                c.shard_new = c.new_edges;
                c.iter += 1;
                c.g += 1;
                c.level = 0;
                c.mode = kModeNew;
                c.g_iter_start = c.g;
                c.rounds_in_iter = 0;
                c.phase = kPhasePause;
            } else if (c.new_edges == 0ull) {
                c.phase = kPhaseDone;
            } else if (c.max_iter && c.iter >= c.max_iter) {
                c.status = kStatusIterCap;
                c.phase = kPhaseDone;
            } else if (!read_new) {
                // the next iteration's product equals this one's: it adds no
                // edge, so it is the last one and is counted without passes
                c.iters_done = c.iter + 1u;
                c.phase = kPhaseDone;
            } else {
                c.iter += 1;
                c.g += 1;
                c.level = 0;
                c.mode = kModeNew;
                c.g_iter_start = c.g;
                c.rounds_in_iter = 0;
            }
            c.new_edges = 0;
        }
        if (c.phase == kPhaseRun && c.passes >= c.max_passes) {
            c.status = kStatusPassCap;
            c.phase = kPhaseDone;
        }
        c.changed_rows = 0;
        running |= (c.phase == kPhaseRun);
        mirror[q] = c;
    }
    running = __syncthreads_or(running);
    // Live work of the next pass: the items of the current level of every
    // running query.  All 2 * kClasses + 1 counts of a query sit in registers
    // and are scanned together across the CTA (warp shuffles, then the warp
    // totals), one chunk of blockDim queries at a time.
    constexpr int K = 2 * kClasses + 1;
    __shared__ uint32_t s_wsum[32][K];
    __shared__ uint32_t s_carry[K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)((blockDim.x + 31) >> 5);
    if (threadIdx.x < K) s_carry[threadIdx.x] = 0u;
    __syncthreads();
    for (uint32_t c0 = 0; c0 < nq; c0 += blockDim.x) {
        const uint32_t q = c0 + threadIdx.x;
        uint32_t cnt[K];
#pragma unroll
        for (int k = 0; k < K; ++k) cnt[k] = 0u;
        if (q < nq) {
            const QCtl &c = *ctls[q];
            const bool run = c.phase == kPhaseRun;
            const uint32_t L = c.level, base = q * T.maxL1 + L;
            const bool last = run && (L + 1 == c.n_levels);
#pragma unroll
            for (int v = 0; v < kClasses; ++v) {
                const uint32_t gb = run ? T.g_lvl[v][base] : 0u, ge = run ? T.g_lvl[v][base + 1] : 0u;
                T.g_beg[v][q] = gb;
                cnt[v] = ge - gb;
                const uint32_t xb = last ? T.x_rng[v][q] : 0u, xe = last ? T.x_rng[v][q + 1] : 0u;
                T.x_beg[v][q] = xb;
                cnt[kClasses + v] = xe - xb;
            }
            T.t_job_beg[q] = run ? T.t_lvl[base] : 0u;
            T.t_job_end[q] = run ? T.t_lvl[base + 1] : 0u;
            cnt[K - 1] = run ? T.t_lvl_tiles[base] : 0u;
        }
        uint32_t inc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            uint32_t x = cnt[k];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            inc[k] = x;
            if (lane == 31) s_wsum[wid][k] = x;
        }
        __syncthreads();
        if (wid == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                uint32_t w = lane < nw ? s_wsum[lane][k] : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                    if (lane >= o) w += y;
                }
                if (lane < nw) s_wsum[lane][k] = w;  // inclusive prefix of warp totals
            }
        }
        __syncthreads();
        if (q < nq) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const uint32_t pre = s_carry[k] + (wid ? s_wsum[wid - 1][k] : 0u) + inc[k] - cnt[k];
                if (k < kClasses) T.g_pre[k][q] = pre;
                else if (k < 2 * kClasses) T.x_pre[k - kClasses][q] = pre;
                else T.t_pre[q] = pre;
            }
        }
        __syncthreads();
        if (threadIdx.x < K) s_carry[threadIdx.x] += s_wsum[nw - 1][threadIdx.x];
        __syncthreads();
    }
    // The tile jobs of the next pass: those of the live levels that take part
    // (their activity depends only on the loop state just written).
    if (T.jobs) {
        __shared__ uint32_t s_aj;
        if (threadIdx.x == 0) s_aj = 0u;
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x) {
            const uint32_t jb = T.t_job_beg[q], je = T.t_job_end[q];
            for (uint32_t j = jb; j < je; ++j) {
                uint32_t thr, it, g;
                if (tc_job_active(T.jobs[j], &thr, &it, &g)) T.aj[atomicAdd(&s_aj, 1u)] = j;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) *T.aj_n = s_aj;
    }
    if (threadIdx.x < K) {
        const int k = threadIdx.x;
        if (k < kClasses) T.g_next[k] = 0u;  // dynamic gather units of the next pass
        if (k < kClasses) T.g_total[k] = s_carry[k];
        else if (k < 2 * kClasses) T.x_total[k - kClasses] = s_carry[k];
        else *T.t_total = s_carry[k];
    }
    if (threadIdx.x == 0) {
        if (use_handle) cudaGraphSetConditional(handle, running ? 1u : 0u);
        if (running_out) *running_out = running;
    }
}

__global__ void __launch_bounds__(1024) k_control(QCtl *const *ctls, uint32_t nq, QCtl *mirror,
                                                  cudaGraphConditionalHandle handle, int use_handle, int *running_out,
                                                  ExecTables T, int advance) {
    control_body(ctls, nq, mirror, handle, use_handle, running_out, T, advance);
}

// Reset the loop state of queries [0, nq) (start of a run).
__global__ void k_ctl_reset(QCtl *const *ctls, uint32_t nq, uint32_t max_iter, uint32_t max_rounds,
                            uint32_t max_passes, uint32_t n_levels, unsigned long long cyclic_mask,
                            unsigned long long *box_edges, uint32_t n_boxes, uint32_t n,
                            const uint32_t *box_new_it, unsigned long long nt_read_mask) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        QCtl c;
        memset(&c, 0, sizeof(c));
        c.g = 2;
        c.iter = 1;
        c.mode = kModeNew;
        c.phase = kPhaseRun;
        c.g_iter_start = 2;
        c.col_v0 = 0u;
        c.col_v1 = 0xFFFFFFFFu;
        c.max_iter = max_iter;
        c.max_rounds = max_rounds;
        c.max_passes = max_passes;
        c.level = 0;
        c.n_levels = n_levels;
        c.cyclic_mask = cyclic_mask;
        c.box_edges = box_edges;
        c.n_boxes = n_boxes;
        c.n = n;
        c.dense_mask = 0;
        c.box_new_it = box_new_it;
        c.nt_read_mask = nt_read_mask;
        *ctls[q] = c;
    }
}

// Epsilon case of Listing 1: a box whose start state is final derives the
// empty word, so M2^b[i,i] = 1 for every vertex i.  These edges are new edges
// of the first iteration (A2^b rows = e_i), so that they take part in the
// product like any other nonterminal edge.
struct EpsDesc {
    uint64_t *m2, *a2;
    uint32_t *a2_it, *box_new_it;
    QCtl *ctl;
    unsigned long long *box_edges;
    uint32_t n, W;
};
__global__ void k_eps_init(const EpsDesc *__restrict__ eds, uint32_t ned) {
    for (uint32_t e = 0; e < ned; ++e) {
        const EpsDesc d = eds[e];
        const size_t total = (size_t)d.n * d.W;
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
            const uint32_t row = (uint32_t)(i / d.W), w = (uint32_t)(i % d.W);
            const uint64_t bit = (w == (row >> 6)) ? (1ull << (row & 63)) : 0ull;
            d.a2[i] = bit;
            if (bit) d.m2[i] |= bit;
            if (w == 0) d.a2_it[row] = 1;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *d.box_new_it = 1;
            atomicAdd(&d.ctl->edges_total, (unsigned long long)d.n);
            if (d.box_edges) atomicAdd(d.box_edges, (unsigned long long)d.n);
        }
    }
}

// --------------------------------------------------------------------------
// Graph staging: edge list -> deduplicated CSR per used terminal label.
// --------------------------------------------------------------------------
__global__ void k_stage_count(const uint32_t *__restrict__ src, const uint32_t *__restrict__ lbl,
                              const uint32_t *__restrict__ dst, size_t m, uint32_t n, uint32_t n_term,
                              const int32_t *__restrict__ label_map, uint32_t *cnt, int *err) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (size_t)gridDim.x * blockDim.x) {
        const uint32_t s = src[e], l = lbl[e], d = dst[e];
        if (s >= n || d >= n || l >= n_term) { atomicOr(err, 1); continue; }
        const int32_t li = label_map[l];
        if (li >= 0) atomicAdd(&cnt[(size_t)li * n + s], 1u);
    }
}

__global__ void k_stage_fill(const uint32_t *__restrict__ src, const uint32_t *__restrict__ lbl,
                             const uint32_t *__restrict__ dst, size_t m, uint32_t n, uint32_t n_term,
                             const int32_t *__restrict__ label_map, const uint32_t *__restrict__ off,
                             uint32_t *fill, uint32_t *col) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (size_t)gridDim.x * blockDim.x) {
        const uint32_t s = src[e], l = lbl[e], d = dst[e];
        if (s >= n || d >= n || l >= n_term) continue;
        const int32_t li = label_map[l];
        if (li < 0) continue;
        const size_t r = (size_t)li * n + s;
        col[off[r] + atomicAdd(&fill[r], 1u)] = d;
    }
}

// Sort each adjacency row and drop duplicates; ucnt[r] = distinct count.
// Rows longer than kUniqueMax are left as they are: a repeated edge only
// repeats an idempotent OR of the same source row, so duplicates cost time,
// never correctness, and the per-row work stays bounded.
constexpr uint32_t kUniqueMax = 256;
__global__ void k_stage_unique(const uint32_t *__restrict__ off, uint32_t *col, uint32_t *ucnt, size_t rows) {
    for (size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (size_t)gridDim.x * blockDim.x) {
        const uint32_t a = off[r], b = off[r + 1];
        if (b - a > kUniqueMax) { ucnt[r] = b - a; continue; }
        for (uint32_t i = a + 1; i < b; ++i) {
            const uint32_t v = col[i];
            uint32_t j = i;
            while (j > a && col[j - 1] > v) { col[j] = col[j - 1]; --j; }
            col[j] = v;
        }
        uint32_t k = a;
        for (uint32_t i = a; i < b; ++i)
            if (i == a || col[i] != col[k - 1]) col[k++] = col[i];
        ucnt[r] = k - a;
    }
}

__global__ void k_stage_compact(const uint32_t *__restrict__ off, const uint32_t *__restrict__ col,
                                const uint32_t *__restrict__ uoff, uint32_t *ucol, size_t rows) {
    for (size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (size_t)gridDim.x * blockDim.x) {
        const uint32_t a = off[r], u0 = uoff[r], k = uoff[r + 1] - u0;
        for (uint32_t i = 0; i < k; ++i) ucol[u0 + i] = col[a + i];
    }
}

// Exclusive scan of n uint32 (n < 2^32 total): out[0..n], out[n] = total.
constexpr int kScanThreads = 1024, kScanPer = 4, kScanChunk = kScanThreads * kScanPer;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULLMASK, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULLMASK, s, o);
            if (lane >= o) s += t;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    const uint32_t base = wid ? warp_sums[wid - 1] : 0u;
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_local(const uint32_t *__restrict__ in, uint32_t *out,
                                                             uint32_t *block_sums, size_t n) {
    const size_t base = (size_t)blockIdx.x * kScanChunk + (size_t)threadIdx.x * kScanPer;
    uint32_t v[kScanPer], s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) { v[i] = (base + i < n) ? in[base + i] : 0u; s += v[i]; }
    uint32_t tot;
    uint32_t ex = block_exclusive_scan(s, &tot);
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint32_t *block_sums, uint32_t nb, uint32_t *total_out) {
    // nb <= kScanChunk
    const uint32_t base = threadIdx.x * kScanPer;
    uint32_t v[kScanPer], s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) { v[i] = (base + i < nb) ? block_sums[base + i] : 0u; s += v[i]; }
    uint32_t tot;
    uint32_t ex = block_exclusive_scan(s, &tot);
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < nb) block_sums[base + i] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0) *total_out = tot;
}

__global__ void k_scan_add(uint32_t *out, const uint32_t *__restrict__ block_sums, size_t n, const uint32_t *total,
                           uint32_t *out_total) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += block_sums[i / kScanChunk];
    if (i == 0) *out_total = *total;
}

// Terminal adjacency as bit rows (needed when terminal sources run on the
// tensor cores): bits[l][x] has bit y for every CSR edge (x, l, y).
__global__ void k_csr_to_bits(const uint32_t *__restrict__ off, const uint32_t *__restrict__ col, size_t rows,
                              uint32_t W, uint64_t *bits) {
    for (size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (size_t)gridDim.x * blockDim.x) {
        uint64_t *row = bits + r * W;
        for (uint32_t e = off[r]; e < off[r + 1]; ++e) {
            const uint32_t y = col[e];
            row[y >> 6] |= 1ull << (y & 63u);
        }
    }
}

// bits[l * W + w] bit b = row (l, 64 w + b) of the CSR has an edge.
__global__ void k_nonempty_bits(const uint32_t *__restrict__ off, uint32_t n, uint32_t n_term, uint32_t W,
                                uint64_t *bits) {
    const size_t total = (size_t)n_term * W;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t l = (uint32_t)(i / W), w = (uint32_t)(i % W);
        uint64_t word = 0;
        for (uint32_t b = 0; b < 64u; ++b) {
            const uint32_t y = w * 64u + b;
            if (y >= n) break;
            const size_t r = (size_t)l * n + y;
            if (off[r + 1] > off[r]) word |= 1ull << b;
        }
        bits[i] = word;
    }
}

// --------------------------------------------------------------------------
// Result helpers.
// --------------------------------------------------------------------------
__global__ void k_popcount(const uint64_t *__restrict__ p, size_t nwords, unsigned long long *out) {
    unsigned long long s = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += (size_t)gridDim.x * blockDim.x)
        s += (unsigned long long)__popcll(p[i]);
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(FULLMASK, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// Copy rows of several blocks into a dense staging buffer:
// job k copies row rows[k] of block ptrs[k] (W words) to out + k * W.
__global__ void k_copy_rows(const uint64_t *const *__restrict__ ptrs, const uint32_t *__restrict__ rows, uint32_t njobs,
                            uint32_t W, uint64_t *out) {
    for (uint32_t k = blockIdx.x; k < njobs; k += gridDim.x) {
        const uint64_t *p = ptrs[k];
        for (uint32_t w = threadIdx.x; w < W; w += blockDim.x) out[(size_t)k * W + w] = p ? p[(size_t)rows[k] * W + w] : 0ull;
    }
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
int vpl_for_words(uint32_t W) {
    if (W <= 64) return 1;
    if (W <= 128) return 2;
    if (W <= 256) return 4;
    if (W <= 512) return 8;
    if (W <= 1024) return 16;
    return 0;
}

static int g_gather_sms[64];

cudaError_t launch_gather(int vpl, bool nt, const GItem *items, uint32_t n_items, const SrcDesc *srcs,
                          const ExecTables &T, int cls, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    const uint32_t sms = (dev >= 0 && dev < 64 && g_gather_sms[dev]) ? (uint32_t)g_gather_sms[dev] : 0u;
    // dynamic scheduling: a persistent grid (resident CTAs), at most one warp
    // per unit; otherwise one CTA per live item, at most kStrideWaves waves of
    // resident CTAs (the CTAs stride over the live items): n_items bounds the
    // live items of any pass, and a batch's pass with few live queries would
    // otherwise launch tens of thousands of CTAs that exit at once
    auto grid_of = [&](bool dyn, int occ) -> uint32_t {
        if (!sms) return n_items;
        if (!dyn) return std::min<uint32_t>(n_items, sms * (uint32_t)occ * kStrideWaves);
        const uint32_t want = (n_items * kGatherParts + 7u) / 8u;
        return std::max<uint32_t>(1u, std::min<uint32_t>(want, sms * (uint32_t)occ));
    };
#define CFPQ_GATHER(V)                                                                                          \
    if (nt) k_gather<V, true><<<grid_of(GatherDyn<V, true>::on, GatherOcc<V>::value), 256, GatherRing<V>::bytes, \
                                st>>>(items, srcs, T, cls);                                                     \
    else k_gather<V, false><<<grid_of(false, GatherOcc<V>::value), 256, 0, st>>>(items, srcs, T, cls);
    switch (vpl) {
        case 1: CFPQ_GATHER(1) break;
        case 2: CFPQ_GATHER(2) break;
        case 4: CFPQ_GATHER(4) break;
        case 8: CFPQ_GATHER(8) break;
        case 16: CFPQ_GATHER(16) break;
        default: return cudaErrorInvalidValue;
    }
#undef CFPQ_GATHER
    return cudaGetLastError();
}

// Shared-memory limits of the general gather variants (call outside any
// stream capture).
cudaError_t prepare_gather_launch() {
#define CFPQ_RING(V)                                                                                      \
    {                                                                                                     \
        const cudaError_t e = cudaFuncSetAttribute(k_gather<V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                                   (int)GatherRing<V>::bytes);                            \
        if (e != cudaSuccess) return e;                                                                   \
    }
    CFPQ_RING(4) CFPQ_RING(8) CFPQ_RING(16)
#undef CFPQ_RING
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_gather_sms[dev] = sms;
    return cudaSuccess;
}

// With fused control (ctls != null) this launch also runs the pass's loop
// control in its last CTA; done_counter must be 0 before the first launch.
cudaError_t launch_extract(int vpl, const XItem *items, uint32_t n_items, const FDesc *fds, const ExecTables &T,
                           int cls, QCtl *const *ctls, uint32_t nq, QCtl *mirror, cudaGraphConditionalHandle h,
                           int use_handle, int *running_out, unsigned int *done_counter, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    FusedControl fc{ctls, mirror, running_out, done_counter, h, nq, use_handle, ctls != nullptr ? 1 : 0};
    // (the CTAs stride over the live items; see launch_gather)
    int dev = 0;
    cudaGetDevice(&dev);
    const uint32_t sms = (dev >= 0 && dev < 64 && g_gather_sms[dev]) ? (uint32_t)g_gather_sms[dev] : 0u;
    const uint32_t grid = sms ? std::min<uint32_t>(n_items, sms * 8u * kStrideWaves) : n_items;
    switch (vpl) {
        case 1: k_extract<1><<<grid, 256, 0, st>>>(items, fds, T, cls, fc); break;
        case 2: k_extract<2><<<grid, 256, 0, st>>>(items, fds, T, cls, fc); break;
        case 4: k_extract<4><<<grid, 256, 0, st>>>(items, fds, T, cls, fc); break;
        case 8: k_extract<8><<<grid, 256, 0, st>>>(items, fds, T, cls, fc); break;
        case 16: k_extract<16><<<grid, 256, 0, st>>>(items, fds, T, cls, fc); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_control(QCtl *const *ctls, uint32_t nq, QCtl *mirror, cudaGraphConditionalHandle h, int use_handle,
                           int *running_out, const ExecTables &T, int advance, cudaStream_t st) {
    // one thread per query up to 1024 (a single warp for small batches keeps
    // the per-pass scans to shuffles)
    uint32_t threads = ((nq + 31u) / 32u) * 32u;
    if (threads < 32u) threads = 32u;
    if (threads > 1024u) threads = 1024u;
    k_control<<<1, threads, 0, st>>>(ctls, nq, mirror, h, use_handle, running_out, T, advance);
    return cudaGetLastError();
}

cudaError_t launch_ctl_reset(QCtl *const *ctls, uint32_t nq, uint32_t max_iter, uint32_t max_rounds,
                             uint32_t max_passes, uint32_t n_levels, unsigned long long cyclic_mask,
                             unsigned long long *box_edges, uint32_t n_boxes, uint32_t n,
                             const uint32_t *box_new_it, unsigned long long nt_read_mask, cudaStream_t st) {
    k_ctl_reset<<<(nq + 255) / 256, 256, 0, st>>>(ctls, nq, max_iter, max_rounds, max_passes, n_levels, cyclic_mask,
                                                  box_edges, n_boxes, n, box_new_it, nt_read_mask);
    return cudaGetLastError();
}

cudaError_t launch_eps_init(const void *eds, uint32_t ned, uint32_t grid, cudaStream_t st) {
    if (ned == 0) return cudaSuccess;
    k_eps_init<<<grid, 256, 0, st>>>(static_cast<const EpsDesc *>(eds), ned);
    return cudaGetLastError();
}

size_t eps_desc_size() { return sizeof(EpsDesc); }
void fill_eps_desc(void *dst, uint64_t *m2, uint64_t *a2, uint32_t *a2_it, uint32_t *box_new_it, QCtl *ctl,
                   unsigned long long *box_edges, uint32_t n, uint32_t W) {
    EpsDesc d{m2, a2, a2_it, box_new_it, ctl, box_edges, n, W};
    memcpy(dst, &d, sizeof(d));
}

static uint32_t grid_for(size_t work, uint32_t threads, uint32_t cap = 4096) {
    size_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (uint32_t)g;
}

// Exclusive scan with total: out has n+1 entries.  tmp needs
// ceil(n / kScanChunk) + 1 words.
cudaError_t scan_exclusive(const uint32_t *in, uint32_t *out, size_t n, uint32_t *tmp, cudaStream_t st) {
    const size_t nb = (n + kScanChunk - 1) / kScanChunk;
    if (nb > (size_t)kScanChunk) return cudaErrorInvalidValue;
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(uint32_t), st);
    k_scan_local<<<(uint32_t)nb, kScanThreads, 0, st>>>(in, out, tmp, n);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(tmp, (uint32_t)nb, tmp + nb);
    k_scan_add<<<(uint32_t)((n + 255) / 256), 256, 0, st>>>(out, tmp, n, tmp + nb, out + n);
    return cudaGetLastError();
}

cudaError_t launch_stage_count(const uint32_t *src, const uint32_t *lbl, const uint32_t *dst, size_t m, uint32_t n,
                               uint32_t n_term, const int32_t *label_map, uint32_t *cnt, int *err, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_stage_count<<<grid_for(m, 256), 256, 0, st>>>(src, lbl, dst, m, n, n_term, label_map, cnt, err);
    return cudaGetLastError();
}
cudaError_t launch_stage_fill(const uint32_t *src, const uint32_t *lbl, const uint32_t *dst, size_t m, uint32_t n,
                              uint32_t n_term, const int32_t *label_map, const uint32_t *off, uint32_t *fill,
                              uint32_t *col, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_stage_fill<<<grid_for(m, 256), 256, 0, st>>>(src, lbl, dst, m, n, n_term, label_map, off, fill, col);
    return cudaGetLastError();
}
cudaError_t launch_stage_unique(const uint32_t *off, uint32_t *col, uint32_t *ucnt, size_t rows, cudaStream_t st) {
    if (rows == 0) return cudaSuccess;
    k_stage_unique<<<grid_for(rows, 128), 128, 0, st>>>(off, col, ucnt, rows);
    return cudaGetLastError();
}
cudaError_t launch_stage_compact(const uint32_t *off, const uint32_t *col, const uint32_t *uoff, uint32_t *ucol,
                                 size_t rows, cudaStream_t st) {
    if (rows == 0) return cudaSuccess;
    k_stage_compact<<<grid_for(rows, 128), 128, 0, st>>>(off, col, uoff, ucol, rows);
    return cudaGetLastError();
}
cudaError_t launch_csr_to_bits(const uint32_t *off, const uint32_t *col, size_t rows, uint32_t W, uint64_t *bits,
                               cudaStream_t st) {
    if (rows == 0) return cudaSuccess;
    k_csr_to_bits<<<grid_for(rows, 128), 128, 0, st>>>(off, col, rows, W, bits);
    return cudaGetLastError();
}
cudaError_t launch_nonempty_bits(const uint32_t *off, uint32_t n, uint32_t n_term, uint32_t W, uint64_t *bits,
                                 cudaStream_t st) {
    const size_t total = (size_t)n_term * W;
    if (total == 0) return cudaSuccess;
    k_nonempty_bits<<<grid_for(total, 256), 256, 0, st>>>(off, n, n_term, W, bits);
    return cudaGetLastError();
}
cudaError_t launch_popcount(const uint64_t *p, size_t nwords, unsigned long long *out, cudaStream_t st) {
    if (nwords == 0) return cudaSuccess;
    k_popcount<<<grid_for(nwords, 256, 2048), 256, 0, st>>>(p, nwords, out);
    return cudaGetLastError();
}
cudaError_t launch_copy_rows(const uint64_t *const *ptrs, const uint32_t *rows, uint32_t njobs, uint32_t W,
                             uint64_t *out, cudaStream_t st) {
    if (njobs == 0) return cudaSuccess;
    k_copy_rows<<<njobs < 4096 ? njobs : 4096, 128, 0, st>>>(ptrs, rows, njobs, W, out);
    return cudaGetLastError();
}

}  // namespace cfpq
