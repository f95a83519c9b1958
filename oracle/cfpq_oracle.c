/*
 * cfpq_oracle.c -- plain CPU oracle for Kronecker-product CFPQ / RPQ.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file.  It shares no code, header, table or helper
 * with the CUDA library; every routine is written for obviousness, not speed.
 *
 * Reference: Shemetova et al., "One Algorithm to Evaluate Them All" (arXiv
 * 2103.14688).  Conventions follow the paper:
 *   - graph  <V,E,L>, V = {0..n-1} (Sec. 2.1, Def. of an edge-labelled graph);
 *   - Boolean decomposition: one n x n Boolean matrix per label (Sec. 2.1);
 *   - RSM boxes with disjoint state sets, one start state per box, final sets,
 *     transitions over terminals and box labels (Sec. 2.3, Def. of an RSM);
 *   - Kronecker index: row/column = state * n + vertex (Sec. 2.4, Def. of the
 *     Kronecker product; Listing 1's getStates/getCoordinates).
 *
 * Functions:
 *   orc_kron_fixpoint  Oracle A: Listing 1 with M3 rebuilt and its closure
 *                      recomputed from scratch every iteration (the naive
 *                      variant the evaluation section describes).
 *   orc_worklist       Oracle B: CFL-reachability by a worklist over RSM
 *                      configurations (Sec. 2.3, execution rules), independent
 *                      of Kronecker products and closures.
 *   orc_rsm_accepts    RSM word membership by a chart fixpoint (Sec. 2.3).
 *   orc_brute_reach    Oracle C: enumerate all paths up to a length bound and
 *                      test their words (Sec. 2.1, reachability semantics).
 *   orc_brute_paths    Oracle C for all-path semantics between two vertices.
 *   orc_closure_rows   Rows of C = M3^+ for given M2, by BFS over M3's edges.
 *
 * Parity status: every function is pinned by tests (worked example of
 * Sec. 3.3, closed forms, cross-oracle agreement, brute force, invariants).
 *
 * Return codes: 0 ok, -1 invalid argument, -2 iteration cap reached,
 * -3 allocation failure, -4 output buffer too small.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TERM 0u
#define ORC_NONTERM 1u

typedef struct {
    uint32_t Q, B;
    const uint32_t *box_start, *state_box;
    const uint8_t *state_final;
    uint32_t T;
    const uint32_t *tr_from, *tr_kind, *tr_sym, *tr_to;
} orc_rsm;

static inline int bget(const uint64_t *row, uint64_t i) { return (int)((row[i >> 6] >> (i & 63)) & 1u); }
static inline void bset(uint64_t *row, uint64_t i) { row[i >> 6] |= (uint64_t)1 << (i & 63); }
static inline uint64_t words_for(uint64_t bits) { return (bits + 63) / 64; }

static int check_rsm(const orc_rsm *r, uint32_t n_term) {
    if (r->Q == 0 || r->B == 0) return -1;
    for (uint32_t b = 0; b < r->B; ++b)
        if (r->box_start[b] >= r->Q || r->state_box[r->box_start[b]] != b) return -1;
    for (uint32_t s = 0; s < r->Q; ++s)
        if (r->state_box[s] >= r->B) return -1;
    for (uint32_t t = 0; t < r->T; ++t) {
        if (r->tr_from[t] >= r->Q || r->tr_to[t] >= r->Q) return -1;
        if (r->state_box[r->tr_from[t]] != r->state_box[r->tr_to[t]]) return -1;
        if (r->tr_kind[t] == ORC_TERM) { if (r->tr_sym[t] >= n_term) return -1; }
        else if (r->tr_kind[t] == ORC_NONTERM) { if (r->tr_sym[t] >= r->B) return -1; }
        else return -1;
    }
    return 0;
}

static int check_graph(uint32_t n, uint32_t n_term, uint64_t m, const uint32_t *src,
                       const uint32_t *lbl, const uint32_t *dst) {
    if (n == 0) return -1;
    for (uint64_t e = 0; e < m; ++e)
        if (src[e] >= n || dst[e] >= n || lbl[e] >= n_term) return -1;
    return 0;
}

/* Label index in the set of graph matrices M2: terminals first, then boxes. */
static inline uint32_t label_of(const orc_rsm *r, uint32_t n_term, uint32_t t) {
    return r->tr_kind[t] == ORC_TERM ? r->tr_sym[t] : n_term + r->tr_sym[t];
}

/* ------------------------------------------------------------------------ */
/* Transitive closure of a Boolean matrix given as adjacency lists:          */
/* C[u] = set of vertices reachable from u by a path of one or more edges.   */
/* ------------------------------------------------------------------------ */
/* Threads of closure_from_lists (rows are independent).  1 = the plain
 * sequential loop; the CPU baseline of the benchmark may raise it.  The
 * result does not depend on it. */
static int orc_threads = 1;
int orc_set_threads(int k) {
    orc_threads = k < 1 ? 1 : k;
    return 0;
}

static int closure_from_lists(uint64_t N, const uint64_t *off, const uint32_t *adj, uint64_t *C) {
    uint64_t wN = words_for(N);
    int failed = 0;
    memset(C, 0, sizeof(uint64_t) * N * wN);
#pragma omp parallel num_threads(orc_threads)
    {
        uint32_t *stack = (uint32_t *)malloc(sizeof(uint32_t) * (N + 1));
        if (!stack) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t uu = 0; uu < (int64_t)N; ++uu) {
            if (!stack) continue;
            uint64_t u = (uint64_t)uu;
            uint64_t *row = C + u * wN;
            uint64_t sp = 0;
            for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
                uint32_t v = adj[e];
                if (!bget(row, v)) { bset(row, v); stack[sp++] = v; }
            }
            while (sp) {
                uint32_t w = stack[--sp];
                for (uint64_t e = off[w]; e < off[w + 1]; ++e) {
                    uint32_t v = adj[e];
                    if (!bget(row, v)) { bset(row, v); stack[sp++] = v; }
                }
            }
        }
        free(stack);
    }
    return failed ? -3 : 0;
}

/* Row-major dense N x N bit matrix -> adjacency lists. */
static int lists_from_bits(uint64_t N, const uint64_t *M, uint64_t **off_out, uint32_t **adj_out) {
    uint64_t wN = words_for(N), nnz = 0;
    for (uint64_t i = 0; i < N * wN; ++i) nnz += (uint64_t)__builtin_popcountll(M[i]);
    uint64_t *off = (uint64_t *)malloc(sizeof(uint64_t) * (N + 1));
    uint32_t *adj = (uint32_t *)malloc(sizeof(uint32_t) * (nnz ? nnz : 1));
    if (!off || !adj) { free(off); free(adj); return -3; }
    uint64_t k = 0;
    for (uint64_t u = 0; u < N; ++u) {
        off[u] = k;
        for (uint64_t v = 0; v < N; ++v)
            if (bget(M + u * wN, v)) adj[k++] = (uint32_t)v;
    }
    off[N] = k;
    *off_out = off;
    *adj_out = adj;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Oracle A: Listing 1, naive variant.                                        */
/* ------------------------------------------------------------------------ */
/*
 * Inputs: graph (n, n_term, edge triples), RSM.  max_iter bounds the loop.
 * Outputs:
 *   out_m2    [B * n * wn]  final M2^N for every box N (wn = ceil(n/64));
 *   out_iters number of loop iterations, counting the last one that adds no
 *             edge (the loop runs "while M2 is changing");
 *   trace_m3  optional [max_iter * N * wN]: M3 of every iteration;
 *   trace_c   optional [max_iter * N * wN]: C3 = M3^+ of every iteration;
 *   out_c     optional [N * wN]: C3 of the final iteration;
 *   trace_new optional [max_iter]: number of M2 bits added by each iteration.
 * N = Q * n, wN = ceil(N/64).
 */
int orc_kron_fixpoint(uint32_t n, uint32_t n_term, uint64_t m, const uint32_t *src, const uint32_t *lbl,
                      const uint32_t *dst, uint32_t Q, uint32_t B, const uint32_t *box_start,
                      const uint32_t *state_box, const uint8_t *state_final, uint32_t T,
                      const uint32_t *tr_from, const uint32_t *tr_kind, const uint32_t *tr_sym,
                      const uint32_t *tr_to, uint32_t max_iter, uint64_t *out_m2, uint32_t *out_iters,
                      uint64_t *trace_m3, uint64_t *trace_c, uint64_t *out_c, uint64_t *trace_new) {
    orc_rsm r = {Q, B, box_start, state_box, state_final, T, tr_from, tr_kind, tr_sym, tr_to};
    if (check_graph(n, n_term, m, src, lbl, dst) || check_rsm(&r, n_term)) return -1;
    const uint64_t wn = words_for(n), N = (uint64_t)Q * n, wN = words_for(N);
    const uint32_t L = n_term + B;
    uint64_t *M2 = (uint64_t *)calloc((size_t)L * n * wn, sizeof(uint64_t));
    uint64_t *M3 = (uint64_t *)calloc((size_t)(N * wN), sizeof(uint64_t));
    uint64_t *C = (uint64_t *)calloc((size_t)(N * wN), sizeof(uint64_t));
    if (!M2 || !M3 || !C) { free(M2); free(M3); free(C); return -3; }
#define M2ROW(l, x) (M2 + ((uint64_t)(l) * n + (x)) * wn)
    /* M2 <- Boolean decomposition of the input graph (Sec. 2.1). */
    for (uint64_t e = 0; e < m; ++e) bset(M2ROW(lbl[e], src[e]), dst[e]);
    /* Epsilon case of Listing 1: for a state s with a nonterminal S such that s
     * is both the start and a final state of S's box, M2^S[i,i] = 1 for all i. */
    for (uint32_t b = 0; b < B; ++b)
        if (state_final[box_start[b]])
            for (uint32_t i = 0; i < n; ++i) bset(M2ROW(n_term + b, i), i);

    int rc = -2;
    uint32_t it;
    for (it = 1; it <= max_iter; ++it) {
        /* M3 = OR over labels l of M1^l (x) M2^l, built entry by entry from the
         * definition C[s*n + x, t*n + y] = M1^l[s,t] & M2^l[x,y]. */
        memset(M3, 0, sizeof(uint64_t) * N * wN);
        for (uint32_t t = 0; t < T; ++t) {
            uint32_t l = label_of(&r, n_term, t), s = tr_from[t], u = tr_to[t];
            for (uint32_t x = 0; x < n; ++x)
                for (uint32_t y = 0; y < n; ++y)
                    if (bget(M2ROW(l, x), y)) bset(M3 + ((uint64_t)s * n + x) * wN, (uint64_t)u * n + y);
        }
        /* C3 = transitive closure of M3, from scratch. */
        uint64_t *off = NULL;
        uint32_t *adj = NULL;
        if (lists_from_bits(N, M3, &off, &adj)) { rc = -3; break; }
        int crc = closure_from_lists(N, off, adj, C);
        free(off);
        free(adj);
        if (crc) { rc = crc; break; }
        if (trace_m3) memcpy(trace_m3 + (uint64_t)(it - 1) * N * wN, M3, sizeof(uint64_t) * N * wN);
        if (trace_c) memcpy(trace_c + (uint64_t)(it - 1) * N * wN, C, sizeof(uint64_t) * N * wN);
        /* Extraction: C3[i,j] with s = i / n, f = j / n, x = i mod n, y = j mod n;
         * for S in getNonterminals(R, s, f) = {box b : s = start(b), f final in b}
         * set M2^S[x,y]. */
        uint64_t added = 0;
        for (uint32_t b = 0; b < B; ++b) {
            uint32_t s = box_start[b];
            for (uint32_t f = 0; f < Q; ++f) {
                if (state_box[f] != b || !state_final[f]) continue;
                for (uint32_t x = 0; x < n; ++x)
                    for (uint32_t y = 0; y < n; ++y)
                        if (bget(C + ((uint64_t)s * n + x) * wN, (uint64_t)f * n + y) &&
                            !bget(M2ROW(n_term + b, x), y)) {
                            bset(M2ROW(n_term + b, x), y);
                            ++added;
                        }
            }
        }
        if (trace_new) trace_new[it - 1] = added;
        if (added == 0) { rc = 0; break; }
    }
    if (rc == 0 || rc == -2) {
        *out_iters = rc == 0 ? it : max_iter;
        memcpy(out_m2, M2ROW(n_term, 0), sizeof(uint64_t) * (uint64_t)B * n * wn);
        if (out_c) memcpy(out_c, C, sizeof(uint64_t) * N * wN);
    }
#undef M2ROW
    free(M2);
    free(M3);
    free(C);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Oracle B: worklist CFL-reachability over RSM configurations.               */
/* ------------------------------------------------------------------------ */
/*
 * Facts P(x, s, y): a run of box(s) entered at vertex x in its start state is
 * in state s at vertex y.  Sum_b(x, y): box b entered at x can accept at y.
 * Rules (Sec. 2.3, the three configuration transitions):
 *   enter(b, x)                             => P(x, start(b), x)
 *   P(x,s,y), s -a-> t, (y,a,z) in E        => P(x, t, z)        (read)
 *   P(x,s,y), s -b'-> t                     => enter(b', y)      (call)
 *   P(x,s,y), s -b'-> t, Sum_b'(y, z)       => P(x, t, z)        (return)
 *   P(x,s,y), s final in box(s)             => Sum_box(s)(x, y)  (accept)
 * With sources == NULL every box is entered at every vertex, so out_sum
 * [B * n * wn] holds the full Sum_b of every box b (all-pairs reachability per
 * nonterminal).  With a source list only the start box is entered at the
 * sources and other boxes on demand, at the vertex where they are called; the
 * rows of the start box at the sources are then complete.
 */
int orc_worklist(uint32_t n, uint32_t n_term, uint64_t m, const uint32_t *src, const uint32_t *lbl,
                 const uint32_t *dst, uint32_t Q, uint32_t B, uint32_t start_box, const uint32_t *box_start,
                 const uint32_t *state_box, const uint8_t *state_final, uint32_t T, const uint32_t *tr_from,
                 const uint32_t *tr_kind, const uint32_t *tr_sym, const uint32_t *tr_to, uint32_t n_sources,
                 const uint32_t *sources, uint64_t *out_sum) {
    orc_rsm r = {Q, B, box_start, state_box, state_final, T, tr_from, tr_kind, tr_sym, tr_to};
    if (check_graph(n, n_term, m, src, lbl, dst) || check_rsm(&r, n_term) || start_box >= B) return -1;
    const uint64_t wn = words_for(n);
    /* terminal adjacency lists per (label, vertex) */
    uint64_t *aoff = (uint64_t *)calloc((size_t)n_term * n + 1, sizeof(uint64_t));
    uint32_t *aadj = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint64_t *P = (uint64_t *)calloc((size_t)Q * n * wn, sizeof(uint64_t));
    uint64_t *PT = (uint64_t *)calloc((size_t)Q * n * wn, sizeof(uint64_t));
    uint64_t *pend = (uint64_t *)calloc((size_t)Q * n * wn, sizeof(uint64_t));
    uint64_t *Sum = (uint64_t *)calloc((size_t)B * n * wn, sizeof(uint64_t));
    uint64_t *pendS = (uint64_t *)calloc((size_t)B * n * wn, sizeof(uint64_t));
    uint8_t *inq = (uint8_t *)calloc((size_t)Q * n, 1);
    uint8_t *inqS = (uint8_t *)calloc((size_t)B * n, 1);
    uint8_t *entered = (uint8_t *)calloc((size_t)B * n, 1);
    uint64_t qcap = (uint64_t)(Q + B) * n + 1;
    uint64_t *queue = (uint64_t *)malloc(sizeof(uint64_t) * qcap);
    uint64_t *fill = (uint64_t *)calloc((size_t)n_term * n + 1, sizeof(uint64_t));
    int rc = 0;
    if (!aoff || !aadj || !P || !PT || !pend || !Sum || !pendS || !inq || !inqS || !entered || !queue || !fill) {
        rc = -3;
        goto done;
    }
    for (uint64_t e = 0; e < m; ++e) aoff[(uint64_t)lbl[e] * n + src[e] + 1]++;
    for (uint64_t i = 0; i < (uint64_t)n_term * n; ++i) aoff[i + 1] += aoff[i];
    for (uint64_t e = 0; e < m; ++e) {
        uint64_t k = (uint64_t)lbl[e] * n + src[e];
        aadj[aoff[k] + fill[k]++] = dst[e];
    }
    /* queue entries: (kind << 62) | (index << 32) | x ; kind 0 = P row (s, x), 1 = Sum row (b, x) */
    uint64_t qh = 0, qt = 0;
#define QPUSH(v) do { queue[qt] = (v); qt = (qt + 1) % qcap; } while (0)
#define ADD_P(xx, ss, yy) do {                                                        \
        uint64_t _x = (xx), _s = (ss), _y = (yy);                                     \
        uint64_t *_row = P + (_s * n + _x) * wn;                                      \
        if (!bget(_row, _y)) {                                                        \
            bset(_row, _y); bset(PT + (_s * n + _y) * wn, _x);                        \
            bset(pend + (_s * n + _x) * wn, _y);                                      \
            if (!inq[_s * n + _x]) { inq[_s * n + _x] = 1; QPUSH((_s << 32) | _x); }  \
        } } while (0)
#define ADD_SUM(bb, xx, yy) do {                                                      \
        uint64_t _b = (bb), _x = (xx), _y = (yy);                                     \
        uint64_t *_row = Sum + (_b * n + _x) * wn;                                    \
        if (!bget(_row, _y)) {                                                        \
            bset(_row, _y); bset(pendS + (_b * n + _x) * wn, _y);                     \
            if (!inqS[_b * n + _x]) { inqS[_b * n + _x] = 1;                          \
                QPUSH(((uint64_t)1 << 62) | (_b << 32) | _x); }                       \
        } } while (0)
#define ENTER(bb, yy) do {                                                            \
        uint64_t _b2 = (bb), _y2 = (yy);                                              \
        if (!entered[_b2 * n + _y2]) { entered[_b2 * n + _y2] = 1;                    \
            ADD_P(_y2, box_start[_b2], _y2); } } while (0)

    if (sources) {
        for (uint32_t i = 0; i < n_sources; ++i) {
            if (sources[i] >= n) { rc = -1; goto done; }
            ENTER(start_box, sources[i]);
        }
    } else {
        for (uint32_t b = 0; b < B; ++b)
            for (uint32_t x = 0; x < n; ++x) ENTER(b, x);
    }
    while (qh != qt) {
        uint64_t v = queue[qh];
        qh = (qh + 1) % qcap;
        uint64_t kind = v >> 62, idx = (v >> 32) & 0x3fffffffu, x = v & 0xffffffffu;
        if (kind == 0) {
            uint64_t s = idx;
            inq[s * n + x] = 0;
            uint64_t *pr = pend + (s * n + x) * wn;
            for (uint64_t w = 0; w < wn; ++w) {
                uint64_t bits = pr[w];
                pr[w] = 0;
                while (bits) {
                    uint64_t y = w * 64 + (uint64_t)__builtin_ctzll(bits);
                    bits &= bits - 1;
                    if (state_final[s]) ADD_SUM(state_box[s], x, y);
                    for (uint32_t t = 0; t < T; ++t) {
                        if (tr_from[t] != s) continue;
                        uint64_t to = tr_to[t];
                        if (tr_kind[t] == ORC_TERM) {
                            uint64_t k = (uint64_t)tr_sym[t] * n + y;
                            for (uint64_t e = aoff[k]; e < aoff[k + 1]; ++e) ADD_P(x, to, aadj[e]);
                        } else {
                            uint64_t b2 = tr_sym[t];
                            ENTER(b2, y);
                            const uint64_t *sr = Sum + (b2 * n + y) * wn;
                            for (uint64_t w2 = 0; w2 < wn; ++w2) {
                                uint64_t sb = sr[w2];
                                while (sb) {
                                    uint64_t z = w2 * 64 + (uint64_t)__builtin_ctzll(sb);
                                    sb &= sb - 1;
                                    ADD_P(x, to, z);
                                }
                            }
                        }
                    }
                }
            }
        } else {
            uint64_t b = idx;
            inqS[b * n + x] = 0;
            uint64_t *pr = pendS + (b * n + x) * wn;
            for (uint64_t w = 0; w < wn; ++w) {
                uint64_t bits = pr[w];
                pr[w] = 0;
                while (bits) {
                    uint64_t z = w * 64 + (uint64_t)__builtin_ctzll(bits);
                    bits &= bits - 1;
                    /* new Sum_b(x, z): every waiting caller P(x', s', x) with s' -b-> t' */
                    for (uint32_t t = 0; t < T; ++t) {
                        if (tr_kind[t] != ORC_NONTERM || tr_sym[t] != b) continue;
                        uint64_t s2 = tr_from[t], to = tr_to[t];
                        const uint64_t *ptr = PT + (s2 * n + x) * wn;
                        for (uint64_t w2 = 0; w2 < wn; ++w2) {
                            uint64_t cb = ptr[w2];
                            while (cb) {
                                uint64_t x2 = w2 * 64 + (uint64_t)__builtin_ctzll(cb);
                                cb &= cb - 1;
                                ADD_P(x2, to, z);
                            }
                        }
                    }
                }
            }
        }
    }
    memcpy(out_sum, Sum, sizeof(uint64_t) * (uint64_t)B * n * wn);
#undef QPUSH
#undef ADD_P
#undef ADD_SUM
#undef ENTER
done:
    free(aoff); free(aadj); free(P); free(PT); free(pend); free(Sum); free(pendS);
    free(inq); free(inqS); free(entered); free(queue); free(fill);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* RSM membership by a chart fixpoint.                                        */
/* ------------------------------------------------------------------------ */
/*
 * A(s, i, j): started in state s before w[i], the box of s can read w[i..j)
 * and stop in one of its final states with every call it made returned.
 *   A(s, i, i)  if s is final;
 *   A(s, i, j)  if s -a-> t, w[i] = a and A(t, i+1, j);
 *   A(s, i, j)  if s -b-> t and A(start(b), i, k) and A(t, k, j) for some k.
 * Iterated to a fixpoint so that unit and empty cycles terminate.
 */
static int chart_accepts(const orc_rsm *r, uint32_t box, const uint32_t *w, uint32_t len, uint8_t *A) {
    const uint32_t L1 = len + 1;
#define AIDX(s, i, j) (((uint64_t)(s) * L1 + (i)) * L1 + (j))
    memset(A, 0, (size_t)r->Q * L1 * L1);
    int changed = 1;
    while (changed) {
        changed = 0;
        for (uint32_t s = 0; s < r->Q; ++s)
            for (uint32_t i = 0; i <= len; ++i)
                for (uint32_t j = i; j <= len; ++j) {
                    if (A[AIDX(s, i, j)]) continue;
                    int v = (i == j) && r->state_final[s];
                    for (uint32_t t = 0; t < r->T && !v; ++t) {
                        if (r->tr_from[t] != s) continue;
                        uint32_t to = r->tr_to[t];
                        if (r->tr_kind[t] == ORC_TERM) {
                            if (i < j && w[i] == r->tr_sym[t] && A[AIDX(to, i + 1, j)]) v = 1;
                        } else {
                            uint32_t q0 = r->box_start[r->tr_sym[t]];
                            for (uint32_t k = i; k <= j && !v; ++k)
                                if (A[AIDX(q0, i, k)] && A[AIDX(to, k, j)]) v = 1;
                        }
                    }
                    if (v) { A[AIDX(s, i, j)] = 1; changed = 1; }
                }
    }
    int acc = A[AIDX(r->box_start[box], 0, len)];
#undef AIDX
    return acc;
}

int orc_rsm_accepts(uint32_t n_term, uint32_t Q, uint32_t B, const uint32_t *box_start, const uint32_t *state_box,
                    const uint8_t *state_final, uint32_t T, const uint32_t *tr_from, const uint32_t *tr_kind,
                    const uint32_t *tr_sym, const uint32_t *tr_to, uint32_t box, const uint32_t *word,
                    uint32_t len) {
    orc_rsm r = {Q, B, box_start, state_box, state_final, T, tr_from, tr_kind, tr_sym, tr_to};
    if (check_rsm(&r, n_term) || box >= B) return -1;
    uint8_t *A = (uint8_t *)malloc((size_t)Q * (len + 1) * (len + 1));
    if (!A) return -3;
    int acc = chart_accepts(&r, box, word, len, A);
    free(A);
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Oracle C: brute-force path enumeration.                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t n;
    uint64_t me;               /* distinct edges, sorted by (src, label, dst) */
    uint32_t *es, *el, *ed;
    uint64_t *off;             /* out-edge ranges per source vertex */
} orc_edges;

static int cmp_triple(const void *a, const void *b) {
    const uint32_t *x = (const uint32_t *)a, *y = (const uint32_t *)b;
    for (int i = 0; i < 3; ++i)
        if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
    return 0;
}

static int dedupe_edges(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *lbl, const uint32_t *dst,
                        orc_edges *E) {
    uint32_t *tr = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (m ? m : 1));
    if (!tr) return -3;
    for (uint64_t e = 0; e < m; ++e) { tr[3 * e] = src[e]; tr[3 * e + 1] = lbl[e]; tr[3 * e + 2] = dst[e]; }
    qsort(tr, m, sizeof(uint32_t) * 3, cmp_triple);
    uint64_t k = 0;
    for (uint64_t e = 0; e < m; ++e)
        if (k == 0 || cmp_triple(tr + 3 * e, tr + 3 * (k - 1)) != 0) {
            memmove(tr + 3 * k, tr + 3 * e, sizeof(uint32_t) * 3);
            ++k;
        }
    E->n = n;
    E->me = k;
    E->es = (uint32_t *)malloc(sizeof(uint32_t) * (k ? k : 1));
    E->el = (uint32_t *)malloc(sizeof(uint32_t) * (k ? k : 1));
    E->ed = (uint32_t *)malloc(sizeof(uint32_t) * (k ? k : 1));
    E->off = (uint64_t *)calloc(n + 1, sizeof(uint64_t));
    if (!E->es || !E->el || !E->ed || !E->off) { free(tr); return -3; }
    for (uint64_t e = 0; e < k; ++e) {
        E->es[e] = tr[3 * e]; E->el[e] = tr[3 * e + 1]; E->ed[e] = tr[3 * e + 2];
        E->off[tr[3 * e] + 1]++;
    }
    for (uint32_t v = 0; v < n; ++v) E->off[v + 1] += E->off[v];
    free(tr);
    return 0;
}

static void free_edges(orc_edges *E) { free(E->es); free(E->el); free(E->ed); free(E->off); }

/* Depth-first enumeration of every path of length <= max_len starting at x;
 * calls visit(path of edge ids, length) at every prefix including the empty one. */
typedef struct {
    const orc_edges *E;
    const orc_rsm *r;
    uint32_t max_len;
    uint32_t *path, *word;
    uint8_t *chart;
    /* reach mode */
    uint64_t *reach;
    uint64_t wn;
    uint32_t x;
    /* paths mode */
    uint32_t box, vf;
    uint32_t *out_edges;
    uint64_t edge_cap, edge_used;
    uint64_t *out_off;
    uint64_t path_cap, n_paths;
    int overflow;
} orc_dfs;

static void dfs_reach(orc_dfs *d, uint32_t v, uint32_t len) {
    for (uint32_t b = 0; b < d->r->B; ++b) {
        uint64_t *row = d->reach + ((uint64_t)b * d->E->n + d->x) * d->wn;
        if (bget(row, v)) continue;
        if (chart_accepts(d->r, b, d->word, len, d->chart)) bset(row, v);
    }
    if (len == d->max_len) return;
    for (uint64_t e = d->E->off[v]; e < d->E->off[v + 1]; ++e) {
        d->word[len] = d->E->el[e];
        dfs_reach(d, d->E->ed[e], len + 1);
    }
}

int orc_brute_reach(uint32_t n, uint32_t n_term, uint64_t m, const uint32_t *src, const uint32_t *lbl,
                    const uint32_t *dst, uint32_t Q, uint32_t B, const uint32_t *box_start,
                    const uint32_t *state_box, const uint8_t *state_final, uint32_t T, const uint32_t *tr_from,
                    const uint32_t *tr_kind, const uint32_t *tr_sym, const uint32_t *tr_to, uint32_t max_len,
                    uint64_t *out_reach) {
    orc_rsm r = {Q, B, box_start, state_box, state_final, T, tr_from, tr_kind, tr_sym, tr_to};
    if (check_graph(n, n_term, m, src, lbl, dst) || check_rsm(&r, n_term)) return -1;
    orc_edges E;
    memset(&E, 0, sizeof(E));
    if (dedupe_edges(n, m, src, lbl, dst, &E)) { free_edges(&E); return -3; }
    orc_dfs d;
    memset(&d, 0, sizeof(d));
    d.E = &E; d.r = &r; d.max_len = max_len; d.wn = words_for(n); d.reach = out_reach;
    d.word = (uint32_t *)malloc(sizeof(uint32_t) * (max_len + 1));
    d.chart = (uint8_t *)malloc((size_t)Q * (max_len + 1) * (max_len + 1));
    int rc = 0;
    if (!d.word || !d.chart) rc = -3;
    else {
        memset(out_reach, 0, sizeof(uint64_t) * (uint64_t)B * n * d.wn);
        /* A pair (x, y) is only marked once; the early exit is a pure speed-up
         * because every word reaching y is tested until one is accepted. */
        for (uint32_t x = 0; x < n; ++x) { d.x = x; dfs_reach(&d, x, 0); }
    }
    free(d.word); free(d.chart); free_edges(&E);
    return rc;
}

static void dfs_paths(orc_dfs *d, uint32_t v, uint32_t len) {
    if (v == d->vf && chart_accepts(d->r, d->box, d->word, len, d->chart)) {
        if (d->n_paths >= d->path_cap || d->edge_used + 3ull * len > d->edge_cap) {
            d->overflow = 1;
        } else {
            for (uint32_t i = 0; i < len; ++i) {
                uint64_t e = d->path[i];
                d->out_edges[d->edge_used++] = d->E->es[e];
                d->out_edges[d->edge_used++] = d->E->el[e];
                d->out_edges[d->edge_used++] = d->E->ed[e];
            }
            d->n_paths++;
            d->out_off[d->n_paths] = d->edge_used / 3;
        }
    }
    if (len == d->max_len) return;
    for (uint64_t e = d->E->off[v]; e < d->E->off[v + 1]; ++e) {
        d->path[len] = (uint32_t)e;
        d->word[len] = d->E->el[e];
        dfs_paths(d, d->E->ed[e], len + 1);
    }
}

/*
 * All paths vs -> vf with at most max_len edges whose word is in L(box).
 * out_edges receives (src, label, dst) triples, out_off[k]..out_off[k+1] the
 * edge range of path k (in edges, out_off[0] = 0).  Paths come in depth-first
 * order; the caller sorts them.  Returns -4 if a capacity was exceeded.
 */
int orc_brute_paths(uint32_t n, uint32_t n_term, uint64_t m, const uint32_t *src, const uint32_t *lbl,
                    const uint32_t *dst, uint32_t Q, uint32_t B, const uint32_t *box_start,
                    const uint32_t *state_box, const uint8_t *state_final, uint32_t T, const uint32_t *tr_from,
                    const uint32_t *tr_kind, const uint32_t *tr_sym, const uint32_t *tr_to, uint32_t box,
                    uint32_t vs, uint32_t vf, uint32_t max_len, uint32_t *out_edges, uint64_t edge_cap,
                    uint64_t *out_off, uint64_t path_cap, uint64_t *n_paths) {
    orc_rsm r = {Q, B, box_start, state_box, state_final, T, tr_from, tr_kind, tr_sym, tr_to};
    if (check_graph(n, n_term, m, src, lbl, dst) || check_rsm(&r, n_term) || box >= B || vs >= n || vf >= n)
        return -1;
    orc_edges E;
    memset(&E, 0, sizeof(E));
    if (dedupe_edges(n, m, src, lbl, dst, &E)) { free_edges(&E); return -3; }
    orc_dfs d;
    memset(&d, 0, sizeof(d));
    d.E = &E; d.r = &r; d.max_len = max_len; d.box = box; d.vf = vf;
    d.out_edges = out_edges; d.edge_cap = edge_cap; d.out_off = out_off; d.path_cap = path_cap;
    d.path = (uint32_t *)malloc(sizeof(uint32_t) * (max_len + 1));
    d.word = (uint32_t *)malloc(sizeof(uint32_t) * (max_len + 1));
    d.chart = (uint8_t *)malloc((size_t)Q * (max_len + 1) * (max_len + 1));
    int rc = 0;
    if (!d.path || !d.word || !d.chart) rc = -3;
    else {
        out_off[0] = 0;
        dfs_paths(&d, vs, 0);
        *n_paths = d.n_paths;
        if (d.overflow) rc = -4;
    }
    free(d.path); free(d.word); free(d.chart); free_edges(&E);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Rows of C = M3^+ for a given set of nonterminal matrices.                  */
/* ------------------------------------------------------------------------ */
/*
 * m2_nt [B * n * wn]: M2^b for every box (the final graph's nonterminal edges).
 * For every requested product vertex (row_state[k], row_vertex[k]) the output
 * row out[k * wN ...] holds the product vertices t*n + y reachable by a path of
 * one or more M3 edges, M3 = OR_l M1^l (x) M2^l.
 */
int orc_closure_rows(uint32_t n, uint32_t n_term, uint64_t m, const uint32_t *src, const uint32_t *lbl,
                     const uint32_t *dst, uint32_t Q, uint32_t B, const uint32_t *box_start,
                     const uint32_t *state_box, const uint8_t *state_final, uint32_t T, const uint32_t *tr_from,
                     const uint32_t *tr_kind, const uint32_t *tr_sym, const uint32_t *tr_to,
                     const uint64_t *m2_nt, uint32_t n_rows, const uint32_t *row_state,
                     const uint32_t *row_vertex, uint64_t *out) {
    orc_rsm r = {Q, B, box_start, state_box, state_final, T, tr_from, tr_kind, tr_sym, tr_to};
    if (check_graph(n, n_term, m, src, lbl, dst) || check_rsm(&r, n_term)) return -1;
    const uint64_t wn = words_for(n), N = (uint64_t)Q * n, wN = words_for(N);
    orc_edges E;
    memset(&E, 0, sizeof(E));
    if (dedupe_edges(n, m, src, lbl, dst, &E)) { free_edges(&E); return -3; }
    uint32_t *stack = (uint32_t *)malloc(sizeof(uint32_t) * (N + 1));
    if (!stack) { free_edges(&E); return -3; }
    int rc = 0;
    for (uint32_t k = 0; k < n_rows && rc == 0; ++k) {
        if (row_state[k] >= Q || row_vertex[k] >= n) { rc = -1; break; }
        uint64_t *row = out + (uint64_t)k * wN;
        memset(row, 0, sizeof(uint64_t) * wN);
        uint64_t sp = 0;
        /* successors of (s, x): (t, y) with s -l-> t and M2^l[x, y] */
        uint64_t start = (uint64_t)row_state[k] * n + row_vertex[k];
        uint64_t cur = start;
        int first = 1;
        while (first || sp) {
            if (!first) cur = stack[--sp];
            first = 0;
            uint32_t s = (uint32_t)(cur / n), x = (uint32_t)(cur % n);
            for (uint32_t t = 0; t < T; ++t) {
                if (tr_from[t] != s) continue;
                uint32_t to = tr_to[t];
                if (tr_kind[t] == ORC_TERM) {
                    for (uint64_t e = E.off[x]; e < E.off[x + 1]; ++e) {
                        if (E.el[e] != tr_sym[t]) continue;
                        uint64_t v = (uint64_t)to * n + E.ed[e];
                        if (!bget(row, v)) { bset(row, v); stack[sp++] = (uint32_t)v; }
                    }
                } else {
                    const uint64_t *mr = m2_nt + ((uint64_t)tr_sym[t] * n + x) * wn;
                    for (uint32_t y = 0; y < n; ++y)
                        if (bget(mr, y)) {
                            uint64_t v = (uint64_t)to * n + y;
                            if (!bget(row, v)) { bset(row, v); stack[sp++] = (uint32_t)v; }
                        }
                }
            }
        }
    }
    free(stack);
    free_edges(&E);
    return rc;
}
