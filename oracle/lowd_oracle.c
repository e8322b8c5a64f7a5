/*
 * Plain sequential CPU oracle for LOWD ("Locally Optimal Weight Distribution",
 * arXiv 2307.15969) with pruning and extraction, plus exact test-only solvers.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code with the
 * CUDA library: it is written from the paper's definitions and algorithms, in
 * double precision for the iteration and exact 64/128-bit integers for weights,
 * degrees and densities.
 *
 * Weights arrive as integer "units": unit weights use 1 unit per edge (scale 1);
 * weighted graphs use units of 2^-20 (scale 2^20), the grid the inputs are put on,
 * so that every degree, W(H) and W(S_k) below is an exact integer and every density
 * comparison W_a/k_a < W_b/k_b is done exactly as W_a*k_b < W_b*k_a in 128 bits.
 *
 * Contents (paper section in brackets):
 *   orc_canonicalize   undirected, loop-free, duplicate-free edge list   [Sec. IV, datasets]
 *   orc_degrees        weighted degree d_S(u)                           [Sec. II, Table I]
 *   orc_degree_order   counting sort of nodes by degree                 [Sec. III-D]
 *   orc_prune          Algorithm 2 (pruning), synchronous rounds        [Sec. III-D, Alg. 2]
 *   orc_lowd_update    body of Algorithm 1 for one edge                 [Alg. 1]
 *   orc_lowd_init      equal split, initial loads                       [Alg. 1 init]
 *   orc_lowd_iterate   T passes of the edge loop in a given edge order  [Alg. 1]
 *   orc_extract        argsort by load, peel lowest, best prefix        [Alg. 1 extraction]
 *   orc_level_colouring  pass order for graphs of any size (conflict-free batches; the
 *                      paper visits edges in any order, Fig. 1 caption)
 *   orc_star_update    exact minimiser of sum l^2 over one star's splits (the local
 *                      optimality of Sec. III-C over a block of edges)
 *   orc_star_round     star updates over a list of stars, in order
 *   orc_greedy         Charikar peeling (test-only cross-check)         [Alg. 3]
 *   orc_densest_flow   exact rho* and maximal densest set by min cut    [Sec. I, Goldberg]
 *   orc_ldd            exact locally-dense decomposition by min cuts    [Sec. II, Def. LDD]
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef __int128 i128;

/* ------------------------------------------------------------------ utilities */

/* a/b < c/d for b,d > 0, exactly */
static int frac_less(int64_t a, int64_t b, int64_t c, int64_t d) {
    return (i128)a * (i128)d < (i128)c * (i128)b;
}

typedef struct { uint64_t key; int64_t idx; } keyidx;

static int cmp_keyidx(const void* x, const void* y) {
    const keyidx* a = (const keyidx*)x;
    const keyidx* b = (const keyidx*)y;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

/* CSR adjacency of an undirected edge list: for node x, the entries
 * adj[off[x] .. off[x+1]) hold (neighbour, edge id). */
typedef struct { int64_t* off; int32_t* nbr; int64_t* eid; } adjacency;

static int build_adj(int32_t n, int64_t m, const int32_t* u, const int32_t* v, adjacency* A) {
    A->off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    A->nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    A->eid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * m + 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!A->off || !A->nbr || !A->eid || !fill) { free(fill); return -1; }
    for (int64_t e = 0; e < m; ++e) { A->off[u[e] + 1]++; A->off[v[e] + 1]++; }
    for (int32_t x = 0; x < n; ++x) A->off[x + 1] += A->off[x];
    memcpy(fill, A->off, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t e = 0; e < m; ++e) {
        A->nbr[fill[u[e]]] = v[e]; A->eid[fill[u[e]]++] = e;
        A->nbr[fill[v[e]]] = u[e]; A->eid[fill[v[e]]++] = e;
    }
    free(fill);
    return 0;
}

static void free_adj(adjacency* A) { free(A->off); free(A->nbr); free(A->eid); }

/* ------------------------------------------------------------------ input */

/* Undirected, loop-free, duplicate-free edge list (the paper removes multiple
 * edges and self-loops and ignores direction, Sec. IV).  Loops are rejected
 * (return -2), out-of-range ids too (-1); a repeated pair keeps the weight of
 * its first occurrence in input order.  Output is sorted by (lo, hi).
 * Returns the number of edges written. */
int64_t orc_canonicalize(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                         const double* w, int32_t* out_u, int32_t* out_v, double* out_w,
                         int64_t* n_dup) {
    keyidx* k = (keyidx*)malloc(sizeof(keyidx) * (size_t)(m + 1));
    if (!k) return -3;
    for (int64_t e = 0; e < m; ++e) {
        if (u[e] < 0 || u[e] >= n || v[e] < 0 || v[e] >= n) { free(k); return -1; }
        if (u[e] == v[e]) { free(k); return -2; }
        uint64_t lo = (uint64_t)(u[e] < v[e] ? u[e] : v[e]);
        uint64_t hi = (uint64_t)(u[e] < v[e] ? v[e] : u[e]);
        k[e].key = (lo << 32) | hi;
        k[e].idx = e;
    }
    qsort(k, (size_t)m, sizeof(keyidx), cmp_keyidx);
    int64_t out = 0, dup = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (i > 0 && k[i].key == k[i - 1].key) { dup++; continue; }
        out_u[out] = (int32_t)(k[i].key >> 32);
        out_v[out] = (int32_t)(k[i].key & 0xffffffffu);
        if (out_w) out_w[out] = w ? w[k[i].idx] : 1.0;
        out++;
    }
    if (n_dup) *n_dup = dup;
    free(k);
    return out;
}

/* ------------------------------------------------------------------ degrees + counting sort */

/* d(u) = total weight of edges at u (Table I; Sec. II). */
void orc_degrees(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                 const int64_t* wu, int64_t* deg) {
    for (int32_t x = 0; x < n; ++x) deg[x] = 0;
    for (int64_t e = 0; e < m; ++e) { deg[u[e]] += wu[e]; deg[v[e]] += wu[e]; }
}

static int cmp_deg_id(const void* x, const void* y) {
    const keyidx* a = (const keyidx*)x;
    const keyidx* b = (const keyidx*)y;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

/* Nodes ordered by degree ascending, equal degrees by id ascending.
 * Unit weights: the counting sort the paper describes (one bucket per degree
 * 0..d_max, nodes appended to their bucket in id order, buckets read in order;
 * Sec. III-D).  Weighted degrees: a comparison sort with the same order. */
void orc_degree_order(int32_t n, const int64_t* deg, int32_t weighted, int32_t* perm) {
    if (!weighted) {
        int64_t dmax = 0;
        for (int32_t x = 0; x < n; ++x) if (deg[x] > dmax) dmax = deg[x];
        int64_t* start = (int64_t*)calloc((size_t)dmax + 2, sizeof(int64_t));
        for (int32_t x = 0; x < n; ++x) start[deg[x] + 1]++;
        for (int64_t d = 0; d <= dmax; ++d) start[d + 1] += start[d];
        for (int32_t x = 0; x < n; ++x) perm[start[deg[x]]++] = x;
        free(start);
        return;
    }
    keyidx* k = (keyidx*)malloc(sizeof(keyidx) * ((size_t)n + 1));
    for (int32_t x = 0; x < n; ++x) { k[x].key = (uint64_t)deg[x]; k[x].idx = x; }
    qsort(k, (size_t)n, sizeof(keyidx), cmp_deg_id);
    for (int32_t x = 0; x < n; ++x) perm[x] = (int32_t)k[x].idx;
    free(k);
}

/* ------------------------------------------------------------------ Algorithm 2 */

/* Pruning (Alg. 2): H <- G; delta <- rho(H); while some nodes of H have
 * d_H(u) < delta, remove all of them at once with their edges and set
 * delta <- rho(H) again.  The test d_H(u) < W(H)/|H| is done as
 * d_H(u)*|H| < W(H) in exact integers.  removal_round[x] is the 1-based round
 * in which x was removed, or -1 if x is kept.  Returns the number of rounds
 * that removed something.
 *
 * Unit weights follow the paper's counting-sort scheme: nodes sit in buckets by
 * current degree, and a round only inspects the buckets below the new bound,
 * a node whose degree drops being moved to its new bucket.  Weighted graphs scan
 * all remaining nodes each round, as the paper states for that case. */
int32_t orc_prune(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                  const int64_t* wu, int32_t weighted, int32_t* removal_round,
                  int64_t* W_out, int32_t* N_out) {
    adjacency A;
    if (build_adj(n, m, u, v, &A)) return -1;
    int64_t* deg = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    orc_degrees(n, m, u, v, wu, deg);
    int64_t W = 0;
    for (int64_t e = 0; e < m; ++e) W += wu[e];
    int64_t N = n;
    for (int32_t x = 0; x < n; ++x) removal_round[x] = -1;
    int32_t* batch = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t rounds = 0;

    /* buckets for the unit-weight case: doubly linked lists per degree */
    int64_t dmax = 0;
    for (int32_t x = 0; x < n; ++x) if (deg[x] > dmax) dmax = deg[x];
    int32_t *head = NULL, *next = NULL, *prev = NULL;
    if (!weighted) {
        head = (int32_t*)malloc(sizeof(int32_t) * ((size_t)dmax + 1));
        next = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
        prev = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
        for (int64_t d = 0; d <= dmax; ++d) head[d] = -1;
        for (int32_t x = n - 1; x >= 0; --x) {       /* ascending ids inside a bucket */
            int64_t d = deg[x];
            next[x] = head[d]; prev[x] = -1;
            if (head[d] >= 0) prev[head[d]] = x;
            head[d] = x;
        }
    }
    while (N > 0) {
        int32_t nb = 0;
        if (!weighted) {
            /* all buckets d with d*N < W */
            for (int64_t d = 0; d <= dmax && (i128)d * N < (i128)W; ++d)
                for (int32_t x = head[d]; x >= 0; x = next[x]) batch[nb++] = x;
        } else {
            for (int32_t x = 0; x < n; ++x)
                if (removal_round[x] < 0 && (i128)deg[x] * N < (i128)W) batch[nb++] = x;
        }
        if (nb == 0) break;
        rounds++;
        for (int32_t i = 0; i < nb; ++i) removal_round[batch[i]] = rounds;
        for (int32_t i = 0; i < nb; ++i) {
            int32_t x = batch[i];
            if (!weighted) {   /* unlink x from its bucket */
                int64_t d = deg[x];
                if (prev[x] >= 0) next[prev[x]] = next[x]; else head[d] = next[x];
                if (next[x] >= 0) prev[next[x]] = prev[x];
            }
        }
        for (int32_t i = 0; i < nb; ++i) {
            int32_t x = batch[i];
            for (int64_t p = A.off[x]; p < A.off[x + 1]; ++p) {
                int32_t y = A.nbr[p];
                int64_t w = wu[A.eid[p]];
                if (removal_round[y] >= 0 && removal_round[y] < rounds) continue; /* gone */
                if (removal_round[y] == rounds) {          /* both ends removed now */
                    if (x < y) W -= w;
                    continue;
                }
                W -= w;
                if (!weighted) {   /* move y to the bucket of its new degree */
                    int64_t d = deg[y];
                    if (prev[y] >= 0) next[prev[y]] = next[y]; else head[d] = next[y];
                    if (next[y] >= 0) prev[next[y]] = prev[y];
                    deg[y] -= w;
                    d = deg[y];
                    next[y] = head[d]; prev[y] = -1;
                    if (head[d] >= 0) prev[head[d]] = y;
                    head[d] = y;
                } else {
                    deg[y] -= w;
                }
            }
        }
        N -= nb;
    }
    if (W_out) *W_out = W;
    if (N_out) *N_out = (int32_t)N;
    free(head); free(next); free(prev);
    free(batch); free(deg); free_adj(&A);
    return rounds;
}

/* ------------------------------------------------------------------ Algorithm 1 */

/* One application of the loop body of Alg. 1 to edge e = (u, v):
 * if l_u > l_v, move d = min((l_u - l_v)/2, f_e(u)) from u to v,
 * otherwise move d = min((l_v - l_u)/2, f_e(v)) from v to u.
 * Returns d (the amount moved, always >= 0). */
double orc_lowd_update(double* lu, double* lv, double* fu, double* fv) {
    double d;
    if (*lu > *lv) {
        d = fmin((*lu - *lv) / 2.0, *fu);
        *lu -= d; *fu -= d; *lv += d; *fv += d;
    } else {
        d = fmin((*lv - *lu) / 2.0, *fv);
        *lu += d; *fu += d; *lv -= d; *fv -= d;
    }
    return d;
}

/* Alg. 1 initialisation: f_e(u) = f_e(v) = w_e/2, l_u = sum of f_e(u) over e at u. */
void orc_lowd_init(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                   const double* w, double* fu, double* fv, double* l) {
    for (int32_t x = 0; x < n; ++x) l[x] = 0.0;
    for (int64_t e = 0; e < m; ++e) {
        fu[e] = w[e] / 2.0;
        fv[e] = w[e] / 2.0;
    }
    for (int64_t e = 0; e < m; ++e) { l[u[e]] += fu[e]; l[v[e]] += fv[e]; }
}

/* T passes of Alg. 1's edge loop.  Edges are visited in the order given by
 * order[0..m) (a permutation of edge ids), or 0..m-1 if order is NULL; each
 * update sees the loads left by the previous one.  If sumsq is not NULL, the
 * sum of squared loads after every pass is written to sumsq[0..T). */
void orc_lowd_iterate(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                      const int32_t* order, int32_t T, double* fu, double* fv, double* l,
                      double* sumsq) {
    for (int32_t t = 0; t < T; ++t) {
        for (int64_t i = 0; i < m; ++i) {
            int64_t e = order ? order[i] : i;
            orc_lowd_update(&l[u[e]], &l[v[e]], &fu[e], &fv[e]);
        }
        if (sumsq) {
            double s = 0.0;
            for (int32_t x = 0; x < n; ++x) s += l[x] * l[x];
            sumsq[t] = s;
        }
    }
}

static const double* g_sort_load;
static int cmp_load_id(const void* x, const void* y) {
    int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
    if (g_sort_load[a] != g_sort_load[b]) return g_sort_load[a] < g_sort_load[b] ? -1 : 1;
    return a < b ? -1 : (a > b);
}

/* Alg. 1 extraction: V_s = nodes sorted by load ascending (ties by id
 * ascending); S* = S = V; for i = 1..N-1 remove V_s(i) from S and keep S as the
 * new S* when rho(S*) < rho(S) strictly.  The empty set (i = N) is not a
 * candidate.  W(S) is kept exactly in weight units.  Writes the ids of S* to
 * S_out (ascending), its weight to *W_best; returns |S*|. */
int32_t orc_extract(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                    const int64_t* wu, const double* l, int32_t* S_out, int64_t* W_best) {
    if (n <= 0) { if (W_best) *W_best = 0; return 0; }
    adjacency A;
    if (build_adj(n, m, u, v, &A)) return -1;
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t x = 0; x < n; ++x) order[x] = x;
    g_sort_load = l;
    qsort(order, (size_t)n, sizeof(int32_t), cmp_load_id);
    char* in = (char*)malloc((size_t)n);
    memset(in, 1, (size_t)n);
    int64_t W = 0;
    for (int64_t e = 0; e < m; ++e) W += wu[e];
    int64_t bestW = W, bestK = n, removed_at_best = 0;
    int64_t k = n;
    for (int32_t i = 0; i < n - 1; ++i) {
        int32_t x = order[i];
        in[x] = 0;
        for (int64_t p = A.off[x]; p < A.off[x + 1]; ++p)
            if (in[A.nbr[p]]) W -= wu[A.eid[p]];
        k -= 1;
        if (frac_less(bestW, bestK, W, k)) { bestW = W; bestK = k; removed_at_best = i + 1; }
    }
    memset(in, 0, (size_t)n);
    for (int64_t i = removed_at_best; i < n; ++i) in[order[i]] = 1;
    int32_t c = 0;
    for (int32_t x = 0; x < n; ++x) if (in[x]) S_out[c++] = x;
    if (W_best) *W_best = bestW;
    free(in); free(order); free_adj(&A);
    return c;
}

/* ------------------------------------------------------------------ Algorithm 3 (test-only) */

/* Charikar's greedy peeling (Alg. 3): repeatedly delete a node of minimum
 * degree in the remaining graph (ties: smallest id), recording the removal
 * sequence and the density after each removal.  order_out[i] is the i-th node
 * removed; W_after[i] the weight left after it.  O(n^2 + m): test sizes only. */
void orc_greedy(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                const int64_t* wu, int32_t* order_out, int64_t* W_after) {
    adjacency A;
    if (build_adj(n, m, u, v, &A)) return;
    int64_t* deg = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    char* in = (char*)malloc((size_t)n + 1);
    orc_degrees(n, m, u, v, wu, deg);
    memset(in, 1, (size_t)n);
    int64_t W = 0;
    for (int64_t e = 0; e < m; ++e) W += wu[e];
    for (int32_t i = 0; i < n; ++i) {
        int32_t best = -1;
        for (int32_t x = 0; x < n; ++x)
            if (in[x] && (best < 0 || deg[x] < deg[best])) best = x;
        in[best] = 0;
        for (int64_t p = A.off[best]; p < A.off[best + 1]; ++p) {
            int32_t y = A.nbr[p];
            if (in[y]) { deg[y] -= wu[A.eid[p]]; W -= wu[A.eid[p]]; }
        }
        order_out[i] = best;
        W_after[i] = W;
    }
    free(deg); free(in); free_adj(&A);
}

/* ------------------------------------------------------------------ exact min cut (test-only) */

typedef struct { int32_t to; int64_t cap; int64_t rev; } arc;
typedef struct {
    int32_t nv; int64_t na, cap_arcs;
    arc* a; int64_t* head_off; int32_t* level; int64_t* it; int32_t* queue;
    int32_t* src_node; int64_t* arc_cnt;
} flownet;

/* Dinic's maximum flow on a network whose arcs are given as (from, to, cap, rcap)
 * quadruples; built once in CSR form. */
static int net_build(flownet* F, int32_t nv, int64_t ne, const int32_t* fr, const int32_t* to,
                     const int64_t* cap, const int64_t* rcap) {
    F->nv = nv; F->na = 2 * ne;
    F->a = (arc*)malloc(sizeof(arc) * (size_t)(F->na + 1));
    F->head_off = (int64_t*)calloc((size_t)nv + 1, sizeof(int64_t));
    F->level = (int32_t*)malloc(sizeof(int32_t) * (size_t)nv);
    F->it = (int64_t*)malloc(sizeof(int64_t) * (size_t)nv);
    F->queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)nv);
    if (!F->a || !F->head_off || !F->level || !F->it || !F->queue) return -1;
    for (int64_t e = 0; e < ne; ++e) { F->head_off[fr[e] + 1]++; F->head_off[to[e] + 1]++; }
    for (int32_t x = 0; x < nv; ++x) F->head_off[x + 1] += F->head_off[x];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nv);
    memcpy(fill, F->head_off, sizeof(int64_t) * (size_t)nv);
    for (int64_t e = 0; e < ne; ++e) {
        int64_t p = fill[fr[e]]++, q = fill[to[e]]++;
        F->a[p].to = to[e]; F->a[p].cap = cap[e]; F->a[p].rev = q;
        F->a[q].to = fr[e]; F->a[q].cap = rcap[e]; F->a[q].rev = p;
    }
    free(fill);
    return 0;
}

static void net_free(flownet* F) {
    free(F->a); free(F->head_off); free(F->level); free(F->it); free(F->queue);
}

static int net_bfs(flownet* F, int32_t s, int32_t t) {
    for (int32_t x = 0; x < F->nv; ++x) F->level[x] = -1;
    int32_t qh = 0, qt = 0;
    F->queue[qt++] = s; F->level[s] = 0;
    while (qh < qt) {
        int32_t x = F->queue[qh++];
        for (int64_t p = F->head_off[x]; p < F->head_off[x + 1]; ++p)
            if (F->a[p].cap > 0 && F->level[F->a[p].to] < 0) {
                F->level[F->a[p].to] = F->level[x] + 1;
                F->queue[qt++] = F->a[p].to;
            }
    }
    return F->level[t] >= 0;
}

/* blocking flow by iterative DFS along the level graph */
static i128 net_block(flownet* F, int32_t s, int32_t t, int32_t* stack, int64_t* stack_arc) {
    i128 total = 0;
    for (int32_t x = 0; x < F->nv; ++x) F->it[x] = F->head_off[x];
    for (;;) {
        int32_t depth = 0;
        stack[0] = s;
        int found = 0;
        while (depth >= 0) {
            int32_t x = stack[depth];
            if (x == t) { found = 1; break; }
            int advanced = 0;
            for (; F->it[x] < F->head_off[x + 1]; ++F->it[x]) {
                arc* ar = &F->a[F->it[x]];
                if (ar->cap > 0 && F->level[ar->to] == F->level[x] + 1) {
                    stack_arc[depth] = F->it[x];
                    stack[++depth] = ar->to;
                    advanced = 1;
                    break;
                }
            }
            if (!advanced) {
                F->level[x] = -1;   /* dead end */
                depth--;
                if (depth >= 0) F->it[stack[depth]]++;
            }
        }
        if (!found) break;
        int64_t push = INT64_MAX;
        for (int32_t i = 0; i < depth; ++i)
            if (F->a[stack_arc[i]].cap < push) push = F->a[stack_arc[i]].cap;
        for (int32_t i = 0; i < depth; ++i) {
            arc* ar = &F->a[stack_arc[i]];
            ar->cap -= push;
            F->a[ar->rev].cap += push;
        }
        total += push;
    }
    return total;
}

static i128 net_maxflow(flownet* F, int32_t s, int32_t t) {
    int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * ((size_t)F->nv + 1));
    int64_t* stack_arc = (int64_t*)malloc(sizeof(int64_t) * ((size_t)F->nv + 1));
    i128 flow = 0;
    while (net_bfs(F, s, t)) flow += net_block(F, s, t, stack, stack_arc);
    free(stack); free(stack_arc);
    return flow;
}

/* Maximise F(S) = W(S) + c(S) - g|S| over S subset of the nodes with alive[x],
 * g = p/q, by Goldberg's cut construction scaled by q:
 *   s->x: q*Mb,   x->t: q*Mb + 2p - q*(d_x + 2 c_x),   x<->y: q*w_xy,
 * where d_x is the degree among alive nodes and Mb >= max(d_x + 2 c_x).
 * A cut with source side {s} + S costs q*Mb*n_alive + 2q*(g|S| - W(S) - c(S)).
 * in_S receives the LARGEST maximiser: nodes that cannot reach t in the residual
 * network.  Returns 1 if max F > 0, 0 if max F == 0, -1 on overflow/alloc error. */
static int best_set(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const int64_t* wu,
                    const char* alive, const int64_t* c, int64_t p, int64_t q, char* in_S) {
    int64_t* dg = (int64_t*)calloc((size_t)n, sizeof(int64_t));
    int64_t na = 0;
    for (int64_t e = 0; e < m; ++e)
        if (alive[u[e]] && alive[v[e]]) { dg[u[e]] += wu[e]; dg[v[e]] += wu[e]; na++; }
    int32_t nal = 0;
    int64_t Mb = 1;
    for (int32_t x = 0; x < n; ++x)
        if (alive[x]) { nal++; if (dg[x] + 2 * c[x] > Mb) Mb = dg[x] + 2 * c[x]; }
    if ((i128)q * Mb + 2 * (i128)p > ((i128)1 << 60) ||
        (i128)q * Mb * (nal + 1) > ((i128)1 << 120)) { free(dg); return -1; }
    int32_t s = n, t = n + 1;
    int64_t ne = 2 * (int64_t)nal + na;
    int32_t* fr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ne + 1));
    int32_t* to = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ne + 1));
    int64_t* cp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ne + 1));
    int64_t* rc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ne + 1));
    int64_t k = 0;
    for (int32_t x = 0; x < n; ++x) {
        if (!alive[x]) continue;
        fr[k] = s; to[k] = x; cp[k] = q * Mb; rc[k] = 0; k++;
        fr[k] = x; to[k] = t; cp[k] = q * Mb + 2 * p - q * (dg[x] + 2 * c[x]); rc[k] = 0; k++;
    }
    for (int64_t e = 0; e < m; ++e)
        if (alive[u[e]] && alive[v[e]]) {
            fr[k] = u[e]; to[k] = v[e]; cp[k] = q * wu[e]; rc[k] = q * wu[e]; k++;
        }
    flownet F;
    if (net_build(&F, n + 2, k, fr, to, cp, rc)) { free(dg); return -1; }
    free(fr); free(to); free(cp); free(rc);
    i128 flow = net_maxflow(&F, s, t);
    /* nodes that reach t in the residual network: reverse BFS from t */
    char* reach_t = (char*)calloc((size_t)n + 2, 1);
    int32_t* qu = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 2));
    int32_t qh = 0, qt = 0;
    qu[qt++] = t; reach_t[t] = 1;
    while (qh < qt) {
        int32_t y = qu[qh++];
        for (int64_t pp = F.head_off[y]; pp < F.head_off[y + 1]; ++pp) {
            /* arc y->z's reverse is z->y; z reaches y if residual cap(z->y) > 0 */
            int32_t z = F.a[pp].to;
            if (!reach_t[z] && F.a[F.a[pp].rev].cap > 0) { reach_t[z] = 1; qu[qt++] = z; }
        }
    }
    for (int32_t x = 0; x < n; ++x) in_S[x] = (char)(alive[x] && !reach_t[x]);
    i128 full = (i128)q * Mb * nal;
    free(reach_t); free(qu); net_free(&F); free(dg);
    return flow < full ? 1 : 0;
}

/* Exact densest subgraph of the sub-graph induced by alive nodes, with extra node
 * weights c (edges to an already removed set): Dinkelbach's iteration on
 * g = (W(S)+c(S))/|S| starting from the whole alive set; each step solves
 * max_S F(S) by a min cut.  Returns |S| (S in in_S, the maximal maximiser) and
 * the optimum as num/den. */
static int32_t densest_with_c(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                              const int64_t* wu, const char* alive, const int64_t* c,
                              char* in_S, int64_t* num, int64_t* den) {
    int64_t p = 0, q = 0;
    for (int32_t x = 0; x < n; ++x) if (alive[x]) { q++; p += c[x]; }
    for (int64_t e = 0; e < m; ++e) if (alive[u[e]] && alive[v[e]]) p += wu[e];
    if (q == 0) { *num = 0; *den = 1; return 0; }
    char* cur = (char*)malloc((size_t)n + 1);
    for (int iter = 0; iter < 1000; ++iter) {
        int r = best_set(n, m, u, v, wu, alive, c, p, q, cur);
        if (r < 0) { free(cur); return -1; }
        if (r == 0) break;
        int64_t np = 0, nq = 0;
        for (int32_t x = 0; x < n; ++x) if (cur[x]) { nq++; np += c[x]; }
        for (int64_t e = 0; e < m; ++e) if (cur[u[e]] && cur[v[e]]) np += wu[e];
        p = np; q = nq;
    }
    /* at the optimum g the maximal maximiser of F (value 0) is the answer */
    int r = best_set(n, m, u, v, wu, alive, c, p, q, in_S);
    free(cur);
    if (r != 0) return -1;
    int32_t k = 0;
    for (int32_t x = 0; x < n; ++x) k += in_S[x] ? 1 : 0;
    /* g = p/q is attained by the maximal set as well */
    *num = p; *den = q;
    return k;
}

/* rho* = max_S W(S)/|S| (Problem 1) and the maximal densest set B_1, exactly.
 * Returns |B_1|; in_S[x] = 1 for x in B_1; rho* = *W_num / *k_den in weight units. */
int32_t orc_densest_flow(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                         const int64_t* wu, char* in_S, int64_t* W_num, int64_t* k_den) {
    char* alive = (char*)malloc((size_t)n + 1);
    int64_t* c = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    memset(alive, 1, (size_t)n);
    int32_t k = densest_with_c(n, m, u, v, wu, alive, c, in_S, W_num, k_den);
    free(alive); free(c);
    return k;
}

/* Locally-dense decomposition (Def. LDD): B_0 = {}, B_i = the maximal set
 * S strictly containing B_{i-1} that maximises (W(S) - W(B_{i-1}))/|S \ B_{i-1}|.
 * On the nodes outside B_{i-1} this is a densest-subgraph problem in which node x
 * carries c_x = weight of its edges into B_{i-1}.  shell[x] = i for
 * x in B_i \ B_{i-1} (1-based); lambda_i = lam_num[i-1]/lam_den[i-1].
 * Returns the number of shells k, or -1. */
int32_t orc_ldd(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const int64_t* wu,
                int32_t* shell, int64_t* lam_num, int64_t* lam_den) {
    char* alive = (char*)malloc((size_t)n + 1);
    char* in_S = (char*)malloc((size_t)n + 1);
    int64_t* c = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    memset(alive, 1, (size_t)n);
    for (int32_t x = 0; x < n; ++x) shell[x] = 0;
    int32_t left = n, k = 0;
    adjacency A;
    build_adj(n, m, u, v, &A);
    while (left > 0) {
        int64_t num, den;
        int32_t got = densest_with_c(n, m, u, v, wu, alive, c, in_S, &num, &den);
        if (got <= 0) { k = -1; break; }
        lam_num[k] = num; lam_den[k] = den;
        k++;
        for (int32_t x = 0; x < n; ++x)
            if (in_S[x]) { shell[x] = k; alive[x] = 0; left--; }
        for (int32_t x = 0; x < n; ++x)
            if (shell[x] == k)
                for (int64_t p = A.off[x]; p < A.off[x + 1]; ++p)
                    if (alive[A.nbr[p]]) c[A.nbr[p]] += wu[A.eid[p]];
    }
    free_adj(&A); free(alive); free(in_S); free(c);
    return k;
}

/* Sum of l, sum of l^2 and max l in one pass (the quantities of Sec. III:
 * conservation, the QP objective and D = max l). */
void orc_load_stats(int32_t n, const double* l, double* out3) {
    double s = 0.0, s2 = 0.0, mx = -INFINITY;
    for (int32_t x = 0; x < n; ++x) { s += l[x]; s2 += l[x] * l[x]; if (l[x] > mx) mx = l[x]; }
    out3[0] = s; out3[1] = s2; out3[2] = n > 0 ? mx : 0.0;
}

/* ------------------------------------------------------------------ pass order (any size) */

typedef struct { uint64_t key; uint32_t tie; int64_t e; } edgekey;

static int cmp_edgekey(const void* x, const void* y) {
    const edgekey* a = (const edgekey*)x;
    const edgekey* b = (const edgekey*)y;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->tie != b->tie) return a->tie < b->tie ? -1 : 1;
    return a->e < b->e ? -1 : (a->e > b->e);
}

/* The 32-bit finaliser of Appleby's MurmurHash3 (fmix32), a bijection on 32-bit words:
 * it orders edges of equal degree key in a scrambled, fixed order. */
static uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

/* A proper edge colouring whose colour classes, visited in ascending colour, give a pass
 * of Algorithm 1 in the order "edges by ascending key" (any order is allowed, Fig. 1
 * caption): edges sharing an endpoint keep their key order, and edges with no endpoint in
 * common commute.  The key of e = (a, b) is (max(d_a, d_b), min(d_a, d_b), fmix32(e)), d the
 * unweighted degree: light edges first, so early classes are large and the long tail of
 * classes holds the edges of the highest-degree nodes.  Ties of degree are broken by a
 * scrambled edge id, not the id itself: edges listed in id order along a path or a chain
 * of equal-degree nodes would otherwise each wait for the previous one.
 *
 * colour(e) = 1 + the largest colour among the edges that share an endpoint with e and come
 * before it in key order (0 if there is none): the level of e in that dependency order.  Two
 * edges at one node differ in colour, so every class is a matching; a node of degree d has
 * d edges with distinct colours, so there are at least max d colours.  Scanning the edges in
 * key order, the largest earlier colour at a node is the colour of its latest edge so far.
 * Writes colour[e]; returns the number of colours, or -1 on allocation failure. */
int32_t orc_level_colouring(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                            int32_t* colour) {
    int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    edgekey* k = (edgekey*)malloc(sizeof(edgekey) * (size_t)(m + 1));
    int32_t* last = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!deg || !k || !last) { free(deg); free(k); free(last); return -1; }
    for (int64_t e = 0; e < m; ++e) { deg[u[e]]++; deg[v[e]]++; }
    for (int64_t e = 0; e < m; ++e) {
        uint64_t da = (uint64_t)deg[u[e]], db = (uint64_t)deg[v[e]];
        uint64_t hi = da > db ? da : db, lo = da > db ? db : da;
        k[e].key = (hi << 32) | lo;
        k[e].tie = fmix32((uint32_t)e);
        k[e].e = e;
    }
    qsort(k, (size_t)m, sizeof(edgekey), cmp_edgekey);
    for (int32_t x = 0; x < n; ++x) last[x] = -1;
    int32_t C = 0;
    for (int64_t i = 0; i < m; ++i) {
        int64_t e = k[i].e;
        int32_t c = (last[u[e]] > last[v[e]] ? last[u[e]] : last[v[e]]) + 1;
        colour[e] = c;
        last[u[e]] = c;
        last[v[e]] = c;
        if (c + 1 > C) C = c + 1;
    }
    free(deg); free(k); free(last);
    return C;
}


/* ------------------------------------------------------------------ hub-star block update */

typedef struct { double x; int32_t kind; } breakpoint;

static int cmp_breakpoint(const void* a, const void* b) {
    const breakpoint* p = (const breakpoint*)a;
    const breakpoint* q = (const breakpoint*)b;
    if (p->x != q->x) return p->x < q->x ? -1 : 1;
    return p->kind - q->kind;
}

/* Exact minimisation of the sum of squared loads over the splits of one star: hub h with
 * leaves j = 0..q-1 joined by edges of weight w[j]; t[j] = f_e(h) on input and output.  With
 * the other edges fixed, B_h = l_h - sum t and B_j = l_j - (w_j - t_j); the loads after are
 * L_h = B_h + sum t_j and L_j = B_j + w_j - t_j.  Setting the gradient to zero with the box
 * 0 <= t_j <= w_j gives t_j = clip(B_j + w_j - lam, 0, w_j) where lam = L_h solves
 *     g(lam) = B_h + sum_j clip(B_j + w_j - lam, 0, w_j) - lam = 0,
 * g strictly decreasing and piecewise linear with breakpoints B_j and B_j + w_j ("water
 * filling").  The breakpoints are sorted and g is followed from the left until it changes
 * sign; the root is then exact on that linear piece.  Updates lh, l[j] (loads of the leaves)
 * and t; returns lam.  A star of one leaf is Algorithm 1's edge update. */
double orc_star_update(int32_t q, double* lh, double* l, const double* w, double* t) {
    if (q <= 0) return *lh;
    breakpoint* bp = (breakpoint*)malloc(sizeof(breakpoint) * (size_t)(2 * q));
    double Bh = *lh;
    for (int32_t j = 0; j < q; ++j) Bh -= t[j];
    /* g at lam = -inf side: every clip is w_j (lam below all B_j).  Walk the breakpoints in
     * order: at B_j the term j starts falling with slope -1, at B_j + w_j it stops. */
    double sumw = 0.0;
    for (int32_t j = 0; j < q; ++j) {
        const double Bj = l[j] - (w[j] - t[j]);
        bp[2 * j].x = Bj;          bp[2 * j].kind = 0;   /* start of the falling piece */
        bp[2 * j + 1].x = Bj + w[j]; bp[2 * j + 1].kind = 1;   /* end of it */
        sumw += w[j];
    }
    qsort(bp, (size_t)(2 * q), sizeof(breakpoint), cmp_breakpoint);
    /* on a piece, g(lam) = C - (1 + a) lam with a = number of falling terms and
     * C = B_h + sum of w over terms left of their piece + sum of (B_j + w_j) over falling ones */
    double C = Bh + sumw;
    int32_t a = 0;
    double lam = 0.0;
    int found = 0;
    double left = -INFINITY;
    for (int32_t i = 0; i <= 2 * q && !found; ++i) {
        const double right = i < 2 * q ? bp[i].x : INFINITY;
        /* root of C - (1 + a) lam on [left, right] */
        const double r = C / (double)(1 + a);
        if (r <= right && r >= left) { lam = r; found = 1; break; }
        if (i == 2 * q) break;
        if (bp[i].kind == 0) {   /* term enters its falling piece: C += B_j + w_j - w_j = B_j */
            C += bp[i].x - 0.0;   /* adds (B_j + w_j) and removes w_j: net B_j */
            a += 1;
        } else {                 /* term leaves it: C -= (B_j + w_j) */
            C -= bp[i].x;
            a -= 1;
        }
        left = right;
    }
    if (!found) lam = C / (double)(1 + a);
    double Lh = Bh;
    for (int32_t j = 0; j < q; ++j) {
        const double Bj = l[j] - (w[j] - t[j]);
        double tj = Bj + w[j] - lam;
        if (tj < 0.0) tj = 0.0;
        if (tj > w[j]) tj = w[j];
        t[j] = tj;
        l[j] = Bj + w[j] - tj;
        Lh += tj;
    }
    *lh = Lh;
    free(bp);
    return lam;
}

/* One round of star updates: stars s = 0..ns-1 in order (all stars of step 0, then of step
 * 1, ...), star s = hub star_hub[s] with the edges star_edge[beg[s] .. beg[s+1]).  Each is set
 * by orc_star_update from the current loads and splits (fu/fv the shares of u/v).  Returns 0,
 * or -1 if scratch could not be allocated (nothing changed then). */
int32_t orc_star_round(int32_t ns, const int32_t* star_hub, const int64_t* beg, const int32_t* star_edge,
                       const int32_t* u, const int32_t* v, const double* w, double* fu, double* fv, double* l) {
    int64_t qmax = 0;
    for (int32_t s = 0; s < ns; ++s)
        if (beg[s + 1] - beg[s] > qmax) qmax = beg[s + 1] - beg[s];
    double* ll = (double*)malloc(sizeof(double) * (size_t)(qmax > 0 ? qmax : 1));
    double* ww = (double*)malloc(sizeof(double) * (size_t)(qmax > 0 ? qmax : 1));
    double* tt = (double*)malloc(sizeof(double) * (size_t)(qmax > 0 ? qmax : 1));
    if (!ll || !ww || !tt) { free(ll); free(ww); free(tt); return -1; }
    for (int32_t s = 0; s < ns; ++s) {
        const int32_t hub = star_hub[s];
        const int64_t b = beg[s];
        const int32_t q = (int32_t)(beg[s + 1] - b);
        for (int32_t j = 0; j < q; ++j) {
            const int32_t e = star_edge[b + j];
            const int hub_is_u = u[e] == hub;
            ll[j] = l[hub_is_u ? v[e] : u[e]];
            ww[j] = w ? w[e] : 1.0;
            tt[j] = hub_is_u ? fu[e] : fv[e];
        }
        double lh = l[hub];
        orc_star_update(q, &lh, ll, ww, tt);
        l[hub] = lh;
        for (int32_t j = 0; j < q; ++j) {
            const int32_t e = star_edge[b + j];
            const int hub_is_u = u[e] == hub;
            l[hub_is_u ? v[e] : u[e]] = ll[j];
            if (hub_is_u) { fu[e] = tt[j]; fv[e] = ww[j] - tt[j]; }
            else { fv[e] = tt[j]; fu[e] = ww[j] - tt[j]; }
        }
    }
    free(ll); free(ww); free(tt);
    return 0;
}
