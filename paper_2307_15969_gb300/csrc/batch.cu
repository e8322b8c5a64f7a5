// Batched LOWD: many independent graphs pruned, coloured, iterated and extracted by one
// persistent launch.  Each CTA takes graphs from a work queue (in an order chosen on the
// host) and runs the whole method on one graph at a time with its node state in shared
// memory:
//   Algorithm 2: degrees by shared-memory atomics, synchronous rounds (d(u)*|H| < W(H)
//     removes u; removed edges leave the surviving degrees and W(H)), surviving edges
//     appended to a per-graph scratch list;
//   compaction: survivors renumbered by a block-wide scan (ascending original id);
//   schedule: the circle colouring of the core, edges counting-sorted by colour (each
//     class a matching, so its updates run in parallel);
//   Algorithm 1: equal split, then `passes` passes of all classes in colour order with the
//     loads in shared memory; classes padded to 4 edges, staged global -> shared in chunks
//     by the last warp with bulk copies, consumers meeting at a named barrier per class
//     (an unstaged loop with a CTA barrier per class when the stages do not fit);
//   extraction: bitonic sort of (load desc, id desc), prefix weights by per-edge buckets
//     and a scan, the largest k maximising W(S_k)/k.
// Unit weights only.  Limits: a graph's node count must fit the shared-memory budget
// (5 bytes per node) and its core's extraction arrays (16 bytes per padded node); graphs
// beyond report a status instead of a result.
#include "ctx.cuh"
#include "prims.cuh"
#include "async.cuh"

#include <vector>
#include <algorithm>

using namespace lowd;

namespace {

constexpr int kBT = 512;  // threads per CTA (default)
// staged passes (producer warp + bulk copies), as in the single-graph sweep
constexpr int kBMaxStages = 8;
constexpr int kBStoreSlack = 1;
constexpr int kBStoreGroups = 8;
constexpr uint32_t kBWaitLimit = 1u << 22;

enum { BS_OK = 0, BS_TOO_MANY_NODES = 1, BS_CORE_TOO_LARGE = 2, BS_BAD_INPUT = 3, BS_WAIT_EXPIRED = 4 };

struct BatchArgs {
    int32_t B;
    const int64_t* node_off;   // [B+1]
    const int64_t* edge_off;   // [B+1]
    const int32_t* u;          // [m_total] local ids, u < v, strictly increasing per graph
    const int32_t* v;
    uint32_t* eA;              // [m_total + 4 n_total + 16] scratch: packed edges (ping)
    uint32_t* eB;              // same size: packed edges (pong / class-major, padded)
    float* cs;                 // same size: splits in class-major order
    int32_t* oldid;            // [n_total] scratch: core id -> local id
    const int32_t* order;      // [B] processing order
    int32_t* queue;            // work counter
    int32_t passes;
    uint32_t smem_bytes;
    double* rho;               // [B]
    int32_t* S_size;           // [B]
    int32_t* nH;               // [B]
    int32_t* mH;               // [B]
    int32_t* rounds;           // [B]
    int32_t* status;           // [B]
    uint8_t* in_S;             // [n_total]
    float* loads;              // [n_total] loads after the passes (0 for pruned nodes)
    uint8_t* in_core;          // [n_total] 1 if the node survived Algorithm 2
};

__device__ __forceinline__ int32_t block_sum_i32(int32_t x, int32_t* red) {
    x = warp_sum(x);
    __syncthreads();
    if (lane_id() == 0) red[warp_id()] = x;
    __syncthreads();
    int32_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;  // valid in every thread
}

// exclusive scan of a[0..len) in shared memory, in place; returns the total
__device__ int32_t block_scan_smem(int32_t* a, int32_t len, int32_t* red) {
    int32_t carry = 0;
    for (int32_t base = 0; base < len; base += blockDim.x) {
        const int32_t i = base + threadIdx.x;
        const int32_t x = i < len ? a[i] : 0;
        const int32_t inc = warp_incl_scan(x);
        __syncthreads();
        if (lane_id() == 31) red[warp_id()] = inc;
        __syncthreads();
        int32_t wpre = 0, tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const int32_t r = red[w];
            if (w < (int)warp_id()) wpre += r;
            tot += r;
        }
        if (i < len) a[i] = carry + wpre + inc - x;
        carry += tot;
    }
    __syncthreads();
    return carry;
}

__device__ __forceinline__ uint32_t pack(int32_t a, int32_t b) { return (uint32_t)a | ((uint32_t)b << 16); }

__global__ void __launch_bounds__(1024, 1) k_batch_lowd(BatchArgs A) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int32_t red[32];
    __shared__ int32_t s_graph, s_count, s_rem;
    __shared__ volatile int32_t s_bad;   // an edge id outside the core: recorded, never used
    __shared__ volatile int32_t s_abort; // a bounded wait of the staged passes expired
    __shared__ int32_t s_stage_len;
    const int tid = threadIdx.x;
    const int nt = blockDim.x;
    for (;;) {
        if (tid == 0) {
            const int32_t q = atomicAdd(A.queue, 1);
            s_graph = q < A.B ? A.order[q] : -1;
        }
        __syncthreads();
        const int32_t g = s_graph;
        if (tid == 0) { s_bad = 0; s_abort = 0; }
        __syncthreads();
        if (g < 0) break;
        const int64_t n0 = A.node_off[g], m0 = A.edge_off[g];
        const int32_t n = (int32_t)(A.node_off[g + 1] - n0);
        const int32_t m = (int32_t)(A.edge_off[g + 1] - m0);
        const int32_t* gu = A.u + m0;
        const int32_t* gv = A.v + m0;
        // scratch range of this graph: m edges plus up to 3 padding slots per class (<= n
        // classes), starting on a 16-byte boundary
        const int64_t so = ((m0 + 4 * n0) + 3) & ~(int64_t)3;
        uint32_t* eA = A.eA + so;
        uint32_t* eB = A.eB + so;
        float* cs = A.cs + so;
        int32_t* oldid = A.oldid + n0;
        uint8_t* inS = A.in_S + n0;
        float* lout = A.loads + n0;
        uint8_t* cout = A.in_core + n0;
        for (int32_t i = tid; i < n; i += nt) { inS[i] = 0; lout[i] = 0.0f; cout[i] = 0; }
        if ((uint64_t)n * 5u + 64u > A.smem_bytes || n > 65535) {
            if (tid == 0) { A.status[g] = BS_TOO_MANY_NODES; A.rho[g] = 0.0; A.S_size[g] = 0; }
            continue;
        }
        // ---------------- Algorithm 2 in shared memory
        int32_t* deg = reinterpret_cast<int32_t*>(sm);
        uint8_t* state = sm + 4 * (size_t)n;   // 0 live, 1 removed this round, 2 removed
        for (int32_t i = tid; i < n; i += nt) { deg[i] = 0; state[i] = 0; }
        __syncthreads();
        for (int32_t e = tid; e < m; e += nt) {
            atomicAdd(&deg[gu[e]], 1);
            atomicAdd(&deg[gv[e]], 1);
        }
        __syncthreads();
        int64_t W = m;
        int32_t N = n;
        int32_t me = m;              // live edges
        bool from_input = true;      // round 1 reads the input arrays
        uint32_t* cur = eA;
        uint32_t* nxt = eB;
        int32_t r = 0;
        for (;;) {
            int32_t k = 0;
            for (int32_t i = tid; i < n; i += nt)
                if (state[i] == 0 && (int64_t)deg[i] * N < W) { state[i] = 1; ++k; }
            k = block_sum_i32(k, red);
            if (k == 0) break;
            ++r;
            if (tid == 0) s_count = 0;
            __syncthreads();
            int32_t removed = 0;
            for (int32_t base = 0; base < me; base += nt) {
                const int32_t e = base + tid;
                bool keep = false;
                int32_t a = 0, b = 0;
                if (e < me) {
                    if (from_input) { a = gu[e]; b = gv[e]; }
                    else { const uint32_t p = cur[e]; a = (int32_t)(p & 0xffffu); b = (int32_t)(p >> 16); }
                    const uint8_t sa = state[a], sb = state[b];
                    if (sa == 1 || sb == 1) {
                        ++removed;
                        if (sa == 0) atomicSub(&deg[a], 1);
                        if (sb == 0) atomicSub(&deg[b], 1);
                    } else {
                        keep = true;
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                int32_t slot = 0;
                if (lane_id() == 0 && bal) slot = atomicAdd(&s_count, __popc(bal));
                slot = __shfl_sync(0xffffffffu, slot, 0);
                if (keep) nxt[slot + __popc(bal & ((1u << lane_id()) - 1u))] = pack(a, b);
            }
            removed = block_sum_i32(removed, red);
            for (int32_t i = tid; i < n; i += nt)
                if (state[i] == 1) state[i] = 2;
            W -= removed;
            N -= k;
            me = s_count;
            from_input = false;
            uint32_t* t = cur; cur = nxt; nxt = t;
            __syncthreads();
        }
        if (from_input) {  // nothing removed: the live edge list is the input
            for (int32_t e = tid; e < m; e += nt) cur[e] = pack(gu[e], gv[e]);
            __syncthreads();
        }
        // ---------------- compaction: survivors by ascending local id
        int32_t* newid = deg;   // reuse
        for (int32_t i = tid; i < n; i += nt) newid[i] = state[i] == 0 ? 1 : 0;
        __syncthreads();
        const int32_t nH = block_scan_smem(newid, n, red);
        for (int32_t i = tid; i < n; i += nt)
            if (state[i] == 0) oldid[newid[i]] = i;
        for (int32_t e = tid; e < me; e += nt) {
            const uint32_t p = cur[e];
            cur[e] = pack(newid[p & 0xffffu], newid[p >> 16]);
        }
        __syncthreads();
        const int32_t mH = me;
        const int32_t P = (nH + (nH & 1)) - 1 > 0 ? (nH + (nH & 1)) - 1 : 1;
        int32_t npow = 1;
        while (npow < nH) npow <<= 1;
        const size_t need = 4u * ((size_t)nH + 1) + 8u * ((size_t)P + 2) + 8u * (size_t)npow + 8u * (size_t)nH + 64u;
        if (need > A.smem_bytes) {
            if (tid == 0) {
                A.status[g] = BS_CORE_TOO_LARGE; A.rho[g] = 0.0; A.S_size[g] = 0;
                A.nH[g] = nH; A.mH[g] = mH; A.rounds[g] = r;
            }
            continue;
        }
        // ---------------- schedule: counting sort of the core's edges by circle colour,
        // each class padded to a multiple of 4 edges with no-op edges (nH, nH)
        float* L = reinterpret_cast<float*>(sm);                         // [nH + 1]
        int32_t* start = reinterpret_cast<int32_t*>(L + nH + 1);         // [P + 1]
        int32_t* cursor = start + P + 1;                                 // [P + 1]
        const uint32_t Np = (uint32_t)(nH + (nH & 1));
        const uint32_t sentinel = pack(nH, nH);
        for (int32_t i = tid; i <= P; i += nt) start[i] = 0;
        __syncthreads();
        auto colour = [&](uint32_t p) -> int32_t {
            const uint32_t a = p & 0xffffu, b = p >> 16;
            return (int32_t)((b == Np - 1) ? (2u * a) % (uint32_t)P : (a + b) % (uint32_t)P);
        };
        for (int32_t e = tid; e < mH; e += nt) atomicAdd(&start[colour(cur[e])], 1);
        __syncthreads();
        for (int32_t i = tid; i < P; i += nt) cursor[i] = start[i];      // real counts
        for (int32_t i = tid; i <= P; i += nt) start[i] = i < P ? (start[i] + 3) & ~3 : 0;
        __syncthreads();
        const int32_t mHp = block_scan_smem(start, P + 1, red);          // start[P] = padded total
        for (int32_t i = tid; i < P; i += nt) cursor[i] = start[i];
        __syncthreads();
        for (int32_t e = tid; e < mH; e += nt) {
            const uint32_t p = cur[e];
            const int32_t pos = atomicAdd(&cursor[colour(p)], 1);
            nxt[pos] = p;
            cs[pos] = 0.5f;          // Algorithm 1: f_e(u) = f_e(v) = w_e / 2
        }
        __syncthreads();
        for (int32_t c = tid; c < P; c += nt)
            for (int32_t i = cursor[c]; i < start[c + 1]; ++i) { nxt[i] = sentinel; cs[i] = 0.0f; }
        __syncthreads();             // the counters below reuse `cursor`
        // initial loads: degree in the core / 2; slot nH is the padding edges' node
        int32_t* dH = cursor;  // reuse (P + 1 >= nH)
        for (int32_t i = tid; i < nH; i += nt) dH[i] = 0;
        __syncthreads();
        for (int32_t e = tid; e < mHp; e += nt) {
            const uint32_t p = nxt[e];
            if (p == sentinel) continue;
            if ((int32_t)(p & 0xffffu) >= nH || (int32_t)(p >> 16) >= nH) { s_bad = 1; continue; }
            atomicAdd(&dH[p & 0xffffu], 1);
            atomicAdd(&dH[p >> 16], 1);
        }
        __syncthreads();
        for (int32_t i = tid; i <= nH; i += nt) L[i] = i < nH ? 0.5f * (float)dH[i] : 0.0f;
        __syncthreads();
        // ---------------- Algorithm 1 passes
        // Staged form: chunks of G consecutive classes move global -> shared through
        // cp.async.bulk (last warp), consumers update them in shared memory with a named
        // barrier per class, splits go back by bulk stores.  Used when at least 3 stages of
        // the longest chunk fit and a pass has enough chunks for the store ordering;
        // otherwise classes are updated straight from global memory.
        const size_t used = (((4u * (size_t)(nH + 1) + 4u * (size_t)(P + 1)) + 7) & ~(size_t)7);
        const size_t stage_base = ((used + 16u * kBMaxStages) + 127) & ~(size_t)127;
        if (tid < 32) {
            // the largest chunk size G leaving room for 3 stages, then as many stages as fit
            // and the store ordering allows (chunks per pass >= S - slack + groups + 1)
            int32_t pick_g = 0, pick_s = 0, pick_len = 0;
            for (int32_t g2 = 16; g2 >= 1 && mHp > 0 && nt >= 96; g2 >>= 1) {
                int32_t mx = 0;
                for (int32_t c0 = (int32_t)lane_id() * g2; c0 < P; c0 += 32 * g2)
                    mx = max(mx, start[min(c0 + g2, P)] - start[c0]);
                mx = __reduce_max_sync(0xffffffffu, mx);
                const size_t arr = max((size_t)128, ((4u * (size_t)mx) + 127) & ~(size_t)127);
                const int32_t fit = (int32_t)(stage_base < A.smem_bytes ? (A.smem_bytes - stage_base) / (2 * arr) : 0);
                const int32_t NC = (P + g2 - 1) / g2;
                const int32_t sS = min(min(fit, kBMaxStages), NC - (kBStoreGroups + 1 - kBStoreSlack));
                if (sS >= 3) {
                    pick_g = g2; pick_s = sS; pick_len = mx;
                    break;
                }
            }
            if (tid == 0) { s_count = pick_g; s_rem = pick_s; s_stage_len = pick_len; }
        }
        fence_proxy_async_all();   // the class-major edges and splits are read by bulk copies
        __syncthreads();
        const int32_t G = s_count, S = s_rem, chunk_len = s_stage_len;
        if (G > 0 && A.passes > 0) {
            const size_t arr = max((size_t)128, ((4u * (size_t)chunk_len) + 127) & ~(size_t)127);
            uint64_t* full = reinterpret_cast<uint64_t*>(sm + used);
            uint64_t* empty = full + S;
            unsigned char* stages = sm + stage_base;
            const int nc = nt - 32;
            if (tid == 0) {
                s_abort = 0;
                for (int k = 0; k < S; ++k) { mbar_init(&full[k], 1); mbar_init(&empty[k], 1); }
                fence_mbar_init();
                fence_proxy_async_smem();
            }
            __syncthreads();
            const int32_t NC = (P + G - 1) / G;
            const int32_t PT = NC * A.passes;     // chunks over all passes
            const int32_t ahead = S - kBStoreSlack;
            if (tid >= nc) {
                if (tid == nc) {
                    int32_t pf = 0, kf = 0, jf = 0;
                    auto fill = [&]() {
                        const int32_t beg = start[jf * G];
                        const uint32_t bytes = 4u * (uint32_t)(start[min(jf * G + G, P)] - beg);
                        unsigned char* st = stages + 2 * arr * (size_t)kf;
                        mbar_expect_tx(&full[kf], 2u * bytes);
                        bulk_g2s(st, nxt + beg, bytes, &full[kf]);
                        bulk_g2s(st + arr, cs + beg, bytes, &full[kf]);
                        ++pf;
                        kf = (kf + 1 == S) ? 0 : kf + 1;
                        jf = (jf + 1 == NC) ? 0 : jf + 1;
                    };
                    while (pf < ahead && pf < PT) fill();
                    int32_t k = 0, j = 0;
                    uint32_t parity = 0;
                    int32_t q = 0;
                    for (; q < PT; ++q) {
                        uint32_t spins = 0;
                        bool ok = mbar_try_wait_sleep(&empty[k], parity, 1000);
                        while (!ok && !s_abort && ++spins < kBWaitLimit) ok = mbar_try_wait_sleep(&empty[k], parity, 1000);
                        if (!ok) { s_abort = 1; break; }
                        const int32_t beg = start[j * G];
                        bulk_s2g(cs + beg, stages + 2 * arr * (size_t)k + arr,
                                 4u * (uint32_t)(start[min(j * G + G, P)] - beg));
                        bulk_commit();
                        if (pf < PT) {
                            bulk_wait<kBStoreGroups>();
                            bulk_wait_read<kBStoreSlack>();
                            fill();
                        }
                        if (++k == S) { k = 0; parity ^= 1u; }
                        j = (j + 1 == NC) ? 0 : j + 1;
                    }
                    // fills [q, pf) were never handed back: on abort wait (bounded) for them
                    if (q < PT) drain_fills(full, S, q, pf, kBWaitLimit);
                    bulk_wait<0>();
                }
            } else {
                auto wait_full = [&](int32_t kk, uint32_t par) -> bool {
                    uint32_t spins = 0;
                    bool ok = mbar_try_wait(&full[kk], par);
                    while (!ok && ++spins < kBWaitLimit) ok = mbar_try_wait(&full[kk], par);
                    return ok;
                };
                bool bad = false;
                if (tid < 32 && PT > 0) bad = !wait_full(0, 0);
                bad = consumer_sync_or(nc, bad);
                int32_t k = 0, j = 0;
                uint32_t parity = 0;
                for (int32_t q = 0; q < PT && !bad; ++q) {
                    const int32_t c0 = j * G;
                    const int32_t c1 = min(c0 + G, P);
                    const int32_t base = start[c0];
                    unsigned char* st = stages + 2 * arr * (size_t)k;
                    const uint32_t* suv = reinterpret_cast<const uint32_t*>(st);
                    float* ss = reinterpret_cast<float*>(st + arr);
                    int32_t cb = 0;
                    for (int32_t c = c0; c < c1; ++c) {
                        const int32_t ce = start[c + 1] - base;
                        for (int32_t r = cb + tid; r < ce; r += nc) {
                            const uint32_t p = suv[r];
                            const int32_t a = (int32_t)(p & 0xffffu), b = (int32_t)(p >> 16);
                            if (a > nH || b > nH) { s_bad = 1; continue; }   // never taken: ids checked
                            const float la = L[a], lb = L[b], sv = ss[r];
                            const float diff = la - lb;
                            const bool gt = diff > 0.0f;
                            const float cap = gt ? sv : (1.0f - sv);
                            const float d = fminf(fabsf(diff) * 0.5f, cap);
                            const float dd = gt ? d : -d;
                            L[a] = la - dd;
                            L[b] = lb + dd;
                            ss[r] = fminf(sv - dd, 1.0f);
                        }
                        cb = ce;
                        if (c + 1 < c1) consumer_sync(nc);
                    }
                    fence_proxy_async_smem();
                    const int32_t kprev = k;
                    if (++k == S) { k = 0; parity ^= 1u; }
                    j = (j + 1 == NC) ? 0 : j + 1;
                    bool fail = false;
                    if (tid < 32 && q + 1 < PT) fail = !wait_full(k, parity);
                    bad = consumer_sync_or(nc, fail);
                    if (tid == 0) mbar_arrive(&empty[kprev]);
                }
                if (bad && tid == 0) s_abort = 1;
            }
            __syncthreads();
            if (tid == 0)   // the barriers' memory is reused by the extraction and the next graph
                for (int32_t k = 0; k < S; ++k) { mbar_inval(&full[k]); mbar_inval(&empty[k]); }
            __syncthreads();
        } else {
            for (int32_t t = 0; t < A.passes; ++t) {
                for (int32_t c = 0; c < P; ++c) {
                    const int32_t beg = start[c], end = start[c + 1];
                    for (int32_t i = beg + tid; i < end; i += nt) {
                        const uint32_t p = __ldcg(nxt + i);
                        const int32_t a = (int32_t)(p & 0xffffu), b = (int32_t)(p >> 16);
                        if (a > nH || b > nH) { s_bad = 1; continue; }   // never taken: ids checked
                        float la = L[a], lb = L[b], s = __ldcg(cs + i);
                        const float diff = la - lb;
                        const bool gt = diff > 0.0f;
                        const float cap = gt ? s : (1.0f - s);
                        const float d = fminf(fabsf(diff) * 0.5f, cap);
                        const float dd = gt ? d : -d;
                        L[a] = la - dd;
                        L[b] = lb + dd;
                        __stcg(cs + i, fminf(s - dd, 1.0f));
                    }
                    if (end > beg) __syncthreads();
                }
            }
        }
        for (int32_t i = tid; i < nH; i += nt) {
            lout[oldid[i]] = L[i];
            cout[oldid[i]] = 1;
        }
        // ---------------- extraction
        unsigned long long* keys = reinterpret_cast<unsigned long long*>(cursor + P + 1);  // [npow]
        keys = reinterpret_cast<unsigned long long*>(((uintptr_t)keys + 7) & ~(uintptr_t)7);
        int32_t* pos = reinterpret_cast<int32_t*>(keys + npow);                            // [nH]
        int32_t* bucket = pos + nH;                                                        // [nH]
        for (int32_t i = tid; i < npow; i += nt) {
            unsigned long long kk = ~0ull;
            if (i < nH) {
                const uint32_t bits = __float_as_uint(L[i] + 0.0f);
                const uint32_t ord = (bits & 0x80000000u) ? ~bits : (bits | 0x80000000u);
                kk = ((unsigned long long)(~ord) << 32) | (unsigned long long)(0xffffffffu - (uint32_t)i);
            }
            keys[i] = kk;
        }
        __syncthreads();
        for (int32_t size = 2; size <= npow; size <<= 1)
            for (int32_t stride = size >> 1; stride > 0; stride >>= 1) {
                for (int32_t i = tid; i < npow; i += nt) {
                    const int32_t j = i ^ stride;
                    if (j > i) {
                        const bool up = (i & size) == 0;
                        const unsigned long long x = keys[i], y = keys[j];
                        if ((x > y) == up) { keys[i] = y; keys[j] = x; }
                    }
                }
                __syncthreads();
            }
        for (int32_t i = tid; i < nH; i += nt) {
            pos[0xffffffffu - (uint32_t)(keys[i] & 0xffffffffu)] = i;
            bucket[i] = 0;
        }
        __syncthreads();
        for (int32_t e = tid; e < mHp; e += nt) {
            const uint32_t p = nxt[e];
            if (p == sentinel) continue;
            if ((int32_t)(p & 0xffffu) >= nH || (int32_t)(p >> 16) >= nH) { s_bad = 1; continue; }
            atomicAdd(&bucket[max(pos[p & 0xffffu], pos[p >> 16])], 1);
        }
        __syncthreads();
        block_scan_smem(bucket, nH, red);  // exclusive; W(S_k) = bucket[k-1] + count in k-1
        // inclusive prefix weight of the top k+1 nodes: excl[k+1] (or mH for the last)
        int64_t bw = -1, bk = 0;
        for (int32_t i = tid; i < nH; i += nt) {
            const int64_t Wk = (i + 1 < nH) ? bucket[i + 1] : mH;
            const int64_t kk = i + 1;
            if (bw < 0 || Wk * bk > bw * kk || (Wk * bk == bw * kk && kk > bk)) { bw = Wk; bk = kk; }
        }
        // block arg-max with the exact comparator
        __shared__ long long s_w[32], s_k[32];
        for (int o = 16; o > 0; o >>= 1) {
            const long long ow = __shfl_xor_sync(0xffffffffu, (long long)bw, o);
            const long long ok = __shfl_xor_sync(0xffffffffu, (long long)bk, o);
            if (ow >= 0 && (bw < 0 || ow * bk > bw * ok || (ow * bk == bw * ok && ok > bk))) { bw = ow; bk = ok; }
        }
        if (lane_id() == 0) { s_w[warp_id()] = bw; s_k[warp_id()] = bk; }
        __syncthreads();
        if (tid == 0) {
            long long W2 = -1, k2 = 0;
            for (int w = 0; w < (nt >> 5); ++w) {
                const long long ow = s_w[w], ok = s_k[w];
                if (ow >= 0 && (W2 < 0 || ow * k2 > W2 * ok || (ow * k2 == W2 * ok && ok > k2))) { W2 = ow; k2 = ok; }
            }
            if (nH == 0) { W2 = 0; k2 = 0; }
            s_rem = (int32_t)k2;
            A.rho[g] = k2 > 0 ? (double)W2 / (double)k2 : 0.0;
            A.S_size[g] = (int32_t)k2;
            A.nH[g] = nH; A.mH[g] = mH; A.rounds[g] = r; A.status[g] = s_bad ? BS_BAD_INPUT : (s_abort ? BS_WAIT_EXPIRED : BS_OK);
        }
        __syncthreads();
        const int32_t kstar = s_rem;
        for (int32_t i = tid; i < nH; i += nt)
            if (pos[i] < kstar) inS[oldid[i]] = 1;
        __syncthreads();
    }
}

// Input check: local ids in range, u < v, strictly increasing (u, v) inside each graph.
__global__ void k_batch_check(const int64_t* __restrict__ node_off, const int64_t* __restrict__ edge_off,
                              int32_t B, const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                              int64_t m, int32_t* __restrict__ err) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = B;   // graph g with edge_off[g] <= e < edge_off[g+1]
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (edge_off[mid] <= e) lo = mid; else hi = mid;
        }
        const int64_t n = node_off[lo + 1] - node_off[lo];
        const int32_t a = u[e], b = v[e];
        bool ok = a >= 0 && a < b && b < n;
        if (ok && e > edge_off[lo]) {
            const int32_t pa = u[e - 1], pb = v[e - 1];
            ok = pa < a || (pa == a && pb < b);
        }
        if (!ok) atomicOr(err, 1);
    }
}

}  // namespace

struct lowd_batch_ctx {
    cudaStream_t st = nullptr;
    bool own_stream = false;   // created here when the caller passed NULL (capture needs a real stream)
    int mem = LOWD_MEM_HOST;
    int32_t B = 0;
    int64_t n_total = 0, m_total = 0;
    int64_t *node_off = nullptr, *edge_off = nullptr;
    std::vector<int64_t> h_node_off, h_edge_off;
    int32_t *u = nullptr, *v = nullptr;
    uint32_t *eA = nullptr, *eB = nullptr;
    float* cs = nullptr;
    int32_t* oldid = nullptr;
    int32_t* order = nullptr;
    int32_t* queue = nullptr;
    double* rho = nullptr;
    int32_t *S_size = nullptr, *nH = nullptr, *mH = nullptr, *rounds = nullptr, *status = nullptr;
    uint8_t* in_S = nullptr;
    float* loads = nullptr;
    uint8_t* in_core = nullptr;
    // tuned launch
    lowd_batch_options tuned{};
    int have_tuned = 0;
    // captured launch
    cudaGraphExec_t gexec = nullptr;
    lowd_batch_options gopt{};
    char err[256] = {0};

    lowd_status fail(cudaError_t e) {
        snprintf(err, sizeof(err), "%s", cudaGetErrorString(e));
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LOWD_ERR_OUT_OF_MEMORY : LOWD_ERR_CUDA;
    }
};

namespace {

template <class T>
cudaError_t balloc(T** p, size_t count) {
    *p = nullptr;
    return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

void batch_free_all(lowd_batch_ctx* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    if (b->own_stream && b->st) cudaStreamDestroy(b->st);
    b->st = nullptr;
    void* ps[] = {b->node_off, b->edge_off, b->u, b->v, b->eA, b->eB, b->cs, b->oldid, b->order, b->queue,
                  b->rho, b->S_size, b->nH, b->mH, b->rounds, b->status, b->in_S, b->loads, b->in_core};
    for (void* p : ps)
        if (p) cudaFree(p);
}

// graphs ordered by edge count, largest first, or as given
void set_order(lowd_batch_ctx* b, int32_t mode, const std::vector<int32_t>* subset) {
    std::vector<int32_t> ord;
    if (subset) ord = *subset;
    else { ord.resize(b->B); for (int32_t i = 0; i < b->B; ++i) ord[i] = i; }
    if (mode == LOWD_BATCH_ORDER_LARGEST_FIRST)
        std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) {
            return (b->h_edge_off[x + 1] - b->h_edge_off[x]) > (b->h_edge_off[y + 1] - b->h_edge_off[y]);
        });
    cudaMemcpyAsync(b->order, ord.data(), sizeof(int32_t) * ord.size(), cudaMemcpyHostToDevice, b->st);
    cudaStreamSynchronize(b->st);
}

lowd_batch_options resolve(const lowd_batch_ctx* b, const lowd_batch_options* opt) {
    lowd_batch_options o{};
    if (opt) o = *opt;
    if (b->have_tuned) {
        if (o.ctas_per_sm <= 0) o.ctas_per_sm = b->tuned.ctas_per_sm;
        if (o.threads <= 0) o.threads = b->tuned.threads;
        if (o.order <= 0) o.order = b->tuned.order;
    }
    if (o.ctas_per_sm <= 0) o.ctas_per_sm = 1;
    if (o.threads <= 0) o.threads = kBT;
    if (o.order <= 0) o.order = LOWD_BATCH_ORDER_LARGEST_FIRST;
    if (o.passes < 0) o.passes = 0;
    return o;
}

struct LaunchCfg {
    int grid = 1, threads = kBT, smem = 0;
};

// Shared-memory size and grid for a launch; sets the kernel attribute (outside any capture).
cudaError_t prepare(const lowd_batch_options& o, int32_t count, LaunchCfg* cfg) {
    int dev = 0, sms = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int per = o.ctas_per_sm;
    int smem = (optin - 2048) / per - 1024;
    smem &= ~1023;
    e = cudaFuncSetAttribute(k_batch_lowd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    cfg->smem = smem;
    cfg->threads = o.threads;
    cfg->grid = sms * per;
    if (cfg->grid > count) cfg->grid = count > 0 ? count : 1;
    return cudaSuccess;
}

// Queue reset + persistent kernel on the batch's stream (capturable).
cudaError_t enqueue(lowd_batch_ctx* b, const lowd_batch_options& o, int32_t count, const LaunchCfg& cfg) {
    BatchArgs A;
    A.B = count;
    A.node_off = b->node_off; A.edge_off = b->edge_off; A.u = b->u; A.v = b->v;
    A.eA = b->eA; A.eB = b->eB; A.cs = b->cs; A.oldid = b->oldid; A.order = b->order; A.queue = b->queue;
    A.passes = o.passes; A.smem_bytes = (uint32_t)cfg.smem;
    A.rho = b->rho; A.S_size = b->S_size; A.nH = b->nH; A.mH = b->mH; A.rounds = b->rounds;
    A.status = b->status; A.in_S = b->in_S; A.loads = b->loads; A.in_core = b->in_core;
    cudaError_t e = cudaMemsetAsync(b->queue, 0, sizeof(int32_t), b->st);
    if (e != cudaSuccess) return e;
    LOWD_LAUNCH(k_batch_lowd, cfg.grid, cfg.threads, cfg.smem, b->st, A);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

lowd_status lowd_batch_create(int32_t B, const int64_t* node_off, const int64_t* edge_off, const int32_t* u,
                              const int32_t* v, int32_t mem, void* stream, lowd_batch* out) {
    if (!out) return LOWD_ERR_INVALID_ARG;
    *out = nullptr;
    if (B < 1 || !node_off || !edge_off || (mem != LOWD_MEM_HOST && mem != LOWD_MEM_DEVICE))
        return LOWD_ERR_INVALID_ARG;
    lowd_batch_ctx* b = new (std::nothrow) lowd_batch_ctx();
    if (!b) return LOWD_ERR_OUT_OF_MEMORY;
    b->st = (cudaStream_t)stream;
    if (!b->st) {
        if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return LOWD_ERR_CUDA;
        }
        b->own_stream = true;
    }
    b->mem = mem;
    b->B = B;
    b->h_node_off.resize((size_t)B + 1);
    b->h_edge_off.resize((size_t)B + 1);
    const cudaMemcpyKind in = mem == LOWD_MEM_DEVICE ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    cudaError_t e = cudaMemcpy(b->h_node_off.data(), node_off, sizeof(int64_t) * ((size_t)B + 1), in);
    if (e == cudaSuccess) e = cudaMemcpy(b->h_edge_off.data(), edge_off, sizeof(int64_t) * ((size_t)B + 1), in);
    lowd_status s = LOWD_OK;
    if (e != cudaSuccess) s = b->fail(e);
    if (s == LOWD_OK) {
        bool ok = b->h_node_off[0] == 0 && b->h_edge_off[0] == 0;
        for (int32_t g = 0; ok && g < B; ++g)
            ok = b->h_node_off[g + 1] > b->h_node_off[g] && b->h_edge_off[g + 1] >= b->h_edge_off[g];
        if (!ok) s = LOWD_ERR_INVALID_ARG;
    }
    if (s == LOWD_OK) {
        b->n_total = b->h_node_off[B];
        b->m_total = b->h_edge_off[B];
        if (b->m_total > 0 && (!u || !v)) s = LOWD_ERR_INVALID_ARG;
        if (b->m_total >= ((int64_t)1 << 40)) s = LOWD_ERR_TOO_LARGE;
    }
    const size_t m = (size_t)b->m_total, n = (size_t)b->n_total;
    if (s == LOWD_OK) {
        cudaError_t a = cudaSuccess;
        if (a == cudaSuccess) a = balloc(&b->node_off, (size_t)B + 1);
        if (a == cudaSuccess) a = balloc(&b->edge_off, (size_t)B + 1);
        if (a == cudaSuccess) a = balloc(&b->u, m);
        if (a == cudaSuccess) a = balloc(&b->v, m);
        // per graph: its edges plus up to 3 padding edges per colour class, 16-byte aligned
        const size_t mp = m + 4 * n + 16;
        if (a == cudaSuccess) a = balloc(&b->eA, mp);
        if (a == cudaSuccess) a = balloc(&b->eB, mp);
        if (a == cudaSuccess) a = balloc(&b->cs, mp);
        if (a == cudaSuccess) a = balloc(&b->oldid, n);
        if (a == cudaSuccess) a = balloc(&b->order, (size_t)B);
        if (a == cudaSuccess) a = balloc(&b->queue, 16);
        if (a == cudaSuccess) a = balloc(&b->rho, (size_t)B);
        if (a == cudaSuccess) a = balloc(&b->S_size, (size_t)B);
        if (a == cudaSuccess) a = balloc(&b->nH, (size_t)B);
        if (a == cudaSuccess) a = balloc(&b->mH, (size_t)B);
        if (a == cudaSuccess) a = balloc(&b->rounds, (size_t)B);
        if (a == cudaSuccess) a = balloc(&b->status, (size_t)B);
        if (a == cudaSuccess) a = balloc(&b->in_S, n);
        if (a == cudaSuccess) a = balloc(&b->loads, n);
        if (a == cudaSuccess) a = balloc(&b->in_core, n);
        if (a != cudaSuccess) s = b->fail(a);
    }
    if (s == LOWD_OK) {
        const cudaMemcpyKind k = mem == LOWD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        cudaMemcpyAsync(b->node_off, b->h_node_off.data(), sizeof(int64_t) * ((size_t)B + 1), cudaMemcpyHostToDevice, b->st);
        cudaMemcpyAsync(b->edge_off, b->h_edge_off.data(), sizeof(int64_t) * ((size_t)B + 1), cudaMemcpyHostToDevice, b->st);
        if (m > 0) {
            cudaMemcpyAsync(b->u, u, sizeof(int32_t) * m, k, b->st);
            cudaMemcpyAsync(b->v, v, sizeof(int32_t) * m, k, b->st);
        }
        cudaMemsetAsync(b->queue, 0, 16 * sizeof(int32_t), b->st);
        if (m > 0) {
            LOWD_LAUNCH(k_batch_check, lowd_grid_for((int64_t)m, 256), 256, 0, b->st, b->node_off, b->edge_off, B, b->u, b->v,
                        (int64_t)m, b->queue + 8);
        }
        int32_t bad = 0;
        e = cudaMemcpyAsync(&bad, b->queue + 8, sizeof(int32_t), cudaMemcpyDeviceToHost, b->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
        if (e != cudaSuccess) s = b->fail(e);
        else if (bad) {
            snprintf(b->err, sizeof(b->err), "edges must be u < v, in range, strictly increasing per graph");
            s = LOWD_ERR_INVALID_ARG;
        }
    }
    if (s != LOWD_OK) {
        batch_free_all(b);
        delete b;
        return s;
    }
    *out = b;
    return LOWD_OK;
}

lowd_status lowd_batch_run(lowd_batch b, const lowd_batch_options* opt) {
    if (!b) return LOWD_ERR_INVALID_ARG;
    const lowd_batch_options o = resolve(b, opt);
    if (o.threads % 32 != 0 || o.threads < 64 || o.threads > 1024 || o.ctas_per_sm < 1 || o.ctas_per_sm > 4)
        return LOWD_ERR_INVALID_ARG;
    const bool same = b->gexec && b->gopt.passes == o.passes && b->gopt.ctas_per_sm == o.ctas_per_sm &&
                      b->gopt.threads == o.threads && b->gopt.order == o.order;
    cudaError_t e = cudaSuccess;
    if (!same) {
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
        set_order(b, o.order, nullptr);
        LaunchCfg cfg;
        e = prepare(o, b->B, &cfg);
        if (e != cudaSuccess) {
            lowd_status st = b->fail(e);
            snprintf(b->err, sizeof(b->err), "prepare: %s", cudaGetErrorString(e));
            return st;
        }
        // capture the launch (queue reset + persistent kernel) once, replay it afterwards
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = enqueue(b, o, b->B, cfg);
            e = cudaStreamEndCapture(b->st, &graph);
            if (e == cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            lowd_status st = b->fail(e);
            snprintf(b->err, sizeof(b->err), "capture: %s", cudaGetErrorString(e));
            return st;
        }
        b->gopt = o;
    }
    e = cudaGraphLaunch(b->gexec, b->st);
    lowd_note_launch();   // the replayed graph holds one kernel
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return b->fail(e);
    return LOWD_OK;
}

lowd_status lowd_batch_autotune(lowd_batch b, int32_t passes, int32_t sample, lowd_batch_options* best) {
    if (!b || passes < 0) return LOWD_ERR_INVALID_ARG;
    if (sample <= 0 || sample > b->B) sample = b->B;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);   // the order array is rewritten below
    b->gexec = nullptr;
    // a spread sample of the graphs
    std::vector<int32_t> sub;
    for (int32_t i = 0; i < sample; ++i) sub.push_back((int32_t)((int64_t)i * b->B / sample));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = -1.0f;
    lowd_batch_options bo{};
    const int thr[] = {256, 512, 1024};
    for (int order = LOWD_BATCH_ORDER_AS_GIVEN; order <= LOWD_BATCH_ORDER_LARGEST_FIRST; ++order) {
        set_order(b, order, &sub);
        for (int per = 1; per <= 2; ++per)
            for (int t : thr) {
                lowd_batch_options o{};
                o.passes = passes; o.ctas_per_sm = per; o.threads = t; o.order = order;
                if (t * per > 2048) continue;
                LaunchCfg cfg;
                cudaError_t e = prepare(o, sample, &cfg);
                if (e != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return b->fail(e); }
                cudaEventRecord(e0, b->st);
                e = enqueue(b, o, sample, cfg);
                cudaEventRecord(e1, b->st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) {
                    cudaEventDestroy(e0); cudaEventDestroy(e1);
                    return b->fail(e);
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (best_ms < 0.0f || ms < best_ms) { best_ms = ms; bo = o; }
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tuned = bo;
    b->have_tuned = 1;
    if (best) *best = bo;
    return LOWD_OK;
}

lowd_status lowd_batch_results(lowd_batch b, double* rho, int32_t* S_size, uint8_t* in_S, int32_t* n_core,
                               int32_t* m_core, int32_t* rounds, int32_t* status) {
    if (!b) return LOWD_ERR_INVALID_ARG;
    const cudaMemcpyKind k = b->mem == LOWD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t B = (size_t)b->B;
    cudaError_t e = cudaSuccess;
    if (rho && e == cudaSuccess) e = cudaMemcpyAsync(rho, b->rho, sizeof(double) * B, k, b->st);
    if (S_size && e == cudaSuccess) e = cudaMemcpyAsync(S_size, b->S_size, sizeof(int32_t) * B, k, b->st);
    if (in_S && e == cudaSuccess) e = cudaMemcpyAsync(in_S, b->in_S, (size_t)b->n_total, k, b->st);
    if (n_core && e == cudaSuccess) e = cudaMemcpyAsync(n_core, b->nH, sizeof(int32_t) * B, k, b->st);
    if (m_core && e == cudaSuccess) e = cudaMemcpyAsync(m_core, b->mH, sizeof(int32_t) * B, k, b->st);
    if (rounds && e == cudaSuccess) e = cudaMemcpyAsync(rounds, b->rounds, sizeof(int32_t) * B, k, b->st);
    if (status && e == cudaSuccess) e = cudaMemcpyAsync(status, b->status, sizeof(int32_t) * B, k, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return b->fail(e);
    return LOWD_OK;
}

lowd_status lowd_batch_loads(lowd_batch b, float* loads) {
    if (!b || !loads) return LOWD_ERR_INVALID_ARG;
    const cudaMemcpyKind k = b->mem == LOWD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaMemcpyAsync(loads, b->loads, sizeof(float) * (size_t)b->n_total, k, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return b->fail(e);
    return LOWD_OK;
}

lowd_status lowd_batch_core(lowd_batch b, uint8_t* in_core) {
    if (!b || !in_core) return LOWD_ERR_INVALID_ARG;
    const cudaMemcpyKind k = b->mem == LOWD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaMemcpyAsync(in_core, b->in_core, (size_t)b->n_total, k, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return b->fail(e);
    return LOWD_OK;
}

const char* lowd_batch_last_error(lowd_batch b) { return b ? b->err : ""; }

void lowd_batch_free(lowd_batch b) {
    if (!b) return;
    cudaStreamSynchronize(b->st);
    batch_free_all(b);
    delete b;
}

}  // extern "C"
