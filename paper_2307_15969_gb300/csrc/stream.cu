// The streamed LOWD pass (schedule 2): graphs of any size, node loads in global memory.
//
// Schedule.  Algorithm 1 may visit the edges in any fixed order (Fig. 1 caption).  This
// schedule visits them by ascending key (max(d_a, d_b), min(d_a, d_b), fmix32(e)), d the
// unweighted degree: light edges first, high-degree nodes' edges last, ties scrambled by
// MurmurHash3's 32-bit finaliser (a bijection) so that equal-degree chains do not serialise.
// Two edges with no common endpoint commute, so the pass only has to keep the key order at
// each node: edge e can run once the previous edge (in key order) at each of its two ends
// has run.  Its level, 1 + the larger level of those two predecessors, is its colour: every
// class is a matching, a pass visits the classes in ascending colour, and there are at least
// max d classes (exactly max d on the R-MAT graphs, whose tail is the top hub's star).  The
// levels are computed on the GPU by Kahn's algorithm, one frontier per level.
//
// Execution.  One CTA runs the classes in order; the loads of all n nodes stay in global
// memory (L2) as FP32 pairs (hi, lo) moved by error-free transfers, as in the shared-memory
// sweep.  The class-major edge stream is cut into chunks (at most kSegs classes or class
// pieces and at most Emax edges); producer warps stage each chunk in a ring of S shared-
// memory stages: the ends, splits, weights and two 32-bit read descriptors by bulk copies,
// and the two end loads of every edge by 8-byte cp.async gathers, D chunks ahead.  A load
// gathered D chunks ahead is stale if its node was updated in between, so the descriptor of
// each end, computed once per schedule from the previous occurrence of its node, says where
// the current value is: its own gathered slot, or the slot of that previous occurrence (in
// the same chunk or one of the D - 1 before, still resident because S >= 2D).  Consumer warps
// read both loads through the descriptors, update, write the new loads into their own slots
// and meet at a named barrier per class; the producers write each released chunk's loads
// back to global memory (skipped where the next occurrence reads the slot directly) and its
// splits back with a bulk store.  Every wait is bounded; on expiry the kernel raises an
// error flag and all warps leave together.
#include "ctx.cuh"
#include "prims.cuh"
#include "async.cuh"

#include <algorithm>
#include <vector>

using namespace lowd;

namespace {

constexpr int kT = 256;
inline unsigned grid_for(int64_t n) { return lowd_grid_for(n, kT); }

// ------------------------------------------------------------------ level colouring

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {   // MurmurHash3 32-bit finaliser
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__global__ void k_count_degrees(const int32_t* __restrict__ u, const int32_t* __restrict__ v, int64_t m,
                                int32_t* __restrict__ deg) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        atomicAdd(&deg[u[e]], 1);
        atomicAdd(&deg[v[e]], 1);
    }
}

__global__ void k_tie_keys(int64_t m, uint32_t* __restrict__ key, int32_t* __restrict__ val) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        key[e] = fmix32((uint32_t)e);
        val[e] = (int32_t)e;
    }
}

// degree key (max << 32 | min) of the edge at each position of the tie-sorted order
__global__ void k_degree_keys(const int32_t* __restrict__ ord, int64_t m, const int32_t* __restrict__ u,
                              const int32_t* __restrict__ v, const int32_t* __restrict__ deg,
                              uint64_t* __restrict__ key) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = ord[i];
        const uint64_t a = (uint64_t)deg[u[e]], b = (uint64_t)deg[v[e]];
        key[i] = ((a > b ? a : b) << 32) | (a > b ? b : a);
    }
}

// two adjacency entries per edge, in rank (key) order: (end node, rank)
__global__ void k_adj_entries(const int32_t* __restrict__ ord, int64_t m, const int32_t* __restrict__ u,
                              const int32_t* __restrict__ v, uint32_t* __restrict__ node,
                              int32_t* __restrict__ rk) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = ord[k];
        node[2 * k] = (uint32_t)u[e];
        node[2 * k + 1] = (uint32_t)v[e];
        rk[2 * k] = (int32_t)k;
        rk[2 * k + 1] = (int32_t)k;
    }
}

// Entries sorted by node (stable, so by rank inside a node).  For entry j of node x holding
// rank k: the successor of k at x is the next entry's rank; k has a predecessor at x unless
// j is x's first entry.  side: 0 for the edge's u end, 1 for its v end.
__global__ void k_successors(const uint32_t* __restrict__ node, const int32_t* __restrict__ rk, int64_t N,
                             const int32_t* __restrict__ ord, const int32_t* __restrict__ u,
                             int32_t* __restrict__ succ, uint8_t* __restrict__ has_pred) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = node[j];
        const int32_t k = rk[j];
        const int side = (u[ord[k]] == (int32_t)x) ? 0 : 1;
        succ[2 * (int64_t)k + side] = (j + 1 < N && node[j + 1] == x) ? rk[j + 1] : -1;
        has_pred[2 * (int64_t)k + side] = (j > 0 && node[j - 1] == x) ? 1 : 0;
    }
}

// pending predecessors per rank; ranks with none form the first frontier
__global__ void k_pending(const uint8_t* __restrict__ has_pred, int64_t m, int32_t* __restrict__ pend,
                          int32_t* __restrict__ frontier, int32_t* __restrict__ fcount) {
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = base + threadIdx.x;
        int p = 1;
        if (k < m) {
            p = has_pred[2 * k] + has_pred[2 * k + 1];
            pend[k] = p;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, k < m && p == 0);
        int32_t slot = 0;
        if (lane_id() == 0 && bal) slot = atomicAdd(fcount, __popc(bal));
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (k < m && p == 0) frontier[slot + __popc(bal & ((1u << lane_id()) - 1u))] = (int32_t)k;
    }
}

constexpr uint32_t kSpinLimit = 1u << 22;    // bounded waits: mbarrier try_wait rounds

// Kahn's algorithm by levels.  ctl: [0..2] frontier sizes (rotating), [4] barrier count,
// [5] barrier generation, [6] level count out.  Frontier r lives in fr[r & 1].  While the
// frontier holds at least `small` ranks every block works on it and blocks meet at a grid
// barrier per level; below that, block 0 goes on alone with block barriers.
__global__ void k_levels(int32_t* __restrict__ pend, const int32_t* __restrict__ succ, int32_t* __restrict__ level,
                         int32_t* __restrict__ f0, int32_t* __restrict__ f1, int32_t* __restrict__ ctl,
                         int32_t small, int32_t* __restrict__ err) {
    int32_t* fr[2] = {f0, f1};
    volatile int32_t* vctl = ctl;
    bool alone = false;
    for (int32_t r = 0;; ++r) {
        const int32_t ncur = vctl[r % 3];
        if (ncur == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl[6] = r;
            return;
        }
        if (!alone && ncur < small) {
            if (blockIdx.x != 0) return;
            alone = true;
        }
        const int32_t* cur = fr[r & 1];
        int32_t* nxt = fr[(r + 1) & 1];
        if (threadIdx.x == 0 && blockIdx.x == 0) ctl[(r + 2) % 3] = 0;   // the frontier after next
        const int64_t stride = alone ? (int64_t)blockDim.x : (int64_t)gridDim.x * blockDim.x;
        const int64_t t0 = alone ? (int64_t)threadIdx.x : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        for (int64_t i = t0; i < ncur; i += stride) {
            const int32_t k = cur[i];
            level[k] = r;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int32_t t = succ[2 * (int64_t)k + s];
                if (t >= 0 && atomicSub(&pend[t], 1) == 1) nxt[atomicAdd(&ctl[(r + 1) % 3], 1)] = t;
            }
        }
        if (alone) {
            __threadfence_block();
            __syncthreads();
        } else if (!grid_barrier((unsigned*)&ctl[4], (volatile unsigned*)&ctl[5], gridDim.x, err)) {
            return;
        }
    }
}

// level of every rank; the class-major order is the edges sorted by level, ranks ascending
__global__ void k_level_keys(const int32_t* __restrict__ level, const int32_t* __restrict__ ord, int64_t m,
                             uint32_t* __restrict__ key, int32_t* __restrict__ val) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        key[k] = (uint32_t)level[k];
        val[k] = ord[k];
    }
}

__global__ void k_level_heads(const uint32_t* __restrict__ key, int64_t m, int32_t* __restrict__ coff) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        if (i == 0 || key[i] != key[i - 1]) coff[key[i]] = (int32_t)i;
}

__global__ void k_map_ids(const int32_t* __restrict__ ids, int64_t k, int32_t* __restrict__ x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = ids[x[i]];
}

// ------------------------------------------------------------------ chunked stream

// read descriptor of one end: bits 0..19 shared-memory offset of the load to read, bit 20:
// the offset points into the previous pass (read the own gathered slot in a launch's first
// pass), bits 21..22: when the producer writes this slot back
constexpr uint32_t kOffMask = 0xFFFFFu;
constexpr uint32_t kWrap = 1u << 20;
constexpr int kWbShift = 21;
enum { WB_ALWAYS = 0, WB_NEVER = 1, WB_LAST_PASS = 2 };
constexpr uint32_t kZeroSlot = 0;   // ring offset of an always-zero load (padding ends)
constexpr uint32_t kRingHead = 128; // stages start here

constexpr int kSegs = 64;           // classes (or class pieces) per chunk
constexpr int kHdrInts = 68;        // chunk header: begin, padded size, segment count, 64 ends, pad
constexpr int kSmallSeg = 32;       // segments this small are updated by one warp
constexpr int kConsumers = 512;
constexpr int kProducerWarps = 2;
constexpr int kStoreGroups = 8;
constexpr int kLead = 3;            // D: chunks gathered ahead of the consumers; S = 2D stages

// A stage: the chunk's blob (header, then ends a and b, read descriptors a and b and, if
// weighted, weights, each an array of the chunk's padded size), then the splits and the two
// gathered-or-updated load slots per edge at fixed offsets (read descriptors point there).
struct StreamLayout {
    uint32_t E;          // edges per stage (multiple of 4)
    uint32_t blob, s, la, lb, bytes;   // offsets inside a stage
};

__host__ __device__ inline uint32_t blob_words(uint32_t Ej, bool weighted) {
    return (uint32_t)kHdrInts + (weighted ? 5u : 4u) * Ej;
}

__host__ __device__ inline StreamLayout stream_layout(uint32_t E, bool weighted) {
    StreamLayout L;
    L.E = E;
    L.blob = 0;
    L.s = (4u * blob_words(E, weighted) + 127u) & ~127u;
    L.la = (L.s + 4u * E + 15u) & ~15u;
    L.lb = L.la + 8u * E;
    L.bytes = ((L.lb + 8u * E) + 127u) & ~127u;
    return L;
}

// views into a stage whose blob has landed (Ej = the chunk's padded size)
struct StageView {
    const int32_t* hdr;
    const int32_t* ea;
    const int32_t* eb;
    const uint32_t* sa;
    const uint32_t* sb;
    const float* w;
    uint32_t cnt;
};

__device__ __forceinline__ StageView stage_view(const unsigned char* st, uint32_t E) {
    StageView v;
    v.hdr = reinterpret_cast<const int32_t*>(st);
    v.cnt = min((uint32_t)v.hdr[1], E);
    v.ea = v.hdr + kHdrInts;
    v.eb = v.ea + v.cnt;
    v.sa = reinterpret_cast<const uint32_t*>(v.eb + v.cnt);
    v.sb = v.sa + v.cnt;
    v.w = reinterpret_cast<const float*>(v.sb + v.cnt);
    return v;
}

// largest E (multiple of 4) whose S stages fit the shared-memory budget
inline uint32_t stream_edges_per_stage(int S, bool weighted, size_t budget) {
    uint32_t E = (uint32_t)(budget / (size_t)S / (weighted ? 40u : 36u)) & ~3u;   // 16 B loads + 20/24 B
    while (E > 4 && (size_t)stream_layout(E, weighted).bytes * (size_t)S > budget) E -= 4;
    return E;
}

// chunk holding position p: the largest J with beg[J] <= p (empty chunks only at the end)
__device__ __host__ inline int32_t chunk_of(const int32_t* beg, int32_t NC, int64_t p) {
    int32_t lo = 0, hi = NC - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)beg[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// class-major real position i -> padded position; perm_pad and the streams
__global__ void k_pad_scatter(const int32_t* __restrict__ order, int64_t m, int64_t m_grid,
                              const int32_t* __restrict__ real_beg, const int32_t* __restrict__ pad_beg,
                              int32_t NC, int32_t* __restrict__ perm_pad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < m_grid) {   // grid-wide classes keep their positions
            perm_pad[i] = order[i];
            continue;
        }
        const int32_t J = chunk_of(real_beg, NC, i);
        perm_pad[pad_beg[J] + (i - real_beg[J])] = order[i];
    }
}

__global__ void k_fill_i32s(int32_t* __restrict__ x, int64_t n, int32_t val) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = val;
}

__global__ void k_stream_gather(const int32_t* __restrict__ perm_pad, int64_t m_pad, int32_t n,
                                const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                                const float* __restrict__ w, const float* __restrict__ s_init,
                                int32_t* __restrict__ ea, int32_t* __restrict__ eb, float* __restrict__ cw,
                                float* __restrict__ cs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = perm_pad[i];
        if (e < 0) {
            ea[i] = n; eb[i] = n;
            if (cw) cw[i] = 0.0f;
            cs[i] = 0.0f;
            continue;
        }
        ea[i] = u[e]; eb[i] = v[e];
        const float we = w ? w[e] : 1.0f;
        if (cw) cw[i] = we;
        cs[i] = s_init ? fminf(fmaxf(s_init[e], 0.0f), we) : we * 0.5f;   // Alg. 1: w_e / 2
    }
}

// occurrence records (node, 2p + side) of the chunked positions p >= p0, in position order;
// padding and the grid-wide part sort last (key n)
__global__ void k_occurrences(const int32_t* __restrict__ perm_pad, const int32_t* __restrict__ ea,
                              const int32_t* __restrict__ eb, int64_t m_pad, int64_t p0, int32_t n,
                              uint32_t* __restrict__ key, int64_t* __restrict__ val) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m_pad;
         p += (int64_t)gridDim.x * blockDim.x) {
        const bool pad = perm_pad[p] < 0 || p < p0;
        key[2 * p] = pad ? (uint32_t)n : (uint32_t)ea[p];
        key[2 * p + 1] = pad ? (uint32_t)n : (uint32_t)eb[p];
        val[2 * p] = 2 * p;
        val[2 * p + 1] = 2 * p + 1;
    }
}

__global__ void k_group_bounds(const uint32_t* __restrict__ key, int64_t N, uint32_t n, int64_t* __restrict__ first,
                               int64_t* __restrict__ last) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = key[j];
        if (x >= n) continue;
        if (j == 0 || key[j - 1] != x) first[x] = j;
        if (j + 1 == N || key[j + 1] != x) last[x] = j;
    }
}

__device__ __forceinline__ uint32_t slot_offset(const int32_t* beg, int32_t NC, int32_t S, const StreamLayout& L,
                                                int64_t code) {
    const int64_t p = code >> 1;
    const int32_t J = chunk_of(beg, NC, p);
    return kRingHead + (uint32_t)(J % S) * L.bytes + ((code & 1) ? L.lb : L.la) + 8u * (uint32_t)(p - beg[J]);
}

// Read descriptor and write-back rule of every end (see the header comment).
__global__ void k_descriptors(const uint32_t* __restrict__ key, const int64_t* __restrict__ val, int64_t N,
                              uint32_t n, const int64_t* __restrict__ first, const int64_t* __restrict__ last,
                              const int32_t* __restrict__ beg, int32_t NC, int32_t S, int32_t D, StreamLayout L,
                              uint32_t* __restrict__ srcA, uint32_t* __restrict__ srcB) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t code = val[j];
        const int64_t p = code >> 1;
        uint32_t word;
        const uint32_t x = key[j];
        if (x >= n) {
            word = kZeroSlot | ((uint32_t)WB_NEVER << kWbShift);
        } else {
            const int32_t J = chunk_of(beg, NC, p);
            const int64_t fx = first[x], lx = last[x];
            // previous occurrence (cyclic)
            const bool pwrap = j == fx;
            const int64_t pj = pwrap ? lx : j - 1;
            const int32_t Jp = chunk_of(beg, NC, val[pj] >> 1);
            const int32_t dp = pwrap ? J - Jp + NC : J - Jp;
            word = dp < D ? (slot_offset(beg, NC, S, L, val[pj]) | (pwrap ? kWrap : 0u))
                          : slot_offset(beg, NC, S, L, code);
            // next occurrence (cyclic): does it read this slot directly?
            const bool nwrap = j == lx;
            const int64_t nj = nwrap ? fx : j + 1;
            const int32_t Jn = chunk_of(beg, NC, val[nj] >> 1);
            const int32_t dn = nwrap ? Jn - J + NC : Jn - J;
            const uint32_t wb = dn < D ? (nwrap ? WB_LAST_PASS : WB_NEVER) : WB_ALWAYS;
            word |= wb << kWbShift;
        }
        if (code & 1) srcB[p] = word; else srcA[p] = word;
    }
}

// chunk blobs: header row, then ends a, ends b, read descriptors a, b (and weights) of the
// chunk's padded positions
__global__ void k_blob_headers(const int32_t* __restrict__ ctab, const int64_t* __restrict__ blob_off, int32_t NC,
                               uint32_t* __restrict__ blob) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)NC * kHdrInts;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t J = i / kHdrInts, k = i % kHdrInts;
        blob[blob_off[J] + k] = (uint32_t)ctab[i];
    }
}

__global__ void k_blob_data(const int32_t* __restrict__ beg, const int64_t* __restrict__ blob_off, int32_t NC,
                            int64_t p0, int64_t m_pad, const int32_t* __restrict__ ea, const int32_t* __restrict__ eb,
                            const uint32_t* __restrict__ srcA, const uint32_t* __restrict__ srcB,
                            const float* __restrict__ cw, uint32_t* __restrict__ blob) {
    for (int64_t p = p0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m_pad;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t J = chunk_of(beg, NC, p);
        const int64_t Ej = beg[J + 1] - beg[J];
        const int64_t i = p - beg[J];
        uint32_t* d = blob + blob_off[J] + kHdrInts;
        d[i] = (uint32_t)ea[p];
        d[Ej + i] = (uint32_t)eb[p];
        d[2 * Ej + i] = srcA[p];
        d[3 * Ej + i] = srcB[p];
        if (cw) d[4 * Ej + i] = __float_as_uint(cw[p]);
    }
}

__global__ void k_pack_loads(const float* __restrict__ l, const float* __restrict__ l_lo, int32_t n,
                             float2* __restrict__ lp) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
         i += (int64_t)gridDim.x * blockDim.x)
        lp[i] = i < n ? make_float2(l[i], l_lo[i]) : make_float2(0.0f, 0.0f);
}

// loads back as (l = fl(hi + lo), l_lo = exact remainder)
__global__ void k_unpack_loads(const float2* __restrict__ lp, int32_t n, float* __restrict__ l,
                               float* __restrict__ l_lo) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 x = lp[i];
        const float s = x.x + x.y;
        l[i] = s;
        l_lo[i] = x.y - (s - x.x);
    }
}

// FP64 loads from the splits (streamed layout)
__global__ void k_rederive_ab(int64_t m_pad, const int32_t* __restrict__ ea, const int32_t* __restrict__ eb,
                              const float* __restrict__ cw, const float* __restrict__ cs, int32_t n,
                              double* __restrict__ L64) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = ea[i], b = eb[i];
        if (a >= n) continue;
        const double s = (double)cs[i];
        const double w = cw ? (double)cw[i] : 1.0;
        atomicAdd(&L64[a], s);
        atomicAdd(&L64[b], w - s);
    }
}

// ------------------------------------------------------------------ the pass kernel

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
    s = a + b;
    const float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void comp_add(float2& x, float v) {
    float t, e;
    two_sum(x.x, v, t, e);
    x.x = t;
    x.y += e;
}

// Algorithm 1's edge update on pair loads; returns the new f_e(a)
__device__ __forceinline__ float comp_transfer(float2& A, float2& B, float s, float w) {
    const float diff = (A.x - B.x) + (A.y - B.y);
    const bool gt = diff > 0.0f;
    const float cap = gt ? s : (w - s);
    const float d = fminf(fabsf(diff) * 0.5f, cap);
    const float dd = gt ? d : -d;
    comp_add(A, -dd);
    comp_add(B, dd);
    return fminf(s - dd, w);
}

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// barrier over the producer warps only
__device__ __forceinline__ void producer_sync() {
    asm volatile("bar.sync 2, %0;" ::"r"(kProducerWarps * 32) : "memory");
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(kConsumers + kProducerWarps * 32, 1)
k_sweep_stream(int32_t n, int32_t NC, const int64_t* __restrict__ blob_off, const int32_t* __restrict__ beg,
               const uint32_t* __restrict__ blob, float* __restrict__ cs, float2* __restrict__ lp,
               int32_t passes, int32_t S, int32_t D, uint32_t E, uint32_t smem_bytes, int32_t* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char ring[];
    __shared__ __align__(8) uint64_t mfull[16];   // stage's blob and splits landed (bulk copies)
    __shared__ __align__(8) uint64_t gfull[16];   // stage's gathered loads landed (cp.async)
    __shared__ __align__(8) uint64_t empty[16];   // stage released by the consumers
    __shared__ volatile int32_t abort_flag;
    const StreamLayout L = stream_layout(E, WEIGHTED);
    const int tid = threadIdx.x;
    const int nc = kConsumers;
    const int NP = kProducerWarps * 32;
    const int32_t P = NC * passes;   // the launcher keeps this < 2^31
    if (tid == 0) {
        abort_flag = 0;
        for (int k = 0; k < S; ++k) {
            mbar_init(&mfull[k], 1);
            mbar_init(&gfull[k], NP);   // one cp.async arrival per producer thread
            mbar_init(&empty[k], 1);
        }
        *reinterpret_cast<float2*>(ring + kZeroSlot) = make_float2(0.0f, 0.0f);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    auto stage = [&](int32_t q) -> unsigned char* { return ring + kRingHead + (uint32_t)(q % S) * L.bytes; };
    if (tid >= nc) {
        // ---------------- producers
        const int pt = tid - nc;
        struct Range { int64_t o0, o1; int32_t b0, b1; };
        // chunk q's blob and splits, by two bulk copies (one thread)
        auto meta = [&](int32_t q, const Range& r) {
            if (pt != 0) return;
            unsigned char* st = stage(q);
            uint64_t* bar = &mfull[q % S];
            const uint32_t bb = 4u * (uint32_t)(r.o1 - r.o0);
            const uint32_t sb = 4u * (uint32_t)(r.b1 - r.b0);
            mbar_expect_tx(bar, bb + sb);
            bulk_g2s(st + L.blob, blob + r.o0, bb, bar);
            if (sb) bulk_g2s(st + L.s, cs + r.b0, sb, bar);
        };
        // gathers of the loads chunk q's descriptors ask for (its blob already landed)
        auto gather = [&](int32_t q) {
            unsigned char* st = stage(q);
            const bool first = q < NC;
            const StageView v = stage_view(st, E);
            const uint32_t own0 = (uint32_t)(st - ring);
            for (uint32_t i = pt; i < v.cnt; i += NP) {
                const uint32_t wa = v.sa[i], wb = v.sb[i];
                const uint32_t oa = own0 + L.la + 8u * i, ob = own0 + L.lb + 8u * i;
                const int32_t a = v.ea[i], b = v.eb[i];
                if (((wa & kOffMask) == oa || (first && (wa & kWrap))) && (uint32_t)a < (uint32_t)n)
                    cp_async8(ring + oa, lp + a);
                if (((wb & kOffMask) == ob || (first && (wb & kWrap))) && (uint32_t)b < (uint32_t)n)
                    cp_async8(ring + ob, lp + b);
            }
            cp_async_arrive_noinc(&gfull[q % S]);
        };
        // released chunk q: loads back to global memory, splits by a bulk store
        auto writeback = [&](int32_t q) {
            unsigned char* st = stage(q);
            const StageView v = stage_view(st, E);
            const int32_t b0 = v.hdr[0];
            const bool lastp = q >= P - NC;
            const float2* la = reinterpret_cast<const float2*>(st + L.la);
            const float2* lb = reinterpret_cast<const float2*>(st + L.lb);
            for (uint32_t i = pt; i < v.cnt; i += NP) {
                const uint32_t ca = v.sa[i] >> kWbShift, cb = v.sb[i] >> kWbShift;
                const int32_t a = v.ea[i], b = v.eb[i];
                if ((ca == WB_ALWAYS || (ca == WB_LAST_PASS && lastp)) && (uint32_t)a < (uint32_t)n) lp[a] = la[i];
                if ((cb == WB_ALWAYS || (cb == WB_LAST_PASS && lastp)) && (uint32_t)b < (uint32_t)n) lp[b] = lb[i];
            }
            if (pt == 0 && v.cnt) {
                bulk_s2g(cs + b0, st + L.s, 4u * v.cnt);
                bulk_commit();
            }
        };
        auto wait_bar = [&](uint64_t* bar, uint32_t par) -> bool {   // producer thread 0 only
            uint32_t spins = 0;
            bool ok = mbar_try_wait(bar, par);
            while (!ok && !abort_flag && ++spins < kSpinLimit) ok = mbar_try_wait(bar, par);
            return ok;
        };
        // chunk ranges, read one step ahead of their copy
        auto range = [&](int32_t q) -> Range {
            const int32_t J = q % NC;
            Range r;
            r.o0 = __ldg(blob_off + J);
            r.o1 = __ldg(blob_off + J + 1);
            r.b0 = __ldg(beg + J);
            r.b1 = __ldg(beg + J + 1);
            return r;
        };
        // copies run D + 2 chunks ahead of the consumers, gathers D chunks ahead
        int32_t mf = 0, gf = 0;
        Range nr{};
        if (P > 0) nr = range(0);
        while (mf < D + 2 && mf < P) {
            meta(mf, nr);
            if (++mf < P) nr = range(mf);
        }
        bool ok = true;
        while (gf < D && gf < P && ok) {
            if (pt == 0) ok = wait_bar(&mfull[gf % S], (uint32_t)((gf / S) & 1));
            if (pt == 0 && !ok) abort_flag = 1;
            producer_sync();
            if (abort_flag) break;
            gather(gf++);
        }
        int32_t q = 0;
        for (; q < P && !abort_flag; ++q) {
            const int32_t k = q % S;
            if (pt == 0 && !wait_bar(&empty[k], (uint32_t)((q / S) & 1))) abort_flag = 1;
            producer_sync();
            if (abort_flag) break;
            writeback(q);
            if (mf < P) {
                // the stage of chunk mf held chunk mf - S = q - 1 (released, written back):
                // its split store (committed one iteration ago) must have finished reading it,
                // and every store older than the last kStoreGroups must be complete (a
                // chunk's splits are read again a pass later)
                if (pt == 0) {
                    bulk_wait<kStoreGroups>();
                    bulk_wait_read<1>();
                }
                fence_proxy_async_smem();   // generic reads of the stage before async writes
                producer_sync();
                meta(mf, nr);
                if (++mf < P) nr = range(mf);
            }
            if (gf < P) {
                bool okg = true;
                if (pt == 0) okg = wait_bar(&mfull[gf % S], (uint32_t)((gf / S) & 1));
                if (pt == 0 && !okg) abort_flag = 1;
                producer_sync();
                if (abort_flag) break;
                gather(gf++);
            }
        }
        // on abort: wait (bounded) for copies that may still land in the ring
        cp_async_wait_all();
        if (pt == 0) {
            for (int32_t i = q; i < mf; ++i) {
                uint32_t spins = 0;
                while (!mbar_try_wait(&mfull[i % S], (uint32_t)((i / S) & 1)) && ++spins < kSpinLimit) {
                }
            }
            bulk_wait<0>();
            if (abort_flag) atomicOr(err, 1);
        }
        return;
    }
    // ---------------- consumers
    auto wait2 = [&](int32_t qq) -> bool {
        const int32_t kk = qq % S;
        const uint32_t par = (uint32_t)((qq / S) & 1);
        uint32_t spins = 0;
        bool ok = mbar_try_wait(&mfull[kk], par);
        while (!ok && ++spins < kSpinLimit) ok = mbar_try_wait(&mfull[kk], par);
        if (!ok) return false;
        ok = mbar_try_wait(&gfull[kk], par);
        while (!ok && ++spins < kSpinLimit) ok = mbar_try_wait(&gfull[kk], par);
        return ok;
    };
    const uint32_t lim = smem_bytes - 8u;   // largest valid 8-byte slot offset
    bool bad = false;
    if (tid < 32 && P > 0) bad = !wait2(0);
    bad = consumer_sync_or(nc, bad);
    bool oob = false;
    for (int32_t q = 0; q < P && !bad; ++q) {
        const int32_t k = q % S;
        const bool first = q < NC;
        unsigned char* st = stage(q);
        const uint32_t own0 = (uint32_t)(st - ring);
        const StageView v = stage_view(st, E);
        float* ss = reinterpret_cast<float*>(st + L.s);
        float2* la = reinterpret_cast<float2*>(st + L.la);
        float2* lb = reinterpret_cast<float2*>(st + L.lb);
        const int32_t nseg = min(v.hdr[2], kSegs);
        const int32_t cmax = (int32_t)v.cnt;
        int32_t cb = 0;
        int32_t ce = nseg > 0 ? min(v.hdr[3], cmax) : 0;
        for (int32_t g = 0; g < nseg; ++g) {
            // a small segment is updated by warp 0 alone; consecutive small segments are
            // separated by a warp barrier, any other pair by the consumer barrier
            const bool small = ce - cb <= kSmallSeg;
            const int32_t cn = g + 1 < nseg ? min(v.hdr[4 + g], cmax) : ce;
            const bool next_small = cn - ce <= kSmallSeg;
            for (int32_t r = cb + tid; r < ce && (!small || tid < 32); r += nc) {
                const uint32_t wa = v.sa[r], wb = v.sb[r];
                uint32_t oa = (first && (wa & kWrap)) ? own0 + L.la + 8u * r : (wa & kOffMask);
                uint32_t ob = (first && (wb & kWrap)) ? own0 + L.lb + 8u * r : (wb & kOffMask);
                if (oa > lim || ob > lim) { oob = true; oa = kZeroSlot; ob = kZeroSlot; }
                float2 A = *reinterpret_cast<const float2*>(ring + oa);
                float2 B = *reinterpret_cast<const float2*>(ring + ob);
                const float sv = ss[r];
                const float wv = WEIGHTED ? v.w[r] : 1.0f;
                const float ns = comp_transfer(A, B, sv, wv);
                la[r] = A;
                lb[r] = B;
                ss[r] = ns;
            }
            cb = ce;
            ce = cn;
            if (g + 1 < nseg) {
                if (small && next_small) {
                    if (tid < 32) __syncwarp();
                } else {
                    consumer_sync(nc);
                }
            }
        }
        fence_proxy_async_smem();   // the splits leave by a bulk store (async proxy)
        bool fail = false;
        if (tid < 32 && q + 1 < P) fail = !wait2(q + 1);
        bad = consumer_sync_or(nc, fail);
        if (tid == 0) mbar_arrive(&empty[k]);
    }
    if (oob) atomicOr(err, 4);
    if (bad && tid == 0) {
        abort_flag = 1;
        atomicOr(err, 1);
    }
}

// The leading classes of the level order are large (on R-MAT, light edges come first: the
// first few thousand classes hold most edges).  Each of them is one grid-wide step: every
// thread takes edges of the class, reads both loads from global memory (L2, bypassing L1),
// updates and writes them back; a grid barrier separates the classes.  The remaining classes
// (the long tail of small classes around the hubs) go through k_sweep_stream.
constexpr int kGridThreads = 1024;
// A grid-wide step costs about one grid barrier plus one memory round trip (~3 us) whatever
// the class size; the one-CTA stream moves about one tail edge per 17 ns (it is bound by the
// scattered 8-byte gathers and write-backs of a single SM).  Classes above ~3 us / 17 ns
// edges are cheaper as grid steps.
constexpr int32_t kGridMinClass = 192;    // classes at least this large take a grid-wide step

template <bool WEIGHTED>
__global__ void __launch_bounds__(kGridThreads)
k_sweep_grid(int32_t K, const int32_t* __restrict__ coff, const int32_t* __restrict__ ea,
             const int32_t* __restrict__ eb, const float* __restrict__ cw, float* __restrict__ cs,
             float2* __restrict__ lp, unsigned* __restrict__ bar, int32_t* __restrict__ err) {
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // the ends, split and weight of this thread's first edge of the next class are read before
    // the grid barrier (they do not depend on the loads), so a class costs one round trip
    int32_t b0 = K > 0 ? __ldg(coff) : 0;
    int32_t na = 0, nb = 0;
    float nsplit = 0.0f, nw = 1.0f;
    auto fetch = [&](int64_t i, int32_t end) {
        if (i < end) {
            na = __ldg(ea + i);
            nb = __ldg(eb + i);
            nsplit = __ldcg(cs + i);
            nw = WEIGHTED ? __ldg(cw + i) : 1.0f;
        }
    };
    if (K > 0) fetch(b0 + t0, __ldg(coff + 1));
    for (int32_t c = 0; c < K; ++c) {
        const int32_t b1 = __ldg(coff + c + 1);
        for (int64_t i = b0 + t0; i < b1; i += T) {
            int32_t a, b;
            float s, w;
            if (i == b0 + t0) {
                a = na; b = nb; s = nsplit; w = nw;
            } else {
                a = __ldg(ea + i); b = __ldg(eb + i); s = __ldcg(cs + i);
                w = WEIGHTED ? __ldg(cw + i) : 1.0f;
            }
            float2 A = __ldcg(lp + a), B = __ldcg(lp + b);
            const float ns = comp_transfer(A, B, s, w);
            __stcg(lp + a, A);
            __stcg(lp + b, B);
            __stcg(cs + i, ns);
        }
        b0 = b1;
        if (c + 1 < K) fetch(b0 + t0, __ldg(coff + c + 2));
        if (!grid_barrier(bar, bar + 1, gridDim.x, err)) return;
    }
}

}  // namespace

// ------------------------------------------------------------------ host side

// Level colouring, class-major order, chunk tables, streams and descriptors; then the
// initial splits (equal split or the given canonical-order splits) and the loads.
lowd_status lowd_stream_prepare(lowd_ctx* h, const float* init_splits_canon) {
    cudaStream_t st = h->st;
    const int32_t n = h->n;
    StarSplit sp;                       // hub stars: the level order covers the plain edges
    int64_t m = h->m;
    const int32_t* cu = h->u;
    const int32_t* cv = h->v;
    int32_t* deg = nullptr;
    uint32_t* k32[2] = {nullptr, nullptr};
    uint64_t* k64[2] = {nullptr, nullptr};
    int32_t* val[2] = {nullptr, nullptr};
    int32_t *succ = nullptr, *pend = nullptr, *level = nullptr, *fr[2] = {nullptr, nullptr}, *ctl = nullptr;
    uint8_t* has_pred = nullptr;
    uint32_t* okey[2] = {nullptr, nullptr};
    int64_t* oval[2] = {nullptr, nullptr};
    int64_t *gfirst = nullptr, *glast = nullptr;
    int32_t *rb = nullptr, *pb = nullptr;
    lowd_status s = LOWD_OK;
    auto cleanup = [&]() {
        sp.release(h);
        dfree(h, &deg); dfree(h, &k32[0]); dfree(h, &k32[1]); dfree(h, &k64[0]); dfree(h, &k64[1]); dfree(h, &val[0]);
        dfree(h, &val[1]); dfree(h, &succ); dfree(h, &pend); dfree(h, &level); dfree(h, &fr[0]); dfree(h, &fr[1]); dfree(h, &ctl);
        dfree(h, &has_pred); dfree(h, &okey[0]); dfree(h, &okey[1]); dfree(h, &oval[0]); dfree(h, &oval[1]);
        dfree(h, &gfirst); dfree(h, &glast); dfree(h, &rb); dfree(h, &pb);
    };
    const bool weighted = h->w != nullptr;
    do {
        if ((s = h->need_tmp(lowd_sort_tmp_bytes(2 * (h->m > n ? h->m : n) + 2)))) break;
        // ---- 0. hub stars: classify the edges, keep the plain ones for the level order
        if ((s = lowd_star_split(h, h->hub_tau, 2, &sp))) break;
        const int32_t* pid = sp.pid;
        const int64_t ms = sp.ms;
        if (pid) {
            m = sp.m_plain;
            cu = sp.gu;
            cv = sp.gv;
        }
        // ---- 1. key order: stable sort by tie hash, then by degree key
        if ((s = dalloc(h, &deg, n))) break;
        if ((s = dalloc(h, &val[0], 2 * m))) break;
        if ((s = dalloc(h, &val[1], 2 * m))) break;
        int32_t C = 0;
        int32_t* ord = nullptr;      // rank -> edge id
        int32_t* order = nullptr;    // class-major position -> edge id
        if (m > 0) {
            if ((s = dalloc(h, &k32[0], 2 * m))) break;
            if ((s = dalloc(h, &k32[1], 2 * m))) break;
            if ((s = dalloc(h, &k64[0], m))) break;
            if ((s = dalloc(h, &k64[1], m))) break;
            cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)n, st);
            LOWD_LAUNCH(k_count_degrees, grid_for(m), kT, 0, st, cu, cv, m, deg);
            LOWD_LAUNCH(k_tie_keys, grid_for(m), kT, 0, st, m, k32[0], val[0]);
            int c1 = radix_sort_pairs<uint32_t, int32_t>(k32[0], val[0], k32[1], val[1], m, 32, h->tmp, st);
            int32_t* vtie = val[c1];
            int32_t* vother = val[1 - c1];
            LOWD_LAUNCH(k_degree_keys, grid_for(m), kT, 0, st, vtie, m, cu, cv, deg, k64[0]);
            const int32_t dmax = lowd_max_degree(h);
            const int dbits = bit_length_u64((uint64_t)(dmax > 0 ? dmax : 1));
            int c2 = radix_sort_pairs<uint64_t, int32_t>(k64[0], vtie, k64[1], vother, m, 32 + dbits, h->tmp, st);
            ord = c2 ? vother : vtie;
            int32_t* spare = c2 ? vtie : vother;
            // ---- 2. adjacency in key order, successors, pending counts
            LOWD_LAUNCH(k_adj_entries, grid_for(m), kT, 0, st, ord, m, cu, cv, k32[0], spare);
            // sort the 2m entries by node; `spare` (2m) holds the ranks, ping-pong with k32[1]
            int32_t* rk2 = nullptr;
            if ((s = dalloc(h, &rk2, 2 * m))) break;
            const int nbits = bit_length_u64((uint64_t)(n > 1 ? n - 1 : 1));
            int c3 = radix_sort_pairs<uint32_t, int32_t>(k32[0], spare, k32[1], rk2, 2 * m, nbits, h->tmp, st);
            uint32_t* nodes = c3 ? k32[1] : k32[0];
            int32_t* rks = c3 ? rk2 : spare;
            if ((s = dalloc(h, &succ, 2 * m))) { dfree(h, &rk2); break; }
            if ((s = dalloc(h, &has_pred, 2 * m))) { dfree(h, &rk2); break; }
            LOWD_LAUNCH(k_successors, grid_for(2 * m), kT, 0, st, nodes, rks, 2 * m, ord, cu, succ, has_pred);
            dfree(h, &rk2);
            // ord must survive: copy it out of the ping-pong buffers
            int32_t* ord_keep = nullptr;
            if ((s = dalloc(h, &ord_keep, m))) break;
            cudaMemcpyAsync(ord_keep, ord, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToDevice, st);
            ord = ord_keep;
            dfree(h, &val[0]); dfree(h, &val[1]);
            val[0] = ord_keep;   // freed by cleanup
            if ((s = dalloc(h, &pend, m))) break;
            if ((s = dalloc(h, &level, m))) break;
            if ((s = dalloc(h, &fr[0], m))) break;
            if ((s = dalloc(h, &fr[1], m))) break;
            if ((s = dalloc(h, &ctl, 16))) break;
            cudaMemsetAsync(ctl, 0, 16 * sizeof(int32_t), st);
            LOWD_LAUNCH(k_pending, grid_for(m), kT, 0, st, has_pred, m, pend, fr[0], ctl);
            // ---- 3. levels (cooperative: every block must be resident for the grid barrier)
            int dev = 0, nb_per_sm = 0;
            cudaGetDevice(&dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_per_sm, k_levels, kT, 0);
            int nblocks = lowd_device_sms() * (nb_per_sm > 2 ? 2 : (nb_per_sm > 0 ? nb_per_sm : 1));
            int32_t small = 4096;
            int32_t* errp = h->d_i32 + 10;
            cudaMemsetAsync(errp, 0, sizeof(int32_t), st);
            void* args[] = {&pend, &succ, &level, &fr[0], &fr[1], &ctl, &small, &errp};
            cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_levels, dim3(nblocks), dim3(kT), args, 0, st);
            lowd_note_launch();
            if (e != cudaSuccess) { s = h->fail(e); break; }
            int32_t hc[8];
            if (cudaMemcpyAsync(hc, ctl, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpyAsync(hc + 7, errp, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
            if (hc[7] != 0) {
                snprintf(h->err, sizeof(h->err), "level colouring: a bounded grid barrier expired");
                s = LOWD_ERR_CUDA;
                break;
            }
            C = hc[6];
            // ---- 4. class-major order: sort by level (stable over rank order)
            LOWD_LAUNCH(k_level_keys, grid_for(m), kT, 0, st, level, ord, m, k32[0], fr[0]);
            const int lbits = bit_length_u64((uint64_t)(C > 1 ? C - 1 : 1));
            int c4 = radix_sort_pairs<uint32_t, int32_t>(k32[0], fr[0], k32[1], fr[1], m, lbits, h->tmp, st);
            order = c4 ? fr[1] : fr[0];
            if (pid) LOWD_LAUNCH(k_map_ids, grid_for(m), kT, 0, st, pid, m, order);   // subset -> edge ids
            if ((s = dalloc(h, &h->coff_real, (size_t)C + 1))) break;
            LOWD_LAUNCH(k_level_heads, grid_for(m), kT, 0, st, c4 ? k32[1] : k32[0], m, h->coff_real);
            LOWD_LAUNCH(k_fill_i32s, 1, 32, 0, st, h->coff_real + C, (int64_t)1, (int32_t)m);
        } else {
            if ((s = dalloc(h, &h->coff_real, 1))) break;
            cudaMemsetAsync(h->coff_real, 0, sizeof(int32_t), st);
        }
        h->C = C;
        // ---- 5. chunks (host): at most kSegs class pieces and E edges each
        std::vector<int32_t> coff((size_t)C + 1, 0);
        if (cudaMemcpyAsync(coff.data(), h->coff_real, sizeof(int32_t) * ((size_t)C + 1), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
        const int32_t D = kLead, S = 2 * kLead;
        const size_t budget = 227 * 1024 - kRingHead - 1024;
        const uint32_t E = stream_edges_per_stage(S, weighted, budget);
        // header rows: [0] padded begin, [1] padded size, [2] segments, [3 + g] end of segment
        // g relative to the begin; real_beg: the chunk's first real (unpadded) position
        // leading classes of at least kGridMinClass edges take grid-wide steps (positions
        // [0, coff[K]) of the stream, padded to a multiple of 4); the rest are chunked
        int32_t K = 0;
        while (K < C && coff[K + 1] - coff[K] >= kGridMinClass) ++K;
        const int64_t m_grid = coff[K];
        const int64_t grid_pad = (m_grid + 3) & ~(int64_t)3;
        std::vector<int32_t> ctab, real_beg;
        int64_t pad = grid_pad, real = m_grid;
        int32_t cnt = 0, nseg = 0;
        std::vector<int32_t> row(kHdrInts, 0);
        auto open = [&]() {
            std::fill(row.begin(), row.end(), 0);
            row[0] = (int32_t)pad;
            real_beg.push_back((int32_t)real);
            cnt = 0;
            nseg = 0;
        };
        auto close = [&]() {
            const int32_t padded = (cnt + 3) & ~3;
            row[1] = padded;
            row[2] = nseg;
            ctab.insert(ctab.end(), row.begin(), row.end());
            pad += padded;
        };
        open();
        for (int32_t c = K; c < C; ++c) {
            int32_t rem = coff[c + 1] - coff[c];
            while (rem > 0) {
                if (nseg == kSegs || cnt == (int32_t)E) { close(); open(); }
                const int32_t t = rem < (int32_t)E - cnt ? rem : (int32_t)E - cnt;
                cnt += t;
                rem -= t;
                real += t;
                row[3 + nseg] = cnt;
                ++nseg;
            }
        }
        close();
        // pad the chunk count: a multiple of S (a chunk keeps its stage across passes), and
        // enough chunks that a chunk's split store completes before the chunk is read again
        int32_t NC = (int32_t)real_beg.size();
        int32_t NCp = NC < D + kStoreGroups + 3 ? D + kStoreGroups + 3 : NC;
        NCp = (NCp + S - 1) / S * S;
        while ((int32_t)real_beg.size() < NCp) { open(); close(); }
        std::vector<int32_t> pad_beg;
        for (int32_t J = 0; J < NCp; ++J) pad_beg.push_back(ctab[(size_t)J * kHdrInts]);
        pad_beg.push_back((int32_t)pad);
        real_beg.push_back((int32_t)real);
        const int64_t m_pad_plain = pad;       // the star edges follow the plain positions
        const int64_t m_pad = pad + ms;
        h->m_pad = m_pad;
        h->s2_NC = NCp;
        h->s2_K = K;
        h->s2_tail = real > m_grid ? 1 : 0;
        h->s2_E = (int32_t)E;
        h->s2_S = S;
        h->s2_D = D;
        if ((s = dalloc(h, &h->s2_ctab, ctab.size()))) break;
        if ((s = dalloc(h, &h->s2_beg, (size_t)NCp + 1))) break;
        if ((s = dalloc(h, &rb, (size_t)NCp + 1))) break;
        cudaMemcpyAsync(h->s2_ctab, ctab.data(), sizeof(int32_t) * ctab.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(h->s2_beg, pad_beg.data(), sizeof(int32_t) * pad_beg.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(rb, real_beg.data(), sizeof(int32_t) * real_beg.size(), cudaMemcpyHostToDevice, st);
        // ---- 6. padded stream
        if ((s = dalloc(h, &h->s2_ea, m_pad))) break;
        if ((s = dalloc(h, &h->s2_eb, m_pad))) break;
        if ((s = dalloc(h, &h->s2_srcA, m_pad))) break;
        if ((s = dalloc(h, &h->s2_srcB, m_pad))) break;
        if (weighted && (s = dalloc(h, &h->cw, m_pad))) break;
        if ((s = dalloc(h, &h->cs, m_pad))) break;
        if ((s = dalloc(h, &h->l, (size_t)n + 1))) break;
        if ((s = dalloc(h, &h->l_lo, (size_t)n + 1))) break;
        if ((s = dalloc(h, &h->s2_lp, (size_t)n + 1))) break;
        // ---- 6b. star steps at positions [m_pad_plain, m_pad)
        if ((s = dalloc(h, &h->perm, m_pad))) break;
        if ((s = lowd_star_blocks(h, sp, m_pad_plain, C, m))) break;
        if (m_pad > 0) {
            if (m_pad_plain > 0) LOWD_LAUNCH(k_fill_i32s, grid_for(m_pad_plain), kT, 0, st, h->perm, m_pad_plain, -1);
            if (m > 0) LOWD_LAUNCH(k_pad_scatter, grid_for(m), kT, 0, st, order, m, m_grid, rb, h->s2_beg, NCp, h->perm);
            LOWD_LAUNCH(k_stream_gather, grid_for(m_pad), kT, 0, st, h->perm, m_pad, n, h->u, h->v, h->w,
                        init_splits_canon, h->s2_ea, h->s2_eb, h->cw, h->cs);
            // ---- 7. descriptors from each node's occurrences (sorted by node, stable in position)
            const int64_t mp = m_pad_plain;
            if ((s = h->need_tmp(lowd_sort_tmp_bytes(2 * mp + 2)))) break;
            if ((s = dalloc(h, &okey[0], 2 * mp))) break;
            if ((s = dalloc(h, &okey[1], 2 * mp))) break;
            if ((s = dalloc(h, &oval[0], 2 * mp))) break;
            if ((s = dalloc(h, &oval[1], 2 * mp))) break;
            if ((s = dalloc(h, &gfirst, n))) break;
            if ((s = dalloc(h, &glast, n))) break;
            if (mp > 0) {
                LOWD_LAUNCH(k_occurrences, grid_for(mp), kT, 0, st, h->perm, h->s2_ea, h->s2_eb, mp, grid_pad, n,
                            okey[0], oval[0]);
                const int nb1 = bit_length_u64((uint64_t)n);   // keys 0..n (n = padding)
                int c5 = radix_sort_pairs<uint32_t, int64_t>(okey[0], oval[0], okey[1], oval[1], 2 * mp, nb1, h->tmp, st);
                uint32_t* sk = okey[c5];
                int64_t* sv = oval[c5];
                LOWD_LAUNCH(k_group_bounds, grid_for(2 * mp), kT, 0, st, sk, 2 * mp, (uint32_t)n, gfirst, glast);
                const StreamLayout L = stream_layout(E, weighted);
                LOWD_LAUNCH(k_descriptors, grid_for(2 * mp), kT, 0, st, sk, sv, 2 * mp, (uint32_t)n, gfirst, glast,
                            h->s2_beg, NCp, S, D, L, h->s2_srcA, h->s2_srcB);
            }
        }
        // ---- 8. chunk blobs (what the pass kernel copies per chunk)
        {
            std::vector<int64_t> bo((size_t)NCp + 1, 0);
            for (int32_t J = 0; J < NCp; ++J)
                bo[(size_t)J + 1] = bo[(size_t)J] + blob_words((uint32_t)(pad_beg[(size_t)J + 1] - pad_beg[(size_t)J]), weighted);
            if ((s = dalloc(h, &h->s2_blobo, (size_t)NCp + 1))) break;
            if ((s = dalloc(h, &h->s2_blob, (size_t)bo[(size_t)NCp]))) break;
            cudaMemcpyAsync(h->s2_blobo, bo.data(), sizeof(int64_t) * bo.size(), cudaMemcpyHostToDevice, st);
            LOWD_LAUNCH(k_blob_headers, grid_for((int64_t)NCp * kHdrInts), kT, 0, st, h->s2_ctab, h->s2_blobo, NCp,
                        h->s2_blob);
            if (m_pad_plain > grid_pad)
                LOWD_LAUNCH(k_blob_data, grid_for(m_pad_plain - grid_pad), kT, 0, st, h->s2_beg, h->s2_blobo, NCp,
                            grid_pad, m_pad_plain, h->s2_ea, h->s2_eb, h->s2_srcA, h->s2_srcB, h->cw, h->s2_blob);
        }
        if (cudaGetLastError() != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { s = h->fail(e); break; }
        h->sched = 2;
        h->inited = 1;
        double st3[3];
        s = lowd_sweep_rederive(h, st3);
    } while (0);
    cleanup();
    return s;
}

lowd_status lowd_stream_rederive(lowd_ctx* h, double* L64) {
    if (h->m_pad > 0)
        LOWD_LAUNCH(k_rederive_ab, grid_for(h->m_pad), kT, 0, h->st, h->m_pad, h->s2_ea, h->s2_eb, h->cw, h->cs,
                    h->n, L64);
    LOWD_CK_LAUNCH();
    return LOWD_OK;
}

// `passes` streamed passes: loads packed into the pair array, the pass kernel, loads back.
cudaError_t lowd_stream_passes(lowd_ctx* h, int32_t passes) {
    const bool weighted = h->cw != nullptr;
    const StreamLayout L = stream_layout((uint32_t)h->s2_E, weighted);
    const size_t smem = kRingHead + (size_t)L.bytes * (size_t)h->s2_S;
    auto kern = weighted ? k_sweep_stream<true> : k_sweep_stream<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    h->sweep_kernel = 4;
    h->sweep_E = 0;
    LOWD_LAUNCH(k_pack_loads, grid_for((int64_t)h->n + 1), kT, 0, h->st, h->l, h->l_lo, h->n, h->s2_lp);
    auto stream_launch = [&](int32_t k) {
        LOWD_LAUNCH(kern, 1, kConsumers + kProducerWarps * 32, smem, h->st, h->n, h->s2_NC, h->s2_blobo, h->s2_beg,
                    h->s2_blob, h->cs, h->s2_lp, k, h->s2_S, h->s2_D, (uint32_t)h->s2_E, (uint32_t)smem,
                    h->d_i32 + 8);
        return cudaGetLastError();
    };
    cudaMemsetAsync(h->d_i32 + 12, 0, 2 * sizeof(int32_t), h->st);   // grid barrier words
    unsigned* bar = reinterpret_cast<unsigned*>(h->d_i32 + 12);
    int32_t* errp = h->d_i32 + 8;
    if (h->star_S > 0) {
        // per pass: the plain edges (grid steps, then the chunked tail), then the star steps
        auto gk = weighted ? k_sweep_grid<true> : k_sweep_grid<false>;
        int32_t K = h->s2_K;
        const int32_t* coff = h->coff_real;
        const int32_t* pea = h->s2_ea;
        const int32_t* peb = h->s2_eb;
        const float* pcw = h->cw;
        float* pcs = h->cs;
        float2* plp = h->s2_lp;
        void* args[] = {&K, &coff, &pea, &peb, &pcw, &pcs, &plp, &bar, &errp};
        for (int32_t t = 0; t < passes && e == cudaSuccess; ++t) {
            if (K > 0) {
                e = cudaLaunchCooperativeKernel((const void*)gk, dim3(lowd_device_sms()), dim3(kGridThreads), args, 0,
                                                h->st);
                lowd_note_launch();
            }
            if (e == cudaSuccess && h->s2_tail) e = stream_launch(1);
            if (e == cudaSuccess) e = lowd_star_pass(h);
        }
    } else if (h->s2_K == 0) {
        const int32_t per = (int32_t)(0x7fffffff / h->s2_NC);
        for (int32_t done = 0; done < passes && e == cudaSuccess;) {
            const int32_t k = passes - done < per ? passes - done : per;
            e = stream_launch(k);
            done += k;
        }
    } else {
        // per pass: the large classes as grid-wide steps, then the tail through the stream
        auto gk = weighted ? k_sweep_grid<true> : k_sweep_grid<false>;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gk, kGridThreads, 0);
        const int blocks = lowd_device_sms() * (per_sm > 0 ? 1 : 1);   // one block per SM
        int32_t K = h->s2_K;
        const int32_t* coff = h->coff_real;
        const int32_t* pea = h->s2_ea;
        const int32_t* peb = h->s2_eb;
        const float* pcw = h->cw;
        float* pcs = h->cs;
        float2* plp = h->s2_lp;
        void* args[] = {&K, &coff, &pea, &peb, &pcw, &pcs, &plp, &bar, &errp};
        for (int32_t t = 0; t < passes && e == cudaSuccess; ++t) {
            e = cudaLaunchCooperativeKernel((const void*)gk, dim3(blocks), dim3(kGridThreads), args, 0, h->st);
            lowd_note_launch();
            if (e == cudaSuccess && h->s2_tail) e = stream_launch(1);
        }
    }
    if (e != cudaSuccess) return e;
    LOWD_LAUNCH(k_unpack_loads, grid_for(h->n), kT, 0, h->st, h->s2_lp, h->n, h->l, h->l_lo);
    return cudaGetLastError();
}
