// Algorithm 1 on the GPU: conflict-free schedule, initialisation and the LOWD passes.
//
// Schedule.  A pass must be equivalent to visiting the edges one after another
// (Algorithm 1 updates each edge with the loads left by the previous one).  The edges
// are split into colour classes of a proper edge colouring; a class is a matching, so
// its updates touch disjoint node pairs and running them in parallel gives exactly the
// sequential result in any order inside the class.  Classes run in colour order with a
// barrier between them.  The colouring is the round-robin ("circle") tournament
// colouring of the complete graph on the current node set restricted to the actual
// edges: with N' = n rounded up to even and P = N' - 1,
//     colour(a, b) = (a + b) mod P           if b != N' - 1,
//     colour(a, N'-1) = 2a mod P,
// a proper colouring with P colours computed in O(1) per edge.  The pruned graphs this
// path serves are dense cores (maximum degree close to n), where P is within a few
// colours of the lower bound Delta.
//
// Execution.  One CTA keeps every node load in shared memory for all passes of a call, as
// an FP32 pair (hi, lo) updated by error-free transfers (TwoSum), so no update rounds a load.
// The class segments (packed 16-bit endpoint pairs when n <= 65536, the FP32 split and, if
// weighted, the FP32 weight) are staged global -> shared in chunks of consecutive classes by
// a producer warp with cp.async.bulk and mbarriers, and the updated splits go back by bulk
// stores; the consumer warps touch only shared memory and meet at a named barrier after each
// class (k_sweep_tma).  Graphs whose staged layout does not fit use a register-prefetch
// kernel with single FP32 loads (k_sweep_vec, k_sweep_simple).  The split of edge
// e = (lo, hi) is stored once, s_e = f_e(lo); f_e(hi) = w_e - s_e (the tighter dual's
// equality f_e(u) + f_e(v) = w_e, Sec. III-B).
#include "ctx.cuh"
#include "prims.cuh"
#include "async.cuh"

using namespace lowd;

namespace {

constexpr int kT = 256;

inline unsigned grid_for(int64_t n) { return lowd_grid_for(n, kT); }

// Colour of each edge (the circle colouring) and its place inside the class.  Inside a
// class every edge pairs a and b = c - a (mod P); with b < P the high end is fixed by the
// low one and the wrap group g = [a + b >= P], so edges of one group whose low ends are
// distinct mod 16 also have high ends distinct mod 16.  The staged sweep keeps a load as an
// 8-byte pair, and a warp's 8-byte shared-memory access is served half a warp at a time: 16
// lanes touching nodes distinct mod 16 use all 32 banks once.  The first key orders a class
// by (group, low end mod 16); the second deals the edges out in rounds of 16, so each half
// warp's edges mostly have distinct ends mod 16 at both ends.
constexpr int kRankBits = 16;  // rank inside a (class, group, bank) bucket: < 2^16
constexpr int kBankBits = 4;   // 16 load slots of 8 bytes span the 32 four-byte banks

__global__ void k_circle_colour(const int32_t* __restrict__ u, const int32_t* __restrict__ v, int64_t m,
                                int32_t n, uint64_t* __restrict__ key, int32_t* __restrict__ val) {
    const uint32_t Np = (uint32_t)(n + (n & 1));
    const uint32_t P = Np - 1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = (uint32_t)u[e], b = (uint32_t)v[e];
        const uint32_t c = (b == Np - 1) ? (2u * a) % P : (a + b) % P;
        const uint32_t g = (b != Np - 1 && a + b >= P) ? 1u : 0u;
        key[e] = ((uint64_t)c << (kBankBits + 1)) | ((uint64_t)g << kBankBits) |
                 (uint64_t)(a & ((1u << kBankBits) - 1u));
        val[e] = (int32_t)e;
    }
}

// Second key: (colour, group, rank inside its (colour, group, bank) bucket, bank).
__global__ void k_bank_rounds(const uint64_t* __restrict__ key, int64_t m, uint64_t* __restrict__ key2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = key[i];
        int64_t lo = 0, hi = i;  // first index with key == k
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (key[mid] < k) lo = mid + 1; else hi = mid;
        }
        const uint64_t r = (uint64_t)(i - lo);
        key2[i] = ((k >> kBankBits) << (kRankBits + kBankBits)) | (r << kBankBits) |
                  (k & ((1u << kBankBits) - 1u));
    }
}

__global__ void k_class_heads(const uint64_t* __restrict__ key, int64_t m, int shift, int32_t* __restrict__ head) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        head[i] = (i == 0 || (key[i] >> shift) != (key[i - 1] >> shift)) ? 1 : 0;
}

__global__ void k_class_offsets(const int32_t* __restrict__ head, const int32_t* __restrict__ hpos,
                                int64_t m, int32_t C, int32_t* __restrict__ coff) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        if (head[i]) coff[hpos[i]] = (int32_t)i;
    if (blockIdx.x == 0 && threadIdx.x == 0) coff[C] = (int32_t)m;
}

// Class segments padded to a multiple of 4 edges: pcnt[c] = roundup4(size of class c).
__global__ void k_pad_sizes(const int32_t* __restrict__ coff_real, int32_t C, int32_t* __restrict__ pcnt) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (int64_t)gridDim.x * blockDim.x)
        pcnt[c] = (coff_real[c + 1] - coff_real[c] + 3) & ~3;
}

// x[i] = ids[x[i]]: indices into a subset of the edges -> edge ids
__global__ void k_subset_to_ids(const int32_t* __restrict__ ids, int64_t k, int32_t* __restrict__ x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = ids[x[i]];
}

__global__ void k_fill_perm(int32_t* __restrict__ perm_pad, int64_t m_pad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad;
         i += (int64_t)gridDim.x * blockDim.x)
        perm_pad[i] = -1;
}

// Real position i (class-major, unpadded) -> padded position.
__global__ void k_scatter_padded(const int32_t* __restrict__ perm, const int32_t* __restrict__ head,
                                 const int32_t* __restrict__ hpos, const int32_t* __restrict__ coff_real,
                                 const int32_t* __restrict__ coff_pad, int64_t m,
                                 int32_t* __restrict__ perm_pad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = hpos[i] + head[i] - 1;
        perm_pad[coff_pad[c] + (i - coff_real[c])] = perm[i];
    }
}

// Class-major streams over the padded positions: packed ends, weights, initial splits;
// padding edges join the sentinel node n to itself with s = w = 0 (a no-op update).
__global__ void k_gather_streams(const int32_t* __restrict__ perm_pad, int64_t m_pad, int32_t n,
                                 const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                                 const float* __restrict__ w, const float* __restrict__ s_init,
                                 uint32_t* __restrict__ cuv, float* __restrict__ cw,
                                 float* __restrict__ cs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = perm_pad[i];
        if (e < 0) {
            cuv[i] = (uint32_t)n | ((uint32_t)n << 16);
            if (cw) cw[i] = 0.0f;
            cs[i] = 0.0f;
            continue;
        }
        cuv[i] = (uint32_t)u[e] | ((uint32_t)v[e] << 16);
        const float we = w ? w[e] : 1.0f;
        if (cw) cw[i] = we;
        cs[i] = s_init ? fminf(fmaxf(s_init[e], 0.0f), we) : we * 0.5f;  // Alg. 1: w_e / 2
    }
}

// FP64 loads from the splits: l_x = sum over edges at x of f_e(x) (padding skipped).
__global__ void k_rederive(int64_t m_pad, const uint32_t* __restrict__ cuv, const float* __restrict__ cw,
                           const float* __restrict__ cs, double* __restrict__ L64) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = cuv[i];
        const int32_t a = (int32_t)(p & 0xffffu), b = (int32_t)(p >> 16);
        if (a == b) continue;
        const double s = (double)cs[i];
        const double w = cw ? (double)cw[i] : 1.0;
        atomicAdd(&L64[a], s);
        atomicAdd(&L64[b], w - s);
    }
}

// (l, l_lo) = L64 as an FP32 pair; stats[0] += sum l, stats[1] += sum l^2, stats[2] = max l (FP64)
__global__ void k_load_stats(const double* __restrict__ L64, int32_t n, float* __restrict__ l,
                             float* __restrict__ l_lo, double* __restrict__ stats) {
    __shared__ double sh[kT / 32 + 1];
    double s1 = 0.0, s2 = 0.0, mx = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double x = L64[i];
        if (l) {
            const float hi = (float)x;
            l[i] = hi;
            l_lo[i] = (float)(x - (double)hi);   // the pair (hi, lo) carries x to ~2^-48
        }
        s1 += x; s2 += x * x; mx = fmax(mx, x);
    }
    double t1 = block_sum(s1, sh);
    double t2 = block_sum(s2, sh);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ double shm[kT / 32];
    if (lane_id() == 0) shm[warp_id()] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m2 = 0.0;
        for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) m2 = fmax(m2, shm[wv]);
        atomicAdd(&stats[0], t1);
        atomicAdd(&stats[1], t2);
        // loads are >= 0, so the bit pattern orders like the value
        atomicMax((unsigned long long*)&stats[2], (unsigned long long)__double_as_longlong(m2));
    }
}

__global__ void k_splits_from_canonical(const int32_t* __restrict__ perm_pad, int64_t m_pad,
                                        const float* __restrict__ in, float* __restrict__ cs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = perm_pad[i];
        if (e >= 0) cs[i] = in[e];
    }
}

__global__ void k_splits_to_canonical(const int32_t* __restrict__ perm_pad, int64_t m_pad,
                                      const float* __restrict__ cs, float* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = perm_pad[i];
        if (e >= 0) out[e] = cs[i];
    }
}

__global__ void k_real_flags(const int32_t* __restrict__ perm_pad, int64_t m_pad, int32_t* __restrict__ f) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad;
         i += (int64_t)gridDim.x * blockDim.x)
        f[i] = perm_pad[i] >= 0 ? 1 : 0;
}

__global__ void k_compact_perm(const int32_t* __restrict__ perm_pad, const int32_t* __restrict__ f,
                               const int32_t* __restrict__ pos, int64_t m_pad, int32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad;
         i += (int64_t)gridDim.x * blockDim.x)
        if (f[i]) out[pos[i]] = perm_pad[i];
}

// One LOWD update (Algorithm 1's loop body) on e = (a, b) with f_e(a) = s, f_e(b) = w - s,
// written without branches: dd is the weight moved from a to b (negative: from b to a).
// |l_a - l_b| * 0.5 is exactly the paper's (l_u - l_v)/2 or (l_v - l_u)/2.
struct EdgeVal {
    float la, lb, s, w;
};

__device__ __forceinline__ float lowd_transfer(EdgeVal& e) {
    const float diff = e.la - e.lb;
    const bool gt = diff > 0.0f;
    const float cap = gt ? e.s : (e.w - e.s);
    const float d = fminf(fabsf(diff) * 0.5f, cap);
    const float dd = gt ? d : -d;
    e.la -= dd;
    e.lb += dd;
    return fminf(e.s - dd, e.w);
}

// Loads as unevaluated FP32 pairs hi + lo (|lo| <= ulp(hi) / 2).  A transfer moves d with
// Knuth's error-free TwoSum, so no update rounds a load: a node with thousands of updates a
// pass would otherwise carry a rounding walk of several ulp(l) per pass, which is what
// limits the reachable duality gap in plain FP32 (about 1e-6 relative at loads near 700).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
    s = a + b;
    const float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
}

// x.x + x.y += v: the rounding error of the high sum goes to the low part.  The low part is
// not renormalised per update: it gathers a random walk of errors of at most ulp(hi) / 2
// each (about sqrt(updates) ulp(hi), still far below hi), and the kernel renormalises once
// when it writes the loads back.
__device__ __forceinline__ void comp_add(float2& x, float v) {
    float t, e;
    two_sum(x.x, v, t, e);
    x.x = t;
    x.y += e;
}

// Algorithm 1's edge update on pair loads: returns the new split f_e(lo).
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

__device__ __forceinline__ uint32_t end_a(uint32_t uv) { return uv & 0xffffu; }
__device__ __forceinline__ uint32_t end_b(uint32_t uv) { return uv >> 16; }

// Four edges of one class: gather the 8 loads first (the ends are distinct inside a
// class, so no update can see another's write), update, scatter.
template <bool WEIGHTED>
__device__ __forceinline__ float4 update4(float* L, const uint4& uv, const float4& s, const float4& w) {
    EdgeVal e0{L[end_a(uv.x)], L[end_b(uv.x)], s.x, WEIGHTED ? w.x : 1.0f};
    EdgeVal e1{L[end_a(uv.y)], L[end_b(uv.y)], s.y, WEIGHTED ? w.y : 1.0f};
    EdgeVal e2{L[end_a(uv.z)], L[end_b(uv.z)], s.z, WEIGHTED ? w.z : 1.0f};
    EdgeVal e3{L[end_a(uv.w)], L[end_b(uv.w)], s.w, WEIGHTED ? w.w : 1.0f};
    float4 r;
    r.x = lowd_transfer(e0);
    r.y = lowd_transfer(e1);
    r.z = lowd_transfer(e2);
    r.w = lowd_transfer(e3);
    L[end_a(uv.x)] = e0.la; L[end_b(uv.x)] = e0.lb;
    L[end_a(uv.y)] = e1.la; L[end_b(uv.y)] = e1.lb;
    L[end_a(uv.z)] = e2.la; L[end_b(uv.z)] = e2.lb;
    L[end_a(uv.w)] = e3.la; L[end_b(uv.w)] = e3.lb;
    return r;
}

// The sweep.  One CTA; node loads (plus a sentinel slot n used by padding edges) in
// shared memory for all passes; class offsets in shared memory when they fit.  Each
// class segment is padded to a multiple of 4 edges with sentinel edges (both ends = n,
// a no-op), so thread t owns the 16-byte vector t of every class.  The classes of all
// passes form one stream q = 0, 1, ... (class q mod C); every thread keeps the vectors
// of the next kRing classes in a register ring, loading class q + kRing right after
// updating class q.  When a class comes round again in the next pass its splits were
// written by the same thread (this needs C >= kRing; smaller schedules use the simple
// kernel).  Vectors beyond blockDim.x of a class are updated straight from memory.
constexpr int kRingU = 8;  // ring depth, unit weights
constexpr int kRingW = 6;  // ring depth, weighted (one more vector per slot)
constexpr int kVecThreads = 512;

template <bool WEIGHTED>
__device__ __forceinline__ void ring_issue(int32_t cls, bool ok, const int32_t* __restrict__ CO, int tid,
                                           const uint4* __restrict__ cuv, const float4* __restrict__ cw,
                                           const float4* __restrict__ cs, int32_t& vi, uint4& ruv,
                                           float4& rs, float4& rw) {
    vi = -1;
    if (ok) {
        const int32_t i = (CO[cls] >> 2) + tid;
        if (i < (CO[cls + 1] >> 2)) {
            vi = i;
            ruv = __ldg(cuv + i);
            rs = __ldcg(cs + i);
            if (WEIGHTED) rw = __ldg(cw + i);
        }
    }
}

template <bool WEIGHTED>
__device__ __forceinline__ void class_overflow(float* L, int32_t cls, const int32_t* __restrict__ CO, int tid, int B,
                                               const uint4* __restrict__ cuv, const float4* __restrict__ cw,
                                               float4* __restrict__ cs) {
    const int32_t e4 = CO[cls + 1] >> 2;
    for (int32_t i = (CO[cls] >> 2) + B + tid; i < e4; i += B) {
        float4 w4 = WEIGHTED ? __ldg(cw + i) : float4{1.f, 1.f, 1.f, 1.f};
        float4 r = update4<WEIGHTED>(L, __ldg(cuv + i), __ldcg(cs + i), w4);
        __stcg(cs + i, r);
    }
}

template <bool WEIGHTED, int kRing, bool CO_SMEM>
__global__ void __launch_bounds__(kVecThreads, 1)
k_sweep_vec(int32_t n, int32_t C, const int32_t* __restrict__ coff,
            const uint4* __restrict__ cuv, const float4* __restrict__ cw, float4* __restrict__ cs,
            float* __restrict__ l, float* __restrict__ l_lo, int32_t passes) {
    extern __shared__ float L[];
    int32_t* COs = reinterpret_cast<int32_t*>(L + n + 1);
    const int tid = threadIdx.x;
    const int B = blockDim.x;
    // plain FP32 loads here: a pair load's low part is folded in and cleared on exit
    for (int i = tid; i <= n; i += B) L[i] = i < n ? l[i] + l_lo[i] : 0.0f;
    if (CO_SMEM)
        for (int i = tid; i <= C; i += B) COs[i] = coff[i];
    __syncthreads();
    const int32_t* __restrict__ CO = CO_SMEM ? COs : coff;
    const int64_t Q = (int64_t)C * passes;
    int32_t vi[kRing];
    uint4 ruv[kRing];
    float4 rs[kRing], rw[kRing];
    int32_t c_issue = 0;
    int64_t q_issue = 0;
#pragma unroll
    for (int j = 0; j < kRing; ++j) {
        ring_issue<WEIGHTED>(c_issue, q_issue < Q, CO, tid, cuv, cw, cs, vi[j], ruv[j], rs[j], rw[j]);
        c_issue = (c_issue + 1 == C) ? 0 : c_issue + 1;
        ++q_issue;
    }
    int32_t c = 0;
    for (int64_t q0 = 0; q0 < Q; q0 += kRing) {
#pragma unroll
        for (int j = 0; j < kRing; ++j) {
            if (q0 + j < Q) {
                if (vi[j] >= 0) __stcg(cs + vi[j], update4<WEIGHTED>(L, ruv[j], rs[j], rw[j]));
                class_overflow<WEIGHTED>(L, c, CO, tid, B, cuv, cw, cs);
                ring_issue<WEIGHTED>(c_issue, q_issue < Q, CO, tid, cuv, cw, cs, vi[j], ruv[j], rs[j], rw[j]);
                c_issue = (c_issue + 1 == C) ? 0 : c_issue + 1;
                ++q_issue;
                c = (c + 1 == C) ? 0 : c + 1;
                __syncthreads();
            }
        }
    }
    for (int i = tid; i < n; i += B) {
        l[i] = L[i];
        l_lo[i] = 0.0f;
    }
}

// ------------------------------------------------------------------ bulk-copy staged sweep
//
// A CTA barrier waits for the issuing threads' outstanding global loads and stores, so a
// sweep that prefetches into registers pays a memory round trip per class.  Here the
// edge data never passes through registers on its way in or out: a producer warp moves
// each class segment (packed ends, splits, weights) global -> shared with cp.async.bulk,
// completion signalled on one mbarrier per stage, and writes the updated splits back
// shared -> global with bulk stores.  Consumers (all other warps) wait on the stage's
// mbarrier, update the loads in shared memory, write the new splits into the stage, and
// meet at a named barrier of the consumer warps only, then hand the stage back on its
// "empty" mbarrier.  Stage q mod S holds class q mod C of the class stream.  The producer,
// on its own timeline, waits for stage q to be handed back, stores its splits, and loads
// stream position q + S - kStoreSlack into the stage whose store was issued kStoreSlack
// steps earlier (bulk wait_group.read kStoreSlack).  The splits of a class are re-read one
// pass later; wait_group kStoreGroups bounds the stores in flight, and
// C >= S - kStoreSlack + kStoreGroups + 1 makes the previous pass's store older than them.
// Every wait on an mbarrier is bounded; on expiry the kernel records an error flag and
// all threads leave the loop together.

constexpr int kTmaConsumers = 992;   // one edge per consumer thread per class
constexpr int kTmaMaxStages = 16;
constexpr int kStoreSlack = 1;    // bulk stores allowed to be still reading their stage
constexpr int kStoreGroups = 8;   // bulk stores allowed in flight at all
constexpr uint32_t kWaitLimit = 1u << 22;   // try_wait rounds before giving up

struct TmaLayout {
    uint32_t bars, L, CO, stages, stage_bytes, arr_bytes, total;
};

// Shared memory: mbarriers, loads as (hi, lo) pairs, the chunk boundaries (offsets of
// classes 0, G, 2G, ..., C), then the stages.  Offsets of the classes inside a chunk are not
// kept here: each consumer warp holds them in a register, fetched one chunk ahead.
__host__ __device__ inline TmaLayout tma_layout(int32_t n, int32_t C, int32_t S, int32_t Emax, bool weighted,
                                                int32_t G) {
    TmaLayout t;
    t.bars = 0;
    t.L = 16u * kTmaMaxStages;   // S full + S empty mbarriers
    t.CO = t.L + 8u * (uint32_t)(n + 1);
    const uint32_t NC = (uint32_t)((C + G - 1) / G);
    uint32_t end = t.CO + 4u * (NC + 1u);
    t.stages = (end + 127u) & ~127u;
    t.arr_bytes = ((4u * (uint32_t)Emax) + 127u) & ~127u;
    t.stage_bytes = t.arr_bytes * (weighted ? 3u : 2u);
    t.total = t.stages + t.stage_bytes * (uint32_t)S;
    return t;
}

template <bool WEIGHTED, int E>
__global__ void __launch_bounds__(kTmaConsumers + 32, 1)
k_sweep_tma(int32_t n, int32_t C, const int32_t* __restrict__ coff, const uint32_t* __restrict__ cuv,
            const float* __restrict__ cw, float* __restrict__ cs, float* __restrict__ l,
            float* __restrict__ l_lo, int32_t passes, int32_t S, int32_t G, int32_t Emax,
            int32_t* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    const TmaLayout lay = tma_layout(n, C, S, Emax, WEIGHTED, G);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + lay.bars);
    uint64_t* empty = full + S;   // S full barriers, then S empty barriers
    float2* L = reinterpret_cast<float2*>(smem + lay.L);   // (hi, lo) per node; slot n: padding
    int32_t* CK = reinterpret_cast<int32_t*>(smem + lay.CO);   // CK[j] = offset of class j G
    unsigned char* stages = smem + lay.stages;
    __shared__ volatile int32_t abort_flag;
    const int tid = threadIdx.x;
    const int nc = blockDim.x - 32;          // consumer threads; the last warp produces
    const int32_t NC = (C + G - 1) / G;      // chunks of G classes per pass
    for (int i = tid; i <= n; i += blockDim.x) L[i] = i < n ? make_float2(l[i], l_lo[i]) : make_float2(0.0f, 0.0f);
    for (int i = tid; i <= NC; i += blockDim.x) CK[i] = coff[min(i * G, C)];
    if (tid == 0) {
        abort_flag = 0;
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], 1);
        }
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    const int32_t P = NC * passes;           // the launcher keeps this < 2^31
    const int32_t ahead = S - kStoreSlack;   // chunks loaded ahead of the consumers
    if (tid >= nc) {
        // ---------------- producer warp (lane 0 works)
        if (tid == nc) {
            int32_t pf = 0, kf = 0, jf = 0;  // next fill: stream position, stage, chunk
            auto fill = [&]() {
                const int32_t beg = CK[jf];
                const int32_t end = CK[jf + 1];
                const uint32_t bytes = 4u * (uint32_t)(end - beg);
                unsigned char* st = stages + lay.stage_bytes * (uint32_t)kf;
                mbar_expect_tx(&full[kf], bytes * (WEIGHTED ? 3u : 2u));
                bulk_g2s(st, cuv + beg, bytes, &full[kf]);
                bulk_g2s(st + lay.arr_bytes, cs + beg, bytes, &full[kf]);
                if (WEIGHTED) bulk_g2s(st + 2 * lay.arr_bytes, cw + beg, bytes, &full[kf]);
                ++pf;
                kf = (kf + 1 == S) ? 0 : kf + 1;
                jf = (jf + 1 == NC) ? 0 : jf + 1;
            };
            while (pf < ahead && pf < P) fill();
            int32_t k = 0, j = 0;
            uint32_t parity = 0;
            int32_t q = 0;
            for (; q < P; ++q) {
                uint32_t spins = 0;
                bool ok = mbar_try_wait_sleep(&empty[k], parity, 1000);
                while (!ok && !abort_flag && ++spins < kWaitLimit) ok = mbar_try_wait_sleep(&empty[k], parity, 1000);
                if (!ok) { abort_flag = 1; break; }
                const int32_t beg = CK[j];
                const int32_t end = CK[j + 1];
                bulk_s2g(cs + beg, stages + lay.stage_bytes * (uint32_t)k + lay.arr_bytes, 4u * (uint32_t)(end - beg));
                bulk_commit();
                if (pf < P) {
                    // the stage to refill held position pf - S, stored kStoreSlack steps ago
                    bulk_wait<kStoreGroups>();
                    bulk_wait_read<kStoreSlack>();
                    fill();
                }
                if (++k == S) { k = 0; parity ^= 1u; }
                j = (j + 1 == NC) ? 0 : j + 1;
            }
            // fills [q, pf) were never handed back: on abort wait (bounded) for them to land
            if (q < P) drain_fills(full, S, q, pf, kWaitLimit);
            bulk_wait<0>();
            if (abort_flag) atomicOr(err, 1);
        }
        return;
    }
    // ---------------- consumers
    // Thread t updates ranks t, t + nc, ..., t + (E-1) nc of each class, all loads issued
    // before any store (the ends inside a class are distinct).  Classes of a chunk are
    // separated by a consumer barrier; at a chunk's end warp 0 waits for the next stage
    // and the barrier (which also ORs the abort flag) orders that stage's data before
    // every consumer's reads.
    auto wait_full = [&](int32_t kk, uint32_t par) -> bool {
        uint32_t spins = 0;
        bool ok = mbar_try_wait(&full[kk], par);
        while (!ok && ++spins < kWaitLimit) ok = mbar_try_wait(&full[kk], par);
        return ok;
    };
    // lane i of every consumer warp holds the offset of class jc G + i (i <= G) of a chunk
    const int lane = tid & 31;
    auto class_offsets = [&](int32_t jc) -> int32_t {
        const int32_t c = jc * G + lane;
        return (lane <= G && c <= C) ? __ldg(coff + c) : 0;
    };
    int32_t off_cur = class_offsets(0);
    int32_t off_nxt = class_offsets(NC > 1 ? 1 : 0);
    bool bad = false;
    if (tid < 32 && P > 0) bad = !wait_full(0, 0);
    bad = consumer_sync_or(nc, bad);
    int32_t k = 0, j = 0;
    uint32_t parity = 0;
    for (int32_t q = 0; q < P && !bad; ++q) {
        const int32_t c0 = j * G;
        const int32_t c1 = min(c0 + G, C);
        const int32_t base = __shfl_sync(0xffffffffu, off_cur, 0);
        unsigned char* st = stages + lay.stage_bytes * (uint32_t)k;
        const uint32_t* suv = reinterpret_cast<const uint32_t*>(st);
        float* ss = reinterpret_cast<float*>(st + lay.arr_bytes);
        const float* sw = reinterpret_cast<const float*>(st + 2 * lay.arr_bytes);
        int32_t cb = 0;
        for (int32_t c = c0; c < c1; ++c) {
            const int32_t ce = __shfl_sync(0xffffffffu, off_cur, c - c0 + 1) - base;
            if (E == 1) {
                // one edge per thread: the class fits the consumer threads
                const int32_t r = cb + tid;
                if (r < ce) {
                    const uint32_t uv = suv[r];
                    float2* pa = L + end_a(uv);
                    float2* pb = L + end_b(uv);
                    float2 A = *pa, Bv = *pb;
                    const float ns = comp_transfer(A, Bv, ss[r], WEIGHTED ? sw[r] : 1.0f);
                    *pa = A;
                    *pb = Bv;
                    ss[r] = ns;
                }
                cb = ce;
                if (c + 1 < c1) consumer_sync(nc);
                continue;
            }
            for (int32_t r0 = cb + tid; r0 < ce; r0 += E * nc) {
                uint32_t uv[E];
                EdgeVal e[E];
#pragma unroll
                for (int jj = 0; jj < E; ++jj) {
                    const int32_t r = r0 + jj * nc;
                    uv[jj] = r < ce ? suv[r] : ((uint32_t)n | ((uint32_t)n << 16));
                    e[jj].s = r < ce ? ss[r] : 0.0f;
                    e[jj].w = WEIGHTED ? (r < ce ? sw[r] : 0.0f) : 1.0f;
                }
                float2 A[E], Bv[E];
#pragma unroll
                for (int jj = 0; jj < E; ++jj) {
                    A[jj] = L[end_a(uv[jj])];
                    Bv[jj] = L[end_b(uv[jj])];
                }
                float ns[E];
#pragma unroll
                for (int jj = 0; jj < E; ++jj) ns[jj] = comp_transfer(A[jj], Bv[jj], e[jj].s, e[jj].w);
#pragma unroll
                for (int jj = 0; jj < E; ++jj) {
                    const int32_t r = r0 + jj * nc;
                    if (r < ce) {
                        L[end_a(uv[jj])] = A[jj];
                        L[end_b(uv[jj])] = Bv[jj];
                        ss[r] = ns[jj];
                    }
                }
            }
            cb = ce;
            if (c + 1 < c1) consumer_sync(nc);
        }
        fence_proxy_async_smem();
        const int32_t kprev = k;
        if (++k == S) { k = 0; parity ^= 1u; }
        j = (j + 1 == NC) ? 0 : j + 1;
        off_cur = off_nxt;                                   // chunk j's offsets, fetched a chunk ago
        off_nxt = class_offsets(j + 1 == NC ? 0 : j + 1);
        bool fail = false;
        if (tid < 32 && q + 1 < P) fail = !wait_full(k, parity);
        bad = consumer_sync_or(nc, fail);
        if (tid == 0) mbar_arrive(&empty[kprev]);
    }
    if (bad && tid == 0) {
        abort_flag = 1;
        atomicOr(err, 1);
    }
    for (int i = tid; i < n; i += nc) {
        const float2 x = L[i];
        const float u = x.x + x.y;     // renormalise: l = fl(hi + lo), l_lo = exact remainder
        l[i] = u;
        l_lo[i] = x.y - (u - x.x);
    }
}

// ------------------------------------------------------------------ staged sweep without class barriers
//
// The same staging as k_sweep_tma, but consumers do not meet at a barrier after every class.
// Instead every node carries a version in shared memory: the number of its updates done in
// the current pass (bit 15 holds the pass parity).  Each edge end carries its rank among
// its node's updates in the pass order (bit 15: the last one).  An update waits until both
// of its nodes show the version equal to its ranks, updates, then publishes rank + 1 (or
// the next pass's parity after the node's last update).  Every update therefore sees the
// loads left by the updates before it at its two nodes - the sequential pass in class
// order - while warps run ahead into later classes wherever those updates are done: a core
// node takes part in a fraction of the classes only, so most waits are already satisfied.

constexpr uint32_t kFlowSpins = 1u << 22;   // bounded wait on a version

__device__ __forceinline__ void fence_cta() { asm volatile("fence.acq_rel.cta;" ::: "memory"); }

struct FlowLayout {
    uint32_t bars, L, V, CO, stages, stage_bytes, arr_bytes, total;
};

__host__ __device__ inline FlowLayout flow_layout(int32_t n, int32_t C, int32_t S, int32_t Emax, bool weighted,
                                                  int32_t G) {
    FlowLayout t;
    t.bars = 0;
    t.L = 16u * kTmaMaxStages;                       // S full + S empty mbarriers
    t.V = t.L + 8u * (uint32_t)(n + 1);
    t.CO = (t.V + 4u * (uint32_t)(n + 1) + 15u) & ~15u;
    const uint32_t NC = (uint32_t)((C + G - 1) / G);
    const uint32_t end = t.CO + 4u * (NC + 1u);
    t.stages = (end + 127u) & ~127u;
    t.arr_bytes = ((4u * (uint32_t)Emax) + 127u) & ~127u;
    t.stage_bytes = t.arr_bytes * (weighted ? 4u : 3u);   // ends, splits, ranks (, weights)
    t.total = t.stages + t.stage_bytes * (uint32_t)S;
    return t;
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(kTmaConsumers + 32, 1)
k_sweep_flow(int32_t n, int32_t C, const int32_t* __restrict__ coff, const uint32_t* __restrict__ cuv,
             const uint32_t* __restrict__ crk, const float* __restrict__ cw, float* __restrict__ cs,
             float* __restrict__ l, float* __restrict__ l_lo, int32_t passes, int32_t S, int32_t G, int32_t Emax,
             int32_t* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    const FlowLayout lay = flow_layout(n, C, S, Emax, WEIGHTED, G);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + lay.bars);
    uint64_t* empty = full + S;
    float2* L = reinterpret_cast<float2*>(smem + lay.L);
    volatile uint32_t* V = reinterpret_cast<volatile uint32_t*>(smem + lay.V);
    int32_t* CK = reinterpret_cast<int32_t*>(smem + lay.CO);
    unsigned char* stages = smem + lay.stages;
    __shared__ volatile int32_t abort_flag;
    const int tid = threadIdx.x;
    const int nc = blockDim.x - 32;
    const int nwarps = nc >> 5;
    const int32_t NC = (C + G - 1) / G;
    for (int i = tid; i <= n; i += blockDim.x) {
        L[i] = i < n ? make_float2(l[i], l_lo[i]) : make_float2(0.0f, 0.0f);
        V[i] = 0u;
    }
    for (int i = tid; i <= NC; i += blockDim.x) CK[i] = coff[min(i * G, C)];
    if (tid == 0) {
        abort_flag = 0;
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], nwarps);   // every consumer warp releases the stage
        }
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    const int32_t P = NC * passes;           // the launcher keeps this < 2^31
    const int32_t ahead = S - kStoreSlack;
    if (tid >= nc) {
        // ---------------- producer warp (lane 0 works): as in k_sweep_tma, plus the ranks
        if (tid == nc) {
            int32_t pf = 0, kf = 0, jf = 0;
            auto fill = [&]() {
                const int32_t beg = CK[jf];
                const int32_t end = CK[jf + 1];
                const uint32_t bytes = 4u * (uint32_t)(end - beg);
                unsigned char* st = stages + lay.stage_bytes * (uint32_t)kf;
                mbar_expect_tx(&full[kf], bytes * (WEIGHTED ? 4u : 3u));
                bulk_g2s(st, cuv + beg, bytes, &full[kf]);
                bulk_g2s(st + lay.arr_bytes, cs + beg, bytes, &full[kf]);
                bulk_g2s(st + 2 * lay.arr_bytes, crk + beg, bytes, &full[kf]);
                if (WEIGHTED) bulk_g2s(st + 3 * lay.arr_bytes, cw + beg, bytes, &full[kf]);
                ++pf;
                kf = (kf + 1 == S) ? 0 : kf + 1;
                jf = (jf + 1 == NC) ? 0 : jf + 1;
            };
            while (pf < ahead && pf < P) fill();
            int32_t k = 0, j = 0;
            uint32_t parity = 0;
            int32_t q = 0;
            for (; q < P; ++q) {
                uint32_t spins = 0;
                bool ok = mbar_try_wait_sleep(&empty[k], parity, 1000);
                while (!ok && !abort_flag && ++spins < kWaitLimit) ok = mbar_try_wait_sleep(&empty[k], parity, 1000);
                if (!ok) { abort_flag = 1; break; }
                const int32_t beg = CK[j];
                const int32_t end = CK[j + 1];
                bulk_s2g(cs + beg, stages + lay.stage_bytes * (uint32_t)k + lay.arr_bytes, 4u * (uint32_t)(end - beg));
                bulk_commit();
                if (pf < P) {
                    bulk_wait<kStoreGroups>();
                    bulk_wait_read<kStoreSlack>();
                    fill();
                }
                if (++k == S) { k = 0; parity ^= 1u; }
                j = (j + 1 == NC) ? 0 : j + 1;
            }
            if (q < P) drain_fills(full, S, q, pf, kWaitLimit);
            bulk_wait<0>();
            if (abort_flag) atomicOr(err, 1);
        }
        return;
    }
    // ---------------- consumers: each warp walks the chunks on its own
    const int lane = tid & 31;
    auto class_offsets = [&](int32_t jc) -> int32_t {
        const int32_t c = jc * G + lane;
        return (lane <= G && c <= C) ? __ldg(coff + c) : 0;
    };
    int32_t off_cur = class_offsets(0);
    int32_t off_nxt = class_offsets(NC > 1 ? 1 : 0);
    int32_t k = 0, j = 0;
    uint32_t parity = 0;
    bool bad = false;
    for (int32_t q = 0; q < P; ++q) {
        // stage of chunk q landed? (lane 0 waits; the warp synchronises on the answer)
        bool ok = true;
        if (lane == 0) {
            uint32_t spins = 0;
            ok = mbar_try_wait(&full[k], parity);
            while (!ok && !abort_flag && ++spins < kWaitLimit) ok = mbar_try_wait(&full[k], parity);
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) { bad = true; break; }
        const uint32_t tb = (uint32_t)((q / NC) & 1) << 15;   // pass parity
        const int32_t c0 = j * G;
        const int32_t c1 = min(c0 + G, C);
        const int32_t base = __shfl_sync(0xffffffffu, off_cur, 0);
        unsigned char* st = stages + lay.stage_bytes * (uint32_t)k;
        const uint32_t* suv = reinterpret_cast<const uint32_t*>(st);
        float* ss = reinterpret_cast<float*>(st + lay.arr_bytes);
        const uint32_t* srk = reinterpret_cast<const uint32_t*>(st + 2 * lay.arr_bytes);
        const float* sw = reinterpret_cast<const float*>(st + 3 * lay.arr_bytes);
        int32_t cb = 0;
        for (int32_t c = c0; c < c1; ++c) {
            const int32_t ce = __shfl_sync(0xffffffffu, off_cur, c - c0 + 1) - base;
            const int32_t r = cb + tid;
            if (r < ce && !bad) {
                const uint32_t uv = suv[r];
                const uint32_t a = end_a(uv), b = end_b(uv);
                if ((int32_t)a < n) {   // padding edges join the sentinel n to itself
                    const uint32_t rk = srk[r];
                    const uint32_t ea = tb | (rk & 0x7fffu), eb = tb | ((rk >> 16) & 0x7fffu);
                    uint32_t spins = 0;
                    while (V[a] != ea || V[b] != eb) {
                        if (++spins > kFlowSpins || abort_flag) { bad = true; break; }
                    }
                    if (!bad) {
                        fence_cta();   // acquire: the loads below after the versions seen
                        float2 A = L[a], B = L[b];
                        const float sv = ss[r];
                        const float wv = WEIGHTED ? sw[r] : 1.0f;
                        const float ns = comp_transfer(A, B, sv, wv);
                        L[a] = A;
                        L[b] = B;
                        ss[r] = ns;
                        fence_cta();   // release: the loads above before the versions
                        V[a] = (rk & 0x8000u) ? (tb ^ 0x8000u) : ea + 1u;
                        V[b] = (rk & 0x80000000u) ? (tb ^ 0x8000u) : eb + 1u;
                    }
                }
            }
            cb = ce;
        }
        fence_proxy_async_smem();   // this warp's split writes before the bulk store reads them
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[k]);
        if (++k == S) { k = 0; parity ^= 1u; }
        j = (j + 1 == NC) ? 0 : j + 1;
        off_cur = off_nxt;
        off_nxt = class_offsets(j + 1 == NC ? 0 : j + 1);
        if (__any_sync(0xffffffffu, bad)) { bad = true; break; }
    }
    if (bad) {
        abort_flag = 1;
        if (lane == 0) atomicOr(err, 1);
    }
    // every warp must have released every stage before the loads are written back
    asm volatile("bar.sync 1, %0;" ::"r"(nc) : "memory");
    for (int i = tid; i < n; i += nc) {
        const float2 x = L[i];
        const float u = x.x + x.y;
        l[i] = u;
        l_lo[i] = x.y - (u - x.x);
    }
}

// rank of every end among its node's updates in the pass order (bit 15: the last one)
__global__ void k_occurrence_keys(const uint32_t* __restrict__ cuv, int64_t m_pad, uint32_t* __restrict__ key,
                                  int32_t* __restrict__ val) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m_pad;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t uv = cuv[p];
        key[2 * p] = uv & 0xffffu;
        key[2 * p + 1] = uv >> 16;
        val[2 * p] = (int32_t)(2 * p);
        val[2 * p + 1] = (int32_t)(2 * p + 1);
    }
}

__global__ void k_occurrence_ranks(const uint32_t* __restrict__ key, const int32_t* __restrict__ val, int64_t N,
                                   uint32_t n, uint16_t* __restrict__ rk) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = key[j];
        if (x >= n) continue;   // padding ends
        // first entry of x: binary search for the first j' with key[j'] == x
        int64_t lo = 0, hi = j;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (key[mid] < x) lo = mid + 1; else hi = mid;
        }
        const bool last = (j + 1 == N) || key[j + 1] != x;
        rk[val[j]] = (uint16_t)(((j - lo) & 0x7fff) | (last ? 0x8000 : 0));
    }
}

// Schedules with fewer classes than the ring depth: same layout, no prefetch ring.
template <bool WEIGHTED>
__global__ void __launch_bounds__(kVecThreads, 1)
k_sweep_simple(int32_t n, int32_t C, const int32_t* __restrict__ coff, const uint4* __restrict__ cuv,
               const float4* __restrict__ cw, float4* __restrict__ cs, float* __restrict__ l,
               float* __restrict__ l_lo, int32_t passes) {
    extern __shared__ float L[];
    const int tid = threadIdx.x;
    const int B = blockDim.x;
    // plain FP32 loads here: a pair load's low part is folded in and cleared on exit
    for (int i = tid; i <= n; i += B) L[i] = i < n ? l[i] + l_lo[i] : 0.0f;
    __syncthreads();
    for (int32_t t = 0; t < passes; ++t)
        for (int32_t c = 0; c < C; ++c) {
            const int32_t e4 = coff[c + 1] >> 2;
            for (int32_t i = (coff[c] >> 2) + tid; i < e4; i += B) {
                float4 w4 = WEIGHTED ? __ldg(cw + i) : float4{1.f, 1.f, 1.f, 1.f};
                float4 r = update4<WEIGHTED>(L, __ldg(cuv + i), __ldcg(cs + i), w4);
                __stcg(cs + i, r);
            }
            __syncthreads();
        }
    for (int i = tid; i < n; i += B) {
        l[i] = L[i];
        l_lo[i] = 0.0f;
    }
}

template <bool WEIGHTED>
cudaError_t launch_sweep_tma(lowd_ctx* h, int32_t passes, int32_t maxlen, bool* launched) {
    *launched = false;
    const size_t budget = 227 * 1024;
    // chunk size G (classes per staged copy) and stage count S: the largest G whose
    // chunks leave room for at least kMinStages stages, then as many stages as fit
    constexpr int kMinStages = 3;
    int32_t G = 0, S = 0, chunk = 0;
    TmaLayout lay{};
    for (int32_t g : {16, 8, 4, 2, 1}) {
        int32_t mx = 0;  // longest chunk of g classes
        for (int32_t c0 = 0; c0 < h->C; c0 += g) mx = max(mx, h->coff_h[min(c0 + g, h->C)] - h->coff_h[c0]);
        int32_t s = kTmaMaxStages;
        TmaLayout t = tma_layout(h->n, h->C, s, mx, WEIGHTED, g);
        while (s > kMinStages && t.total > budget) t = tma_layout(h->n, h->C, --s, mx, WEIGHTED, g);
        if (t.total <= budget) { G = g; S = s; chunk = mx; lay = t; break; }
    }
    if (G == 0) return cudaSuccess;
    const int32_t NC = (h->C + G - 1) / G;
    // a chunk's splits are re-read one pass later: its store must be older than the
    // kStoreGroups stores allowed in flight when the producer loads it again
    if (NC < S - kStoreSlack + kStoreGroups + 1) return cudaSuccess;
    // edges per consumer thread: enough warps to hide latency, few enough to keep the
    // per-class bookkeeping small
    const int E = maxlen > 2 * kTmaConsumers ? 4 : (maxlen > kTmaConsumers ? 2 : 1);
    int threads = ((((maxlen + E - 1) / E) + 31) / 32) * 32;
    if (threads < 64) threads = 64;
    if (threads > kTmaConsumers) threads = kTmaConsumers;
    auto kern = E == 4 ? k_sweep_tma<WEIGHTED, 4> : (E == 2 ? k_sweep_tma<WEIGHTED, 2> : k_sweep_tma<WEIGHTED, 1>);
    h->sweep_kernel = 1;
    h->sweep_E = E;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
    if (e != cudaSuccess) return e;
    const int32_t per = (int32_t)(0x7fffffff / NC);
    for (int32_t done = 0; done < passes && e == cudaSuccess;) {
        const int32_t k = passes - done < per ? passes - done : per;
        LOWD_LAUNCH(kern, 1, threads + 32, lay.total, h->st, h->n, h->C, h->coff, h->cuv, h->cw, h->cs, h->l,
                    h->l_lo, k, S, G, chunk, h->d_i32 + 8);
        e = cudaGetLastError();
        done += k;
    }
    *launched = true;
    return e;
}

// Ranks of every end among its node's updates in the pass order (the staged sweep without
// class barriers), plain classes only; built on the first request for node versions.  Node
// degrees must fit 15 bits; otherwise (or without memory) h->crk stays null and the staged
// sweep with class barriers runs instead.
void sweep_ranks(lowd_ctx* h) {
    cudaStream_t st = h->st;
    const int32_t n = h->n;
    const int64_t mq = h->coff_h[h->C];
    if (mq <= 0 || lowd_max_degree(h) >= 0x7fff) return;
    uint32_t* ok[2] = {nullptr, nullptr};
    int32_t* ov[2] = {nullptr, nullptr};
    bool good = h->need_tmp(lowd_sort_tmp_bytes(2 * mq)) == LOWD_OK;
    good = good && dalloc(h, &ok[0], 2 * mq) == LOWD_OK;
    good = good && dalloc(h, &ok[1], 2 * mq) == LOWD_OK;
    good = good && dalloc(h, &ov[0], 2 * mq) == LOWD_OK;
    good = good && dalloc(h, &ov[1], 2 * mq) == LOWD_OK;
    good = good && dalloc(h, &h->crk, mq) == LOWD_OK;
    if (good) {
        cudaMemsetAsync(h->crk, 0, sizeof(uint32_t) * (size_t)mq, st);
        LOWD_LAUNCH(k_occurrence_keys, grid_for(mq), kT, 0, st, h->cuv, mq, ok[0], ov[0]);
        const int cur2 = radix_sort_pairs<uint32_t, int32_t>(ok[0], ov[0], ok[1], ov[1], 2 * mq,
                                                             bit_length_u64((uint64_t)n), h->tmp, st);
        LOWD_LAUNCH(k_occurrence_ranks, grid_for(2 * mq), kT, 0, st, ok[cur2], ov[cur2], 2 * mq, (uint32_t)n,
                    reinterpret_cast<uint16_t*>(h->crk));
        if (cudaGetLastError() != cudaSuccess) dfree(h, &h->crk);
    } else {
        dfree(h, &h->crk);
        cudaGetLastError();
    }
    dfree(h, &ok[0]); dfree(h, &ok[1]); dfree(h, &ov[0]); dfree(h, &ov[1]);
}

template <bool WEIGHTED>
cudaError_t launch_sweep_flow(lowd_ctx* h, int32_t passes, int32_t maxlen, bool* launched) {
    *launched = false;
    if (maxlen > kTmaConsumers) return cudaSuccess;
    if (!h->crk) sweep_ranks(h);
    if (!h->crk) return cudaSuccess;
    const size_t budget = 227 * 1024;
    constexpr int kMinStages = 3;
    int32_t G = 0, S = 0, chunk = 0;
    FlowLayout lay{};
    for (int32_t g : {16, 8, 4, 2, 1}) {
        int32_t mx = 0;
        for (int32_t c0 = 0; c0 < h->C; c0 += g) mx = max(mx, h->coff_h[min(c0 + g, h->C)] - h->coff_h[c0]);
        int32_t s = kTmaMaxStages;
        FlowLayout t = flow_layout(h->n, h->C, s, mx, WEIGHTED, g);
        while (s > kMinStages && t.total > budget) t = flow_layout(h->n, h->C, --s, mx, WEIGHTED, g);
        if (t.total > budget) continue;
        const int32_t NC = (h->C + g - 1) / g;
        if (NC < s - kStoreSlack + kStoreGroups + 1) continue;   // split store ordering, as k_sweep_tma
        G = g; S = s; chunk = mx; lay = t;
        break;
    }
    if (G == 0) return cudaSuccess;
    const int32_t NC = (h->C + G - 1) / G;
    int threads = ((maxlen + 31) / 32) * 32;
    if (threads < 64) threads = 64;
    auto kern = k_sweep_flow<WEIGHTED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
    if (e != cudaSuccess) return e;
    h->sweep_kernel = 5;
    h->sweep_E = 1;
    // the pass parity lives in bit 15 of a version: any number of passes per launch works; the
    // stream position stays below 2^31
    const int32_t per = (int32_t)(0x7fffffff / NC);
    for (int32_t done = 0; done < passes && e == cudaSuccess;) {
        const int32_t k = passes - done < per ? passes - done : per;
        LOWD_LAUNCH(kern, 1, threads + 32, lay.total, h->st, h->n, h->C, h->coff, h->cuv, h->crk, h->cw, h->cs,
                    h->l, h->l_lo, k, S, G, chunk, h->d_i32 + 8);
        e = cudaGetLastError();
        done += k;
    }
    *launched = true;
    return e;
}

template <bool WEIGHTED>
cudaError_t launch_sweep(lowd_ctx* h, int32_t passes) {
    {
        int32_t maxlen = 0;
        for (int32_t c = 0; c < h->C; ++c) maxlen = max(maxlen, h->coff_h[c + 1] - h->coff_h[c]);
        bool launched = false;
        cudaError_t e = cudaSuccess;
        if (h->use_versions) {
            e = launch_sweep_flow<WEIGHTED>(h, passes, maxlen, &launched);
            if (e != cudaSuccess || launched) return e;
        }
        e = launch_sweep_tma<WEIGHTED>(h, passes, maxlen, &launched);
        if (e != cudaSuccess || launched) return e;
    }
    const size_t lbytes = sizeof(float) * ((size_t)h->n + 1);
    const size_t cbytes = sizeof(int32_t) * ((size_t)h->C + 1);
    const size_t budget = 227 * 1024;
    const int co_smem = lbytes + cbytes <= budget ? 1 : 0;
    const size_t smem = lbytes + (co_smem ? cbytes : 0);
    int32_t maxv = 0;  // largest class, in 4-edge vectors
    for (int32_t c = 0; c < h->C; ++c) maxv = max(maxv, (h->coff_h[c + 1] - h->coff_h[c]) >> 2);
    int threads = ((maxv + 31) / 32) * 32;
    if (threads < 64) threads = 64;
    if (threads > kVecThreads) threads = kVecThreads;
    const uint4* cuv = reinterpret_cast<const uint4*>(h->cuv);
    const float4* cw = reinterpret_cast<const float4*>(h->cw);
    float4* cs = reinterpret_cast<float4*>(h->cs);
    constexpr int kRing = WEIGHTED ? kRingW : kRingU;
    if (h->C >= kRing) {
        auto kern = co_smem ? k_sweep_vec<WEIGHTED, kRing, true> : k_sweep_vec<WEIGHTED, kRing, false>;
        h->sweep_kernel = 2;
        h->sweep_E = 0;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        LOWD_LAUNCH(kern, 1, threads, smem, h->st, h->n, h->C, h->coff, cuv, cw, cs, h->l, h->l_lo, passes);
    } else {
        auto kern = k_sweep_simple<WEIGHTED>;
        h->sweep_kernel = 3;
        h->sweep_E = 0;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lbytes);
        if (e != cudaSuccess) return e;
        LOWD_LAUNCH(kern, 1, threads, lbytes, h->st, h->n, h->C, h->coff, cuv, cw, cs, h->l, h->l_lo, passes);
    }
    return cudaGetLastError();
}

cudaError_t run_passes(lowd_ctx* h, int32_t passes) {
    if (passes <= 0 || h->m == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(h->d_i32 + 8, 0, sizeof(int32_t), h->st);
    if (e != cudaSuccess) return e;
    if (h->sched == 2) return lowd_stream_passes(h, passes);
    if (h->star_S == 0) return h->cw ? launch_sweep<true>(h, passes) : launch_sweep<false>(h, passes);
    // hub stars: per pass, the plain classes, then the star steps
    e = cudaMemsetAsync(h->d_i32 + 12, 0, 2 * sizeof(int32_t), h->st);   // grid barrier words
    for (int32_t t = 0; t < passes && e == cudaSuccess; ++t) {
        if (h->C > 0) e = h->cw ? launch_sweep<true>(h, 1) : launch_sweep<false>(h, 1);
        if (e == cudaSuccess) e = lowd_star_pass(h);
    }
    return e;
}

}  // namespace

// Build the schedule and the class-major streams, then initialise the splits (equal
// split, or the given canonical-order splits) and the loads.
lowd_status lowd_sweep_prepare(lowd_ctx* h, int schedule_req, const float* init_splits_canon) {
    cudaStream_t st = h->st;
    const int64_t m = h->m;
    const int32_t n = h->n;
    // schedule 2 (streamed, loads in global memory) when asked for, or automatically when
    // the loads do not fit the one-CTA sweep's shared memory
    if (schedule_req == 2 || (schedule_req == 0 && n > LOWD_SMEM_NODES))
        return lowd_stream_prepare(h, init_splits_canon);
    if (n > LOWD_SMEM_NODES) {
        snprintf(h->err, sizeof(h->err), "current graph has %d nodes; the shared-memory sweep holds at most %d",
                 n, LOWD_SMEM_NODES);
        return LOWD_ERR_TOO_LARGE;
    }
    uint64_t* key[2] = {nullptr, nullptr};
    int32_t* val[2] = {nullptr, nullptr};
    int32_t *head = nullptr, *hpos = nullptr, *pcnt = nullptr;
    StarSplit sp;   // hub stars: the circle colouring covers the plain edges
    lowd_status s = LOWD_OK;
    auto cleanup = [&]() {
        sp.release(h);
        dfree(h, &key[0]); dfree(h, &key[1]); dfree(h, &val[0]); dfree(h, &val[1]);
        dfree(h, &head); dfree(h, &hpos); dfree(h, &pcnt);
    };
    do {
        if ((s = lowd_star_split(h, h->hub_tau, 1, &sp))) break;
        const int64_t mc = sp.pid ? sp.m_plain : m;   // edges the colouring covers
        const int32_t* cu = sp.pid ? sp.gu : h->u;
        const int32_t* cv = sp.pid ? sp.gv : h->v;
        if ((s = h->need_tmp(lowd_sort_tmp_bytes(m > n ? m : n)))) break;
        if ((s = dalloc(h, &key[0], m))) break;
        if ((s = dalloc(h, &key[1], m))) break;
        if ((s = dalloc(h, &val[0], m))) break;
        if ((s = dalloc(h, &val[1], m))) break;
        if ((s = dalloc(h, &head, m))) break;
        if ((s = dalloc(h, &hpos, m))) break;
        int32_t C = 0;
        int cur = 0;
        uint64_t* kfin = key[0];
        int32_t* vfin = val[0];
        if (mc > 0) {
            LOWD_LAUNCH(k_circle_colour, grid_for(mc), kT, 0, st, cu, cv, mc, n, key[0], val[0]);
            const uint32_t P = (uint32_t)(n + (n & 1)) - 1u;
            const int cbits = bit_length_u64(P > 0 ? P - 1 : 0);
            cur = radix_sort_pairs<uint64_t, int32_t>(key[0], val[0], key[1], val[1], mc, cbits + kBankBits + 1, h->tmp, st);
            uint64_t* kA = key[cur];
            int32_t* vA = val[cur];
            uint64_t* kB = key[1 - cur];
            int32_t* vB = val[1 - cur];
            LOWD_LAUNCH(k_bank_rounds, grid_for(mc), kT, 0, st, kA, mc, kB);
            const int r2 = radix_sort_pairs<uint64_t, int32_t>(kB, vA, kA, vB, mc, cbits + kBankBits + 1 + kRankBits, h->tmp, st);
            kfin = r2 ? kA : kB;
            vfin = r2 ? vB : vA;
            if (sp.pid) LOWD_LAUNCH(k_subset_to_ids, grid_for(mc), kT, 0, st, sp.pid, mc, vfin);
            LOWD_LAUNCH(k_class_heads, grid_for(mc), kT, 0, st, kfin, mc, kRankBits + kBankBits + 1, head);
            scan_exclusive<int32_t>(head, hpos, mc, h->d_i32 + 5, h->tmp, st);
            if (cudaMemcpyAsync(h->h_pin, h->d_i32 + 5, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
            C = *(int32_t*)h->h_pin;
        }
        h->C = C;
        // real and padded class offsets
        if ((s = dalloc(h, &h->coff_real, (size_t)C + 1))) break;
        if ((s = dalloc(h, &h->coff, (size_t)C + 1))) break;
        if ((s = dalloc(h, &pcnt, (size_t)C + 1))) break;
        if (mc > 0) {
            LOWD_LAUNCH(k_class_offsets, grid_for(mc), kT, 0, st, head, hpos, mc, C, h->coff_real);
            LOWD_LAUNCH(k_pad_sizes, grid_for(C), kT, 0, st, h->coff_real, C, pcnt);
            scan_exclusive<int32_t>(pcnt, h->coff, C, h->coff + C, h->tmp, st);
        } else {
            cudaMemsetAsync(h->coff_real, 0, sizeof(int32_t), st);
            cudaMemsetAsync(h->coff, 0, sizeof(int32_t), st);
        }
        h->coff_h = (int32_t*)malloc(sizeof(int32_t) * ((size_t)C + 1));
        if (!h->coff_h) { s = LOWD_ERR_OUT_OF_MEMORY; break; }
        if (cudaMemcpyAsync(h->coff_h, h->coff, sizeof(int32_t) * ((size_t)C + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
        const int64_t m_pad_plain = h->coff_h[C];
        const int64_t m_pad = m_pad_plain + sp.ms;   // the star edges follow the plain classes
        h->m_pad = m_pad;
        if ((s = dalloc(h, &h->perm, m_pad))) break;
        if (m_pad > 0) LOWD_LAUNCH(k_fill_perm, grid_for(m_pad), kT, 0, st, h->perm, m_pad);
        if (mc > 0)
            LOWD_LAUNCH(k_scatter_padded, grid_for(mc), kT, 0, st, vfin, head, hpos, h->coff_real, h->coff, mc,
                        h->perm);
        if ((s = lowd_star_blocks(h, sp, m_pad_plain, C, mc))) break;
        if ((s = dalloc(h, &h->cuv, m_pad))) break;
        if (h->w && (s = dalloc(h, &h->cw, m_pad))) break;
        if ((s = dalloc(h, &h->cs, m_pad))) break;
        if ((s = dalloc(h, &h->l, (size_t)n + 1))) break;
        if ((s = dalloc(h, &h->l_lo, (size_t)n + 1))) break;
        if (m_pad > 0)
            LOWD_LAUNCH(k_gather_streams, grid_for(m_pad), kT, 0, st, h->perm, m_pad, n, h->u, h->v, h->w,
                        init_splits_canon, h->cuv, h->cw, h->cs);
        if (cudaGetLastError() != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
        h->sched = 1;
        h->inited = 1;
        double st3[3];
        s = lowd_sweep_rederive(h, st3);
    } while (0);
    cleanup();
    return s;
}

// FP64 loads from the splits; FP32 loads refreshed from them; stats3 = (sum, sum sq, max).
lowd_status lowd_sweep_rederive(lowd_ctx* h, double* stats3) {
    cudaStream_t st = h->st;
    double* L64 = nullptr;
    LOWD_TRY(dalloc(h, &L64, h->n));
    cudaMemsetAsync(L64, 0, sizeof(double) * (size_t)h->n, st);
    cudaMemsetAsync(h->d_stats, 0, 3 * sizeof(double), st);
    if (h->sched == 2) {
        lowd_status r = lowd_stream_rederive(h, L64);
        if (r != LOWD_OK) { dfree(h, &L64); return r; }
    } else if (h->m_pad > 0) {
        LOWD_LAUNCH(k_rederive, grid_for(h->m_pad), kT, 0, st, h->m_pad, h->cuv, h->cw, h->cs, L64);
    }
    LOWD_LAUNCH(k_load_stats, grid_for(h->n), kT, 0, st, L64, h->n, h->l, h->l_lo, h->d_stats);
    double tmp3[3];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp3, h->d_stats, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(h, &L64);
    if (e != cudaSuccess) return h->fail(e);
    if (stats3) { stats3[0] = tmp3[0]; stats3[1] = tmp3[1]; stats3[2] = tmp3[2]; }
    return LOWD_OK;
}

lowd_status lowd_sweep_splits_canonical(lowd_ctx* h, float* out_dev) {
    if (h->m_pad > 0)
        LOWD_LAUNCH(k_splits_to_canonical, grid_for(h->m_pad), kT, 0, h->st, h->perm, h->m_pad, h->cs, out_dev);
    LOWD_CK_LAUNCH();
    return LOWD_OK;
}

lowd_status lowd_sweep_load_canonical(lowd_ctx* h, const float* splits_dev) {
    if (h->m_pad > 0)
        LOWD_LAUNCH(k_splits_from_canonical, grid_for(h->m_pad), kT, 0, h->st, h->perm, h->m_pad, splits_dev, h->cs);
    LOWD_CK_LAUNCH();
    return LOWD_OK;
}

// The update order as canonical edge ids (padding removed) into out_dev [m].
lowd_status lowd_sweep_edge_order(lowd_ctx* h, int32_t* out_dev) {
    int32_t *f = nullptr, *pos = nullptr;
    LOWD_TRY(h->need_tmp(lowd_sort_tmp_bytes(h->m_pad)));
    LOWD_TRY(dalloc(h, &f, h->m_pad));
    lowd_status s = dalloc(h, &pos, h->m_pad);
    if (s == LOWD_OK && h->m_pad > 0) {
        LOWD_LAUNCH(k_real_flags, grid_for(h->m_pad), kT, 0, h->st, h->perm, h->m_pad, f);
        scan_exclusive<int32_t>(f, pos, h->m_pad, nullptr, h->tmp, h->st);
        LOWD_LAUNCH(k_compact_perm, grid_for(h->m_pad), kT, 0, h->st, h->perm, f, pos, h->m_pad, out_dev);
        if (cudaGetLastError() != cudaSuccess) s = h->fail(cudaGetLastError());
    }
    cudaStreamSynchronize(h->st);
    dfree(h, &f);
    dfree(h, &pos);
    return s;
}

lowd_status lowd_sweep_run(lowd_ctx* h, int32_t k, const lowd_options* opt, lowd_stats* out) {
    lowd_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    lowd_stats stt;
    memset(&stt, 0, sizeof(stt));
    double st3[3] = {0, 0, 0};
    int32_t done = 0;
    int converged = 0;
    double rho_best = 0.0;
    int32_t best_size = 0;
    const int32_t R = o.rederive_every == 0 ? 50 : (o.rederive_every < 0 ? 0x7fffffff : o.rederive_every);
    int32_t since = 0;        // passes since the loads were last re-derived from the splits
    int32_t since_check = 0;  // passes since the last check
    while (done < k) {
        int32_t step = k - done;
        if (o.check_every > 0 && o.check_every - since_check < step) step = o.check_every - since_check;
        if (R - since < step) step = R - since;
        LOWD_CK(run_passes(h, step));
        LOWD_CK(cudaMemcpyAsync(h->h_pin + 8, h->d_i32 + 8, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
        LOWD_CK(cudaStreamSynchronize(h->st));
        const int32_t kerr = *(int32_t*)(h->h_pin + 8);
        if (kerr != 0) {
            snprintf(h->err, sizeof(h->err), "%s",
                     (kerr & 4) ? "sweep: a read descriptor pointed outside the stages"
                                : ((kerr & 2) ? "sweep: a bounded grid barrier expired"
                                              : "sweep: a bounded wait on a staged copy expired"));
            return LOWD_ERR_CUDA;
        }
        done += step;
        h->iters += step;
        since += step;
        since_check += step;
        const bool check = o.check_every > 0 && (since_check >= o.check_every || done == k);
        if (since >= R && !check && done < k) {
            LOWD_TRY(lowd_sweep_rederive(h, st3));
            since = 0;
        }
        if (check) {
            LOWD_TRY(lowd_sweep_rederive(h, st3));
            since = 0;
            since_check = 0;
            int64_t Wb = 0;
            int32_t kb = 0;
            LOWD_TRY(lowd_extract_best(h, h->l, nullptr, &kb, &Wb));
            double scale = h->wu ? 1048576.0 : 1.0;
            rho_best = kb > 0 ? (double)Wb / scale / (double)kb : 0.0;
            best_size = kb;
            stt.checks_done++;
            if (o.rel_tol > 0 && rho_best > 0 && (st3[2] - rho_best) / rho_best <= o.rel_tol) {
                converged = 1;
                break;
            }
        }
    }
    if (o.check_every <= 0) LOWD_TRY(lowd_sweep_rederive(h, st3));
    stt.iters_done = h->iters;
    stt.sum_load = st3[0];
    stt.sum_load_sq = st3[1];
    stt.max_load = st3[2];
    stt.rho_best = rho_best;
    stt.best_size = best_size;
    stt.converged = converged;
    if (out) *out = stt;
    if (o.rel_tol > 0 && !converged) return LOWD_ERR_NOT_CONVERGED;
    return LOWD_OK;
}
