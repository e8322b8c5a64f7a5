// Graph input and Algorithm 2 (pruning) on the GPU.
//
//  - load: validation, canonical (lo, hi) keys, stable radix sort, removal of repeated
//    pairs keeping the first occurrence (the paper drops multiple edges and self-loops
//    and ignores direction, Sec. IV);
//  - prune: weighted degrees in exact 2^-20 units, the counting sort of nodes by degree
//    (Sec. III-D), then synchronous rounds of Algorithm 2: every node with
//    d_H(u) * |H| < W(H) is removed at once, its edges subtract their weight from the
//    surviving ends, and the bound is recomputed; finally H is compacted with its nodes
//    renumbered by ascending original id and its edges in their original order.
#include "ctx.cuh"
#include "prims.cuh"

using namespace lowd;

namespace {

constexpr int kT = 256;


enum { ERR_RANGE = 1, ERR_LOOP = 2, ERR_WEIGHT = 4, ERR_GRID = 8, UNSORTED = 16 };

// One pass over the input pairs: range, loop and weight checks, and whether the input is
// already strictly increasing in the canonical key lo * n + hi; with keys != null the keys
// (and the input position of each) are written for the sort.
// Weight units with integer arithmetic only (FP64 is slow on this GPU): rint(x * 2^20) for
// a finite x > 0, at least 1.  x = m 2^(e - 150) with a 24-bit integer m, so x 2^20 =
// m 2^(e - 130): a left shift, or a right shift rounded to nearest, ties to even.
__device__ __forceinline__ int64_t weight_units(float x) {
    const uint32_t bits = __float_as_uint(x);
    const int ex = (int)((bits >> 23) & 0xffu);
    if (ex == 0) return 1;   // subnormal: x 2^20 < 1
    const uint64_t m = (uint64_t)((bits & 0x7fffffu) | 0x800000u);
    const int sh = ex - 130;
    if (sh >= 0) return sh >= 39 ? INT64_MAX : (int64_t)(m << sh);
    const int r = -sh;
    if (r > 25) return 1;    // x 2^20 < 1/2: rounds to 0
    const uint64_t q = m >> r, rem = m & ((1ull << r) - 1ull), half = 1ull << (r - 1);
    const uint64_t y = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
    return y < 1ull ? 1 : (int64_t)y;
}

// x 2^20 is an integer (the weight lies on the 2^-20 grid); the product by a power of two is
// exact in FP32 unless it overflows, and an infinite product counts as on the grid, as the
// FP64 product (then a huge integer) would
__device__ __forceinline__ bool on_grid(float x) {
    const float y = x * 1048576.0f;
    return y == rintf(y);
}

__global__ void k_check_keys(const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                             const float* __restrict__ w, int64_t m, int32_t n,
                             uint64_t* __restrict__ keys, uint32_t* __restrict__ idx,
                             int32_t* __restrict__ err) {
    int flags = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = u[e], b = v[e];
        if (a < 0 || a >= n || b < 0 || b >= n) {
            flags |= ERR_RANGE;
            if (keys) { keys[e] = 0; idx[e] = (uint32_t)e; }
            continue;
        }
        if (a == b) flags |= ERR_LOOP;
        uint64_t lo = (uint64_t)min(a, b), hi = (uint64_t)max(a, b);
        uint64_t k = lo * (uint64_t)n + hi;
        if (keys) {
            keys[e] = k;
            idx[e] = (uint32_t)e;
        }
        if (w) {
            float x = w[e];
            if (!(x > 0.0f) || !isfinite(x)) flags |= ERR_WEIGHT;
            if (!on_grid(x)) flags |= ERR_GRID;
        }
        if (e > 0) {
            int32_t pa = u[e - 1], pb = v[e - 1];
            if (pa >= 0 && pa < n && pb >= 0 && pb < n) {
                uint64_t pk = (uint64_t)min(pa, pb) * (uint64_t)n + (uint64_t)max(pa, pb);
                if (!(pk < k)) flags |= UNSORTED;
            }
        }
    }
    flags = __reduce_or_sync(0xffffffffu, flags);
    if (flags && lane_id() == 0) atomicOr(err, flags);
}

// The same checks when no keys are wanted (first look at an input), four edges per thread
// with 16-byte loads (u, v and w 16-byte aligned), the tail edges one per thread.
__device__ __forceinline__ int check_one(int32_t a, int32_t b, bool hw, float x, int32_t n, bool& valid,
                                         uint64_t& k) {
    int f = 0;
    valid = a >= 0 && a < n && b >= 0 && b < n;
    if (!valid) return ERR_RANGE;
    if (a == b) f |= ERR_LOOP;
    k = (uint64_t)min(a, b) * (uint64_t)n + (uint64_t)max(a, b);
    if (hw) {
        if (!(x > 0.0f) || !isfinite(x)) f |= ERR_WEIGHT;
        if (!on_grid(x)) f |= ERR_GRID;
    }
    return f;
}

__global__ void k_check_vec4(const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                             const float* __restrict__ w, int64_t m, int32_t n, int32_t* __restrict__ err) {
    int flags = 0;
    const int64_t m4 = m >> 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m4; q += stride) {
        const int4 a4 = __ldcs(reinterpret_cast<const int4*>(u) + q);
        const int4 b4 = __ldcs(reinterpret_cast<const int4*>(v) + q);
        const float4 w4 = w ? __ldcs(reinterpret_cast<const float4*>(w) + q) : make_float4(1.f, 1.f, 1.f, 1.f);
        const int32_t aa[4] = {a4.x, a4.y, a4.z, a4.w}, bb[4] = {b4.x, b4.y, b4.z, b4.w};
        const float ww[4] = {w4.x, w4.y, w4.z, w4.w};
        bool pvalid = false;
        uint64_t pk = 0;
        if (q > 0) {
            const int32_t pa = u[4 * q - 1], pb = v[4 * q - 1];
            pvalid = pa >= 0 && pa < n && pb >= 0 && pb < n;
            pk = pvalid ? (uint64_t)min(pa, pb) * (uint64_t)n + (uint64_t)max(pa, pb) : 0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            bool valid;
            uint64_t k = 0;
            flags |= check_one(aa[j], bb[j], w != nullptr, ww[j], n, valid, k);
            if (valid && pvalid && !(pk < k)) flags |= UNSORTED;
            pvalid = valid;
            pk = k;
        }
    }
    for (int64_t e = 4 * m4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        bool valid;
        uint64_t k = 0;
        flags |= check_one(u[e], v[e], w != nullptr, w ? w[e] : 1.0f, n, valid, k);
        if (valid && e > 0) {
            const int32_t pa = u[e - 1], pb = v[e - 1];
            if (pa >= 0 && pa < n && pb >= 0 && pb < n) {
                const uint64_t pk = (uint64_t)min(pa, pb) * (uint64_t)n + (uint64_t)max(pa, pb);
                if (!(pk < k)) flags |= UNSORTED;
            }
        }
    }
    flags = __reduce_or_sync(0xffffffffu, flags);
    if (flags && lane_id() == 0) atomicOr(err, flags);
}

__global__ void k_first_flags(const uint64_t* __restrict__ keys, int64_t m, int32_t* __restrict__ f) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        f[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_emit_unique(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ idx,
                              const int32_t* __restrict__ first, const int32_t* __restrict__ pos,
                              int64_t m, int32_t n, const float* __restrict__ w_in,
                              int32_t* __restrict__ u, int32_t* __restrict__ v,
                              float* __restrict__ w, int64_t* __restrict__ wu) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (first && !first[i]) continue;
        int64_t p = pos ? pos[i] : i;
        uint64_t k = keys[i];
        u[p] = (int32_t)(k / (uint64_t)n);
        v[p] = (int32_t)(k % (uint64_t)n);
        if (w_in) {
            float x = w_in[idx[i]];
            w[p] = x;
            wu[p] = weight_units(x);
        }
    }
}

// Add the same x to counter[node] for every lane, one atomic per distinct node of the warp
// (the edge lists are sorted by their low end, so neighbouring lanes often share it).  All
// lanes of the warp take part; lanes with nothing to add pass node = -1.
template <class T>
__device__ __forceinline__ void warp_add(T* counter, int32_t node, T x) {
    const unsigned peers = __match_any_sync(0xffffffffu, node);
    if (node >= 0 && (int)lane_id() == __ffs(peers) - 1) atomicAdd(&counter[node], x * (T)__popc(peers));
}

// Input already strictly increasing in the canonical key: copy it in canonical form.
__global__ void k_emit_sorted(const int32_t* __restrict__ du, const int32_t* __restrict__ dv,
                              const float* __restrict__ w_in, int64_t m, int32_t* __restrict__ u,
                              int32_t* __restrict__ v, float* __restrict__ w, int64_t* __restrict__ wu) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = du[e], b = dv[e];
        u[e] = min(a, b);
        v[e] = max(a, b);
        if (w_in) {
            const float x = w_in[e];
            w[e] = x;
            wu[e] = weight_units(x);
        }
    }
}

// Weighted degree in units (unit weights count 1 per edge) and unweighted degree.
// Degrees of the handle's graph, whose edges are sorted by their low end (canonical order,
// kept by pruning): a warp's low ends form runs of equal nodes, so each run adds its total
// with one atomic from its last lane (a segmented sum by shuffles, no match); the high ends
// are distinct within a run and take one atomic each.  T = int32 counts or u64 weight units.
template <class T>
__global__ void k_degrees_sorted(const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                                 const int64_t* __restrict__ wu, int64_t m, T* __restrict__ deg) {
    const unsigned lane = lane_id();
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = base + threadIdx.x;
        const bool ok = e < m;
        const int32_t a = ok ? u[e] : -1;
        const int32_t b = ok ? v[e] : -1;
        const T x = ok ? (wu ? (T)wu[e] : (T)1) : (T)0;
        if (ok) atomicAdd(&deg[b], x);
        // inclusive segmented sum over runs of equal a (runs are contiguous: u is sorted)
        T s = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, s, o);
            const int32_t ay = __shfl_up_sync(0xffffffffu, a, o);
            if ((int)lane >= o && ay == a) s += y;
        }
        const int32_t an = __shfl_down_sync(0xffffffffu, a, 1);
        if (ok && (lane == 31 || an != a)) atomicAdd(&deg[a], s);
    }
}

__global__ void k_max_i32(const int32_t* __restrict__ x, int64_t n, int32_t* __restrict__ out) {
    int32_t best = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        best = max(best, x[i]);
    best = __reduce_max_sync(0xffffffffu, best);
    if (lane_id() == 0) atomicMax(out, best);
}

__global__ void k_max_u64(const unsigned long long* __restrict__ x, int64_t n,
                          unsigned long long* __restrict__ out) {
    unsigned long long best = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        best = max(best, x[i]);
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane_id() == 0) atomicMax(out, best);
}

__global__ void k_iota(int32_t* __restrict__ x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = (int32_t)i;
}

__global__ void k_fill_i32(int32_t* __restrict__ x, int64_t n, int32_t val) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = val;
}

__device__ __forceinline__ bool below_bound(unsigned long long d, int64_t N, int64_t W) {
    // d * N < W, exactly (d < 2^63, N < 2^31, W < 2^63)
    unsigned __int128 lhs = (unsigned __int128)d * (unsigned __int128)(uint64_t)N;
    return lhs < (unsigned __int128)(uint64_t)W;
}

// Round r of Algorithm 2, node side: among the listed live nodes, mark every node whose
// current degree is below the density bound (its removal round, and its bit in the removed
// set); count them.  keep[i] = 1 for survivors.  Node ids are those of the current id space:
// orig maps them to the input's ids (null: the same ids).
__global__ void k_prune_mark(const int32_t* __restrict__ act, int64_t nact,
                             const unsigned long long* __restrict__ deg, int64_t N, int64_t W,
                             int32_t r, const int32_t* __restrict__ orig, int32_t* __restrict__ rr,
                             uint32_t* __restrict__ dead, int32_t* __restrict__ keep,
                             unsigned long long* __restrict__ removed) {
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nact;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = act[i];
        bool rem = below_bound(deg[x], N, W);
        if (rem) {
            rr[orig ? orig[x] : x] = r;
            atomicOr(&dead[x >> 5], 1u << (x & 31));
            ++c;
        }
        keep[i] = rem ? 0 : 1;
    }
    c = warp_sum(c);
    if (lane_id() == 0 && c) atomicAdd(removed, c);
}

// Round r, edge side: every live edge with an end removed in this round takes its weight
// off W(H) and off the degree of a surviving end; edges with both ends alive go to the next
// round's edge list (in any order: the list only drives the rounds).  The live list holds
// only edges whose ends were alive before this round, so an end is removed in this round
// exactly when its bit in the removed set is on (a 1-bit-per-node set: far fewer cache lines
// than the removal rounds).  A block takes tiles of kPruneTile edges and reserves room for a
// tile's survivors with one atomic; unit-weight decrements are aggregated per warp on equal
// nodes.  A round whose node side removed nothing writes nothing (the caller stops there).
//
// RELABEL (the first round): the survivors are written in a new id space, each surviving
// node numbered by its rank among the survivors (ascending ids, so runs of equal low ends
// stay together).  Each end then takes one 8-byte lookup of its word of the removed set with
// the count of surviving ids in the words before it.  After the first round few nodes
// survive on the graphs of the method's inputs (4.19 M -> 0.62 M on R-MAT scale 22), and the
// removed set of the later rounds, indexed by the new ids, stays in L1: the random lookups
// of the high ends that bound a round mostly hit there.
constexpr int kPruneItems = 8;
constexpr int kPruneTile = kT * kPruneItems;

// Surviving ids below x in the id space of the rank word p = (removed bits, survivors in the
// earlier words).
__device__ __forceinline__ int32_t rank_of(uint2 p, int32_t x) {
    return (int32_t)(p.y + (uint32_t)__popc(~p.x & ((1u << (x & 31)) - 1u)));
}

template <bool RELABEL>
__global__ void __launch_bounds__(kT, 4)
k_prune_edges(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
              const int64_t* __restrict__ ew, int64_t me, const uint32_t* __restrict__ dead,
              const uint2* __restrict__ rank_words, const unsigned long long* __restrict__ removed,
              unsigned long long* __restrict__ deg,
              unsigned long long* __restrict__ removedW,
              int32_t* __restrict__ nu, int32_t* __restrict__ nv,
              int64_t* __restrict__ nw, unsigned long long* __restrict__ ncount) {
    if (*removed == 0) return;   // the same value for every thread: no barrier is skipped
    __shared__ unsigned long long sh_base;
    __shared__ int32_t sh_warp[kT / 32];
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const int warp = (int)(threadIdx.x >> 5);
    unsigned long long acc = 0;
    for (int64_t tb = (int64_t)blockIdx.x * kPruneTile; tb < me; tb += (int64_t)gridDim.x * kPruneTile) {
        int32_t a[kPruneItems], b[kPruneItems];
        int64_t x[kPruneItems];
        unsigned keepm = 0;
        auto load = [&](int i) {
            const int64_t e = tb + (int64_t)i * kT + threadIdx.x;
            const bool ok = e < me;
            a[i] = ok ? eu[e] : -1;
            b[i] = ok ? ev[e] : -1;
            x[i] = ok ? (ew ? ew[e] : 1) : 0;
        };
        // later rounds (lookups mostly in L1): the tile's ends first, so that their loads
        // overlap; the first round keeps one item's loads at a time (its rank words need the
        // registers, and its random lookups set its pace)
        if (!RELABEL) {
#pragma unroll
            for (int i = 0; i < kPruneItems; ++i) load(i);
        }
#pragma unroll
        for (int i = 0; i < kPruneItems; ++i) {
            const int64_t e = tb + (int64_t)i * kT + threadIdx.x;
            const bool ok = e < me;
            if (RELABEL) load(i);
            bool ra, rb;
            int32_t na = 0, nb = 0;   // RELABEL: the ends' ids among the survivors
            if (RELABEL) {
                const uint2 pa = ok ? __ldg(rank_words + (a[i] >> 5)) : make_uint2(0u, 0u);
                const uint2 pb = ok ? __ldg(rank_words + (b[i] >> 5)) : make_uint2(0u, 0u);
                ra = (pa.x >> (a[i] & 31)) & 1u;
                rb = (pb.x >> (b[i] & 31)) & 1u;
                na = rank_of(pa, a[i]);
                nb = rank_of(pb, b[i]);
            } else {
                ra = ok && ((__ldg(dead + (a[i] >> 5)) >> (a[i] & 31)) & 1u);
                rb = ok && ((__ldg(dead + (b[i] >> 5)) >> (b[i] & 31)) & 1u);
            }
            if (ra || rb) acc += (unsigned long long)x[i];
            const int32_t da = (ok && rb && !ra) ? a[i] : -1;   // surviving end of a removed edge
            const int32_t db = (ok && ra && !rb) ? b[i] : -1;
            if (ew) {
                if (da >= 0) atomicAdd(&deg[da], (unsigned long long)(-x[i]));
                if (db >= 0) atomicAdd(&deg[db], (unsigned long long)(-x[i]));
            } else {
                warp_add<unsigned long long>(deg, da, ~0ull);   // -1 per edge, modulo 2^64
                warp_add<unsigned long long>(deg, db, ~0ull);
            }
            if (ok && !ra && !rb) keepm |= 1u << i;
            if (RELABEL) { a[i] = na; b[i] = nb; }   // only survivors are written below
        }
        // survivors: each warp writes item i of its lanes as one contiguous run (coalesced)
        unsigned bal[kPruneItems];
        int32_t wcnt = 0;
#pragma unroll
        for (int i = 0; i < kPruneItems; ++i) {
            bal[i] = __ballot_sync(0xffffffffu, (keepm >> i) & 1u);
            wcnt += __popc(bal[i]);
        }
        if (lane == 0) sh_warp[warp] = wcnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t t = 0;
            for (int w = 0; w < kT / 32; ++w) { const int32_t c = sh_warp[w]; sh_warp[w] = t; t += c; }
            sh_base = t ? atomicAdd(ncount, (unsigned long long)t) : 0ull;
        }
        __syncthreads();
        unsigned long long p = sh_base + (unsigned long long)sh_warp[warp];
        __syncthreads();   // sh_base and sh_warp are rewritten by the next tile
#pragma unroll
        for (int i = 0; i < kPruneItems; ++i) {
            if ((keepm >> i) & 1u) {
                const unsigned long long q = p + __popc(bal[i] & lt);
                nu[q] = a[i]; nv[q] = b[i];
                if (nw) nw[q] = x[i];
            }
            p += __popc(bal[i]);
        }
    }
    acc = warp_sum(acc);
    if (lane_id() == 0 && acc) atomicAdd(removedW, acc);
}

// Rank words of the first round's renumbering: surviving ids per word of the removed set
// (ids past the last node count too, but only the words before a word enter its rank), then,
// after their exclusive scan, each word with the survivors before it.
__global__ void k_word_alive(const uint32_t* __restrict__ dead, int64_t words, int32_t* __restrict__ cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x)
        cnt[i] = 32 - __popc(dead[i]);
}

__global__ void k_rank_words(const uint32_t* __restrict__ dead, const int32_t* __restrict__ pre, int64_t words,
                             uint2* __restrict__ rw) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x)
        rw[i] = make_uint2(dead[i], (uint32_t)pre[i]);
}

// The first round's survivors in the new id space: their degrees and their input ids.
__global__ void k_relabel_nodes(const uint2* __restrict__ rw, int32_t n,
                                const unsigned long long* __restrict__ deg,
                                unsigned long long* __restrict__ deg2, int32_t* __restrict__ orig) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = (int32_t)i;
        const uint2 p = rw[x >> 5];
        if (!((p.x >> (x & 31)) & 1u)) {
            const int32_t k = rank_of(p, x);
            deg2[k] = deg[x];
            orig[k] = x;
        }
    }
}

// Stable compaction of the live node list by flag, survivors renumbered by their rank words.
__global__ void k_compact_ranked(const int32_t* __restrict__ act, const int32_t* __restrict__ flag,
                                 const int32_t* __restrict__ pos, int64_t n, const uint2* __restrict__ rw,
                                 int32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) {
            const int32_t x = act[i];
            out[pos[i]] = rank_of(rw[x >> 5], x);
        }
}

// The removed set over the input's ids, from the removal rounds (one warp per word).
__global__ void k_dead_from_rounds(const int32_t* __restrict__ rr, int32_t n, uint32_t* __restrict__ dead) {
    const int64_t words = ((int64_t)n + 31) / 32;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < words; w += nw) {
        const int64_t x = w * 32 + lane_id();
        const unsigned bits = __ballot_sync(0xffffffffu, x < n && rr[x] >= 0);
        if (lane_id() == 0) dead[w] = bits;
    }
}

template <class T>
__global__ void k_compact_by_flag(const T* __restrict__ in, const int32_t* __restrict__ flag,
                                  const int32_t* __restrict__ pos, int64_t n, T* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) out[pos[i]] = in[i];
}

__global__ void k_keep_nodes(const int32_t* __restrict__ rr, int32_t n, int32_t* __restrict__ keep) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        keep[i] = rr[i] < 0 ? 1 : 0;
}

__global__ void k_node_map(const int32_t* __restrict__ keep, const int32_t* __restrict__ pos,
                           int32_t n, const int32_t* __restrict__ old_map, int32_t* __restrict__ map) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (keep[i]) map[pos[i]] = old_map ? old_map[i] : (int32_t)i;
}

// Stable compaction of G's edges to H (both ends alive), by tiles of kPruneTile edges in
// index order (item i of thread t is edge tile + i kT + t): the first pass counts each
// tile's survivors, a scan of the counts gives each tile's output start, and the second pass
// recomputes the survivors and writes them in index order, positions from per-(item, warp)
// ballots.
__device__ __forceinline__ bool node_dead(const uint32_t* __restrict__ dead, int32_t x) {
    return (__ldg(dead + (x >> 5)) >> (x & 31)) & 1u;
}

__global__ void __launch_bounds__(kT) k_tile_keep_counts(const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                                                         int64_t m, const uint32_t* __restrict__ dead,
                                                         int32_t* __restrict__ tcnt) {
    __shared__ int32_t sh[kT / 32];
    const int64_t tiles = (m + kPruneTile - 1) / kPruneTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        int32_t a[kPruneItems], b[kPruneItems];
#pragma unroll
        for (int i = 0; i < kPruneItems; ++i) {   // loads first, no branches between them
            const int64_t e = t * kPruneTile + (int64_t)i * kT + threadIdx.x;
            a[i] = e < m ? u[e] : 0;
            b[i] = e < m ? v[e] : 0;
        }
        int32_t c = 0;
#pragma unroll
        for (int i = 0; i < kPruneItems; ++i) {
            const int64_t e = t * kPruneTile + (int64_t)i * kT + threadIdx.x;
            c += (int32_t)((e < m) & !node_dead(dead, a[i]) & !node_dead(dead, b[i]));
        }
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane_id() == 0) sh[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t tot = 0;
            for (int w = 0; w < kT / 32; ++w) tot += sh[w];
            tcnt[t] = tot;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kT) k_tile_emit(const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                                                  const float* __restrict__ w, const int64_t* __restrict__ wu,
                                                  int64_t m, const uint32_t* __restrict__ dead,
                                                  const int32_t* __restrict__ tpos, const int32_t* __restrict__ npos,
                                                  int32_t* __restrict__ ou, int32_t* __restrict__ ov,
                                                  float* __restrict__ ow, int64_t* __restrict__ owu) {
    __shared__ int32_t pre[kPruneItems][kT / 32];
    const int warp = (int)(threadIdx.x >> 5);
    const unsigned lt = (1u << lane_id()) - 1u;
    const int64_t tiles = (m + kPruneTile - 1) / kPruneTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        int32_t a[kPruneItems], b[kPruneItems];
        unsigned bal[kPruneItems];
#pragma unroll
        for (int i = 0; i < kPruneItems; ++i) {   // loads first, no branches between them
            const int64_t e = t * kPruneTile + (int64_t)i * kT + threadIdx.x;
            a[i] = e < m ? u[e] : 0;
            b[i] = e < m ? v[e] : 0;
        }
#pragma unroll
        for (int i = 0; i < kPruneItems; ++i) {
            const int64_t e = t * kPruneTile + (int64_t)i * kT + threadIdx.x;
            const bool keep = (e < m) & !node_dead(dead, a[i]) & !node_dead(dead, b[i]);
            bal[i] = __ballot_sync(0xffffffffu, keep);
            if (lane_id() == 0) pre[i][warp] = __popc(bal[i]);
        }
        __syncthreads();
        if (threadIdx.x == 0) {   // exclusive prefix in index order: item-major, then warp
            int32_t run = 0;
            for (int i = 0; i < kPruneItems; ++i)
                for (int q = 0; q < kT / 32; ++q) { const int32_t c = pre[i][q]; pre[i][q] = run; run += c; }
        }
        __syncthreads();
        const int32_t base = tpos[t];
#pragma unroll
        for (int i = 0; i < kPruneItems; ++i) {
            if ((bal[i] >> lane_id()) & 1u) {
                const int64_t e = t * kPruneTile + (int64_t)i * kT + threadIdx.x;
                const int32_t p = base + pre[i][warp] + __popc(bal[i] & lt);
                ou[p] = npos[a[i]];
                ov[p] = npos[b[i]];
                if (w) { ow[p] = w[e]; owu[p] = wu[e]; }
            }
        }
        __syncthreads();   // pre is rewritten by the next tile
    }
}

inline unsigned grid_for(int64_t n) { return lowd_grid_for(n, kT); }

}  // namespace

size_t lowd_sort_tmp_bytes(int64_t n) {
    size_t a = radix_tmp_bytes(n);
    size_t b = scan_tmp_bytes<int64_t>(n) + 256;
    return a > b ? a : b;
}

// ------------------------------------------------------------------ load

lowd_status lowd_graph_load(lowd_ctx* h, const int32_t* du, const int32_t* dv, const float* dw,
                            int64_t m_in) {
    cudaStream_t st = h->st;
    const int32_t n = h->n0;
    h->weighted = dw != nullptr;
    uint64_t* keys[2] = {nullptr, nullptr};
    uint32_t* idx[2] = {nullptr, nullptr};
    int32_t* first = nullptr;
    int32_t* pos = nullptr;
    lowd_status s = LOWD_OK;
    auto cleanup = [&]() {
        dfree(h, &keys[0]); dfree(h, &keys[1]); dfree(h, &idx[0]); dfree(h, &idx[1]);
        dfree(h, &first); dfree(h, &pos);
    };
    do {
        if ((s = dalloc(h, &h->d_i32, 16))) break;
        if ((s = dalloc(h, &h->d_i64, 16))) break;
        if ((s = dalloc(h, &h->d_stats, 16))) break;
        if (cudaMallocHost(&h->h_pin, 16 * sizeof(int64_t)) != cudaSuccess) { s = h->fail(cudaErrorMemoryAllocation); break; }
        cudaMemsetAsync(h->d_i32, 0, 16 * sizeof(int32_t), st);
        if (m_in > 0) {   // checks only: keys are written only if the input needs sorting
            const bool a16 = ((uintptr_t)du & 15) == 0 && ((uintptr_t)dv & 15) == 0 && ((uintptr_t)dw & 15) == 0;
            if (a16)
                LOWD_LAUNCH(k_check_vec4, grid_for((m_in + 3) / 4), kT, 0, st, du, dv, dw, m_in, n, h->d_i32);
            else
                LOWD_LAUNCH(k_check_keys, grid_for(m_in), kT, 0, st, du, dv, dw, m_in, n, (uint64_t*)nullptr,
                            (uint32_t*)nullptr, h->d_i32);
        }
        if (cudaGetLastError() != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
        int32_t err = 0;
        if (cudaMemcpyAsync(&err, h->d_i32, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
        if (err & (ERR_RANGE | ERR_LOOP | ERR_WEIGHT)) {
            snprintf(h->err, sizeof(h->err), "%s%s%s", (err & ERR_RANGE) ? "node id out of range; " : "",
                     (err & ERR_LOOP) ? "self-loop; " : "", (err & ERR_WEIGHT) ? "non-positive or non-finite weight; " : "");
            s = LOWD_ERR_INVALID_ARG;
            break;
        }
        if ((err & ERR_GRID) && !(h->flags & LOWD_LOAD_ALLOW_INEXACT)) {
            snprintf(h->err, sizeof(h->err), "weight not a multiple of 2^-20");
            s = LOWD_ERR_INEXACT_WEIGHTS;
            break;
        }
        h->inexact = (err & ERR_GRID) ? 1 : 0;
        int cur = 0;
        int64_t m = m_in;
        const bool sorted = !(err & UNSORTED);
        if (!sorted && m_in > 1) {
            if ((s = dalloc(h, &keys[0], m_in))) break;
            if ((s = dalloc(h, &idx[0], m_in))) break;
            LOWD_LAUNCH(k_check_keys, grid_for(m_in), kT, 0, st, du, dv, dw, m_in, n, keys[0], idx[0], h->d_i32 + 6);
            if ((s = dalloc(h, &keys[1], m_in))) break;
            if ((s = dalloc(h, &idx[1], m_in))) break;
            if ((s = h->need_tmp(lowd_sort_tmp_bytes(m_in)))) break;
            int bits = bit_length_u64((uint64_t)n * (uint64_t)n - 1);
            cur = radix_sort_pairs<uint64_t, uint32_t>(keys[0], idx[0], keys[1], idx[1], m_in, bits, h->tmp, st);
            if ((s = dalloc(h, &first, m_in))) break;
            if ((s = dalloc(h, &pos, m_in))) break;
            LOWD_LAUNCH(k_first_flags, grid_for(m_in), kT, 0, st, keys[cur], m_in, first);
            scan_exclusive<int32_t>(first, pos, m_in, h->d_i32 + 1, h->tmp, st);
            int32_t mu = 0;
            if (cudaMemcpyAsync(&mu, h->d_i32 + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
            m = mu;
        }
        h->m0 = h->m = m;
        h->dup = m_in - m;
        h->n = n;
        if ((s = dalloc(h, &h->u, m))) break;
        if ((s = dalloc(h, &h->v, m))) break;
        if (h->weighted) {
            if ((s = dalloc(h, &h->w, m))) break;
            if ((s = dalloc(h, &h->wu, m))) break;
        }
        if (m_in > 0 && keys[0] == nullptr)   // already canonical order: a direct copy
            LOWD_LAUNCH(k_emit_sorted, grid_for(m_in), kT, 0, st, du, dv, dw, m_in, h->u, h->v, h->w, h->wu);
        else if (m_in > 0)
            LOWD_LAUNCH(k_emit_unique, grid_for(m_in), kT, 0, st, keys[cur], idx[cur], first, pos, m_in, n, dw,
                        h->u, h->v, h->w, h->wu);
        if (cudaGetLastError() != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
        h->max_deg = -1;   // computed when first needed (lowd_max_degree): pruning does not need G's
    } while (0);
    cleanup();
    return s;
}

int32_t lowd_max_degree(lowd_ctx* h) {
    if (h->max_deg < 0 && lowd_graph_max_degree(h) != LOWD_OK) return h->n > 0 ? h->n - 1 : 0;   // an upper bound
    return h->max_deg;
}

void lowd_degrees_i32(lowd_ctx* h, int32_t* deg) {
    cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)h->n, h->st);
    if (h->m > 0) LOWD_LAUNCH(k_degrees_sorted<int32_t>, grid_for(h->m), kT, 0, h->st, h->u, h->v, nullptr, h->m, deg);
}

lowd_status lowd_graph_max_degree(lowd_ctx* h) {
    cudaStream_t st = h->st;
    int32_t* cnt = nullptr;
    LOWD_TRY(dalloc(h, &cnt, h->n));
    cudaMemsetAsync(h->d_i32 + 2, 0, sizeof(int32_t), st);
    lowd_degrees_i32(h, cnt);
    LOWD_LAUNCH(k_max_i32, grid_for(h->n), kT, 0, st, cnt, h->n, h->d_i32 + 2);
    int32_t md = 0;
    cudaError_t e = cudaMemcpyAsync(&md, h->d_i32 + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(h, &cnt);
    if (e != cudaSuccess) return h->fail(e);
    h->max_deg = md;
    return LOWD_OK;
}

// ------------------------------------------------------------------ Algorithm 2

lowd_status lowd_graph_prune(lowd_ctx* h, int32_t* rounds_out) {
    cudaStream_t st = h->st;
    const int32_t n = h->n;
    const int64_t m = h->m;
    unsigned long long* deg = nullptr;
    uint64_t* dkey[2] = {nullptr, nullptr};
    int32_t* dval[2] = {nullptr, nullptr};
    int32_t *act = nullptr, *act2 = nullptr, *keep = nullptr, *pos = nullptr;
    int32_t *eu[2] = {nullptr, nullptr}, *ev[2] = {nullptr, nullptr};
    int64_t* ew[2] = {nullptr, nullptr};
    int32_t *keepe = nullptr, *epos = nullptr, *nmap = nullptr;
    uint32_t* dead = nullptr;   // nodes removed so far, one bit each
    uint2* rw = nullptr;        // rank words of the first round's renumbering
    int32_t *wcnt = nullptr, *wpre = nullptr, *orig = nullptr;
    unsigned long long* deg2 = nullptr;
    int32_t *nu = nullptr, *nv = nullptr;
    float* nw = nullptr;
    int64_t* nwu = nullptr;
    lowd_status s = LOWD_OK;
    auto cleanup = [&]() {
        dfree(h, &deg); dfree(h, &dkey[0]); dfree(h, &dkey[1]); dfree(h, &dval[0]); dfree(h, &dval[1]);
        dfree(h, &act); dfree(h, &act2); dfree(h, &keep); dfree(h, &pos);
        dfree(h, &eu[0]); dfree(h, &eu[1]); dfree(h, &ev[0]); dfree(h, &ev[1]); dfree(h, &ew[0]); dfree(h, &ew[1]);
        dfree(h, &keepe); dfree(h, &epos); dfree(h, &nmap); dfree(h, &dead); dfree(h, &nu); dfree(h, &nv); dfree(h, &nw); dfree(h, &nwu);
        dfree(h, &rw); dfree(h, &wcnt); dfree(h, &wpre); dfree(h, &orig); dfree(h, &deg2);
    };
    do {
        if ((s = dalloc(h, &deg, n))) break;
        if ((s = dalloc(h, &h->sort_perm, n))) break;
        if ((s = dalloc(h, &h->removal_round, n))) break;
        if ((s = h->need_tmp(lowd_sort_tmp_bytes(m > n ? m : n)))) break;
        cudaMemsetAsync(deg, 0, sizeof(unsigned long long) * (size_t)n, st);
        if (m > 0)
            LOWD_LAUNCH(k_degrees_sorted<unsigned long long>, grid_for(m), kT, 0, st, h->u, h->v, h->wu, m, deg);
        // W(G) = sum of degrees / 2 = sum of weights (units)
        unsigned long long* dmax = (unsigned long long*)(h->d_i64 + 0);
        cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), st);
        LOWD_LAUNCH(k_max_u64, grid_for(n), kT, 0, st, deg, n, dmax);
        // counting sort of nodes by degree (ascending, ties by id): LSD radix passes,
        // each a counting sort on one 8-bit digit of the degree
        if ((s = dalloc(h, &dkey[0], n))) break;
        if ((s = dalloc(h, &dkey[1], n))) break;
        if ((s = dalloc(h, &dval[0], n))) break;
        if ((s = dalloc(h, &dval[1], n))) break;
        cudaMemcpyAsync(dkey[0], deg, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
        LOWD_LAUNCH(k_iota, grid_for(n), kT, 0, st, dval[0], n);
        if (cudaMemcpyAsync(h->h_pin, dmax, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
        int bits = bit_length_u64((uint64_t)h->h_pin[0]);
        int cur = radix_sort_pairs<uint64_t, int32_t>(dkey[0], dval[0], dkey[1], dval[1], n, bits, h->tmp, st);
        cudaMemcpyAsync(h->sort_perm, dval[cur], sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
        LOWD_LAUNCH(k_fill_i32, grid_for(n), kT, 0, st, h->removal_round, n, -1);

        // total weight W(G)
        int64_t W = 0;
        if (h->wu) {
            // sum of units via the degree sum (each edge counted twice)
            int64_t* tot = h->d_i64 + 2;
            scan_exclusive<int64_t>((const int64_t*)deg, (int64_t*)dkey[1 - cur], n, tot, h->tmp, st);
            if (cudaMemcpyAsync(h->h_pin, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
            W = h->h_pin[0] / 2;
        } else {
            W = m;
        }
        int64_t N = n;
        if ((s = dalloc(h, &dead, ((size_t)n + 31) / 32))) break;
        cudaMemsetAsync(dead, 0, sizeof(uint32_t) * (((size_t)n + 31) / 32), st);

        // live node list (degree order) and live edge list
        if ((s = dalloc(h, &act, n))) break;
        if ((s = dalloc(h, &act2, n))) break;
        if ((s = dalloc(h, &keep, n))) break;
        if ((s = dalloc(h, &pos, n))) break;
        cudaMemcpyAsync(act, h->sort_perm, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
        int64_t nact = n;
        if ((s = dalloc(h, &eu[1], m))) break;
        if ((s = dalloc(h, &ev[1], m))) break;
        if (h->wu && (s = dalloc(h, &ew[1], m))) break;
        const int32_t* cu_ = h->u;
        const int32_t* cv_ = h->v;
        const int64_t* cw_ = h->wu;
        int64_t me = m;
        int nxt = 1;
        int32_t r = 0;
        unsigned long long* removed = (unsigned long long*)(h->d_i64 + 4);
        unsigned long long* removedW = (unsigned long long*)(h->d_i64 + 5);
        unsigned long long* ncount = (unsigned long long*)(h->d_i64 + 6);
        const int64_t Wn = ((int64_t)n + 31) / 32;   // words of the removed set over the input's ids
        if ((s = dalloc(h, &rw, Wn))) break;
        if ((s = dalloc(h, &wcnt, Wn))) break;
        if ((s = dalloc(h, &wpre, Wn))) break;
        while (N > 0) {
            int32_t rnext = r + 1;
            const bool relabel = r == 0;   // the first round renumbers its survivors
            cudaMemsetAsync(h->d_i64 + 4, 0, 3 * sizeof(int64_t), st);
            LOWD_LAUNCH(k_prune_mark, grid_for(nact), kT, 0, st, act, nact, deg, N, W, rnext, orig, h->removal_round,
                        dead, keep, removed);
            if (relabel) {
                LOWD_LAUNCH(k_word_alive, grid_for(Wn), kT, 0, st, dead, Wn, wcnt);
                scan_exclusive<int32_t>(wcnt, wpre, Wn, nullptr, h->tmp, st);
                LOWD_LAUNCH(k_rank_words, grid_for(Wn), kT, 0, st, dead, wpre, Wn, rw);
            }
            if (me > 0) {
                const unsigned ge = lowd_grid_for(me, kPruneTile, 4);
                if (relabel)
                    LOWD_LAUNCH(k_prune_edges<true>, ge, kT, 0, st, cu_, cv_, cw_, me, dead, rw, removed, deg,
                                removedW, eu[nxt], ev[nxt], ew[nxt], ncount);
                else
                    LOWD_LAUNCH(k_prune_edges<false>, ge, kT, 0, st, cu_, cv_, cw_, me, dead, rw, removed, deg,
                                removedW, eu[nxt], ev[nxt], ew[nxt], ncount);
            }
            if (cudaGetLastError() != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
            if (cudaMemcpyAsync(h->h_pin, h->d_i64 + 4, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
            int64_t k = h->h_pin[0];
            if (k == 0) break;  // the edge pass saw no removed end and kept every edge
            r = rnext;
            N -= k;
            W -= h->h_pin[1];
            cu_ = eu[nxt]; cv_ = ev[nxt]; cw_ = ew[nxt];
            me = h->h_pin[2];
            if (!eu[1 - nxt] && (s = dalloc(h, &eu[1 - nxt], m))) break;
            if (!ev[1 - nxt] && (s = dalloc(h, &ev[1 - nxt], m))) break;
            if (h->wu && !ew[1 - nxt] && (s = dalloc(h, &ew[1 - nxt], m))) break;
            nxt = 1 - nxt;
            // stable compaction of the live node list
            scan_exclusive<int32_t>(keep, pos, nact, h->d_i32 + 3, h->tmp, st);
            if (relabel) {
                // the survivors' degrees, input ids and live list in the new id space (the edge
                // list already carries the new ids); the removed set restarts there
                if ((s = dalloc(h, &deg2, N))) break;
                if ((s = dalloc(h, &orig, N))) break;
                LOWD_LAUNCH(k_relabel_nodes, grid_for(n), kT, 0, st, rw, n, deg, deg2, orig);
                dfree(h, &deg);
                deg = deg2;
                deg2 = nullptr;
                LOWD_LAUNCH(k_compact_ranked, grid_for(nact), kT, 0, st, act, keep, pos, nact, rw, act2);
                cudaMemsetAsync(dead, 0, sizeof(uint32_t) * (size_t)((N + 31) / 32), st);
            } else {
                LOWD_LAUNCH(k_compact_by_flag<int32_t>, grid_for(nact), kT, 0, st, act, keep, pos, nact, act2);
            }
            int32_t* t = act; act = act2; act2 = t;
            nact = N;
        }
        if (s) break;
        h->prune_rounds = r;
        // the removed set over the input's ids, for the compaction to H
        LOWD_LAUNCH(k_dead_from_rounds, lowd_grid_for(Wn, kT / 32), kT, 0, st, h->removal_round, n, dead);

        // compaction to H: survivors by ascending id, edges in original order (the live list
        // of the last round has exactly H's edges: me of them)
        const int64_t tiles = (m + kPruneTile - 1) / kPruneTile;
        if ((s = dalloc(h, &keepe, tiles))) break;   // survivors per tile
        if ((s = dalloc(h, &epos, tiles))) break;    // their output start
        if ((s = dalloc(h, &nmap, N))) break;
        LOWD_LAUNCH(k_keep_nodes, grid_for(n), kT, 0, st, h->removal_round, n, keep);
        scan_exclusive<int32_t>(keep, pos, n, nullptr, h->tmp, st);
        LOWD_LAUNCH(k_node_map, grid_for(n), kT, 0, st, keep, pos, n, h->map, nmap);
        const int64_t mH = me;
        if ((s = dalloc(h, &nu, mH))) break;
        if ((s = dalloc(h, &nv, mH))) break;
        if (h->w) {
            if ((s = dalloc(h, &nw, mH))) break;
            if ((s = dalloc(h, &nwu, mH))) break;
        }
        if (m > 0) {
            const unsigned gt = lowd_grid_for(m, kPruneTile, 4);
            LOWD_LAUNCH(k_tile_keep_counts, gt, kT, 0, st, h->u, h->v, m, dead, keepe);
            scan_exclusive<int32_t>(keepe, epos, tiles, nullptr, h->tmp, st);
            LOWD_LAUNCH(k_tile_emit, gt, kT, 0, st, h->u, h->v, h->w, h->wu, m, dead, epos, pos, nu, nv, nw, nwu);
        }
        if (cudaGetLastError() != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
        // swap in H
        dfree(h, &h->u); dfree(h, &h->v); dfree(h, &h->w); dfree(h, &h->wu); dfree(h, &h->map);
        h->u = nu; h->v = nv; h->w = nw; h->wu = nwu; h->map = nmap;
        nu = nv = nullptr; nw = nullptr; nwu = nullptr; nmap = nullptr;
        h->n = (int32_t)N;
        h->m = mH;
        h->pruned = 1;
        if (rounds_out) *rounds_out = r;
        s = lowd_graph_max_degree(h);
    } while (0);
    cleanup();
    return s;
}
