// Hub stars: a block update of Algorithm 1's objective over the edges between a hub and its
// low-degree neighbours.
//
// Sec. III-C shows that Algorithm 1's edge update is the exact minimiser of the sum of
// squared loads over one split with all other splits fixed, which is why sum l^2 falls
// monotonically.  The same holds for any block of splits whose exact minimiser is cheap.  A
// star (a hub h and leaves j_1..j_q, one edge each) is such a block: with B_h = l_h - sum t_j
// (t_j the hub's share of edge j) and B_j = l_j - (w_j - t_j) the loads without the star,
// the minimiser gives the hub the load lam solving
//     g(lam) = B_h + sum_j clip(B_j + w_j - lam, 0, w_j) - lam = 0
// and edge j the share t_j = clip(B_j + w_j - lam, 0, w_j) (water filling: every leaf whose
// share is not clipped ends at the hub's load).  A one-leaf star is Algorithm 1's update.
//
// Structure.  Nodes of (unweighted) degree >= tau are hubs; an edge with exactly one hub end
// is a star edge, every other edge is plain.  A leaf's star edges, ordered by hub degree
// (descending) then hub id, go to steps 0, 1, 2, ...; within a step the star edges of one
// hub form a star, and the stars of a step are vertex-disjoint (a leaf has one edge per
// step, hubs are never leaves).  A pass runs Algorithm 1 over the plain edges (their own
// schedule), then the steps in order, the stars of a step in parallel.  The automatic
// threshold depends on the schedule.  Schedule 1 (circle colouring: n - 1 classes whatever
// the stars take away) only needs the stars' faster descent, and the near-universal nodes
// give it with the fewest steps: the smallest power of two >= half the maximum degree.
// Schedule 2 (level order: at least the plain subgraph's maximum degree in classes) also
// needs the hubs' edges out of the plain subgraph: the smallest power of two 2^k (k >= 1)
// with at most 2^(k-1) nodes of degree >= 2^k.
//
// Execution.  One cooperative launch per pass runs every step; blocks take the stars of a
// step, one star per block at a time, and meet at a bounded grid barrier between steps
// (512-thread blocks, one per SM; 128-thread blocks, four per SM, when the steps average at
// least two stars per SM, as on unpruned graphs).  A
// block keeps up to kStarRegs edges per thread in registers (the rest of a large star in a
// scratch array) and solves g(lam) = 0 inside a shrinking bracket, by Newton steps and (when
// a Newton step leaves the bracket) Illinois secant steps (star_root); each evaluation of g
// is one block reduction.  The arithmetic is FP32 in the hub's frame and the loads move by
// error-free transfers of the split changes (see "Arithmetic" below), so loads and splits
// stay consistent; loads are kept as FP32 pairs (hi + lo) like in the pass kernels.
#include "ctx.cuh"
#include "prims.cuh"
#include "async.cuh"

#include <vector>

using namespace lowd;

namespace {

constexpr int kT = 256;
inline unsigned grid_for(int64_t n) { return lowd_grid_for(n, kT); }

// counts of nodes with degree >= 2^k, k = 0..30 (for the automatic threshold)
__global__ void k_degree_powers(const int32_t* __restrict__ deg, int32_t n, unsigned long long* __restrict__ cnt) {
    __shared__ unsigned long long c[32];
    if (threadIdx.x < 32) c[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = deg[i];
        for (int k = 0; k < 31 && d >= (1 << k); ++k) atomicAdd(&c[k], 1ull);
    }
    __syncthreads();
    if (threadIdx.x < 32 && c[threadIdx.x]) atomicAdd(&cnt[threadIdx.x], c[threadIdx.x]);
}

__global__ void k_star_flags(const int32_t* __restrict__ u, const int32_t* __restrict__ v, int64_t m,
                             const int32_t* __restrict__ deg, int32_t tau, int32_t* __restrict__ is_plain,
                             int32_t* __restrict__ is_star) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const bool ha = deg[u[e]] >= tau, hb = deg[v[e]] >= tau;
        is_star[e] = (ha != hb) ? 1 : 0;
        is_plain[e] = (ha != hb) ? 0 : 1;
    }
}

__global__ void k_select_ids(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos, int64_t m,
                             int32_t* __restrict__ ids) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        if (flag[e]) ids[pos[e]] = (int32_t)e;
}

__global__ void k_gather_ends(const int32_t* __restrict__ ids, int64_t k, const int32_t* __restrict__ u,
                              const int32_t* __restrict__ v, int32_t* __restrict__ su, int32_t* __restrict__ sv) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        su[i] = u[ids[i]];
        sv[i] = v[ids[i]];
    }
}

// sort keys of the star edges order[i]: which 0 = hub id, 1 = inverted hub degree, 2 = leaf
// id (three stable passes: leaf ascending, hub degree descending, hub id ascending)
__global__ void k_star_keys(const int32_t* __restrict__ order, int64_t k, const int32_t* __restrict__ u,
                            const int32_t* __restrict__ v, const int32_t* __restrict__ deg, int32_t tau, int which,
                            uint32_t* __restrict__ key) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = order[i];
        const bool ha = deg[u[e]] >= tau;
        const int32_t hub = ha ? u[e] : v[e], leaf = ha ? v[e] : u[e];
        key[i] = which == 0 ? (uint32_t)hub : (which == 1 ? 0x7fffffffu - (uint32_t)deg[hub] : (uint32_t)leaf);
    }
}

// step of each star edge = its rank among its leaf's star edges (leafkey sorted): key (step, hub)
__global__ void k_star_step_keys(const uint32_t* __restrict__ leafkey, const int32_t* __restrict__ order, int64_t k,
                                 const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                                 const int32_t* __restrict__ deg, int32_t tau, uint64_t* __restrict__ key) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = leafkey[i];
        int64_t lo = 0, hi = i;   // first entry of this leaf
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (leafkey[mid] < x) lo = mid + 1; else hi = mid;
        }
        const int32_t e = order[i];
        const int32_t hub = deg[u[e]] >= tau ? u[e] : v[e];
        key[i] = ((uint64_t)(i - lo) << 32) | (uint32_t)hub;
    }
}

__global__ void k_star_heads(const uint64_t* __restrict__ key, int64_t k, int32_t* __restrict__ head) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        head[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

// per star (segment of equal (step, hub) keys): its first position and hub; per step its
// first star
__global__ void k_star_segments(const uint64_t* __restrict__ key, const int32_t* __restrict__ head,
                                const int32_t* __restrict__ hpos, int64_t k, int32_t p0, int32_t* __restrict__ seg_beg,
                                int32_t* __restrict__ seg_hub, int32_t* __restrict__ step_seg) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        if (!head[i]) continue;
        const int32_t sg = hpos[i];
        seg_beg[sg] = p0 + (int32_t)i;
        seg_hub[sg] = (int32_t)(key[i] & 0xffffffffu);
        const uint32_t stp = (uint32_t)(key[i] >> 32);
        if (i == 0 || (uint32_t)(key[i - 1] >> 32) != stp) step_seg[stp] = sg;
    }
}

__global__ void k_set_i32(int32_t* __restrict__ x, int32_t val) { *x = val; }

// ------------------------------------------------------------------ the star steps
//
// Arithmetic.  FP64 runs at a small fraction of the FP32 rate on this GPU, so the star update
// works in FP32 in the frame of the hub's current load lh: per edge a_j = (l_j - lh) + t_j
// (= B_j + w_j - lh, the hub load at which the edge's share starts to fall) and the hub
// shares t_j; in that frame g(d) = sum_j (share_j(d) - t_j) - d with share_j(d) =
// clip(a_j - d, 0, w_j), d = lam - lh, whose terms are small near convergence.  The loads move
// by error-free transfers: with s the stored split f_e(a), every load change of the star is
// +-(s_new - s_old), split into an exact (hi, lo) pair by TwoSum, added to each leaf's pair
// and summed (pairwise, by TwoSum) into the hub's change, so a load stays the exact sum of
// what moved and the star conserves the total weight.

constexpr int kStarThreads = 512;               // block of the star steps: few stars per step
constexpr int kStarThreadsSmall = 128;          // many stars per step: more stars at once per SM
constexpr int kStarWarps = kStarThreads / 32;   // the most warps a block has
constexpr int kStarRegs = 8;       // edges per thread held in registers
constexpr int kStarNewton = 64;    // iteration cap of the root search (bracketed, so it always ends)

// where the ends and loads live: schedule 1 keeps packed 16-bit ends (lo | hi << 16) and the
// loads as two arrays (hi, lo); schedule 2 keeps int32 ends and the loads as float2 pairs
struct StarIO {
    const uint32_t* cuv;
    const int32_t* ea;
    const int32_t* eb;
    float* lhi;
    float* llo;
    float2* lp;
};

template <bool PACKED>
__device__ __forceinline__ void star_ends(const StarIO& io, int32_t p, int32_t& a, int32_t& b) {
    if (PACKED) {
        const uint32_t x = __ldg(io.cuv + p);
        a = (int32_t)(x & 0xffffu);
        b = (int32_t)(x >> 16);
    } else {
        a = __ldg(io.ea + p);
        b = __ldg(io.eb + p);
    }
}

template <bool PACKED>
__device__ __forceinline__ float2 star_load(const StarIO& io, int32_t x) {
    if (PACKED) return make_float2(__ldcg(io.lhi + x), __ldcg(io.llo + x));
    return __ldcg(io.lp + x);
}

template <bool PACKED>
__device__ __forceinline__ void star_store(const StarIO& io, int32_t x, float2 v) {
    if (PACKED) {
        __stcg(io.lhi + x, v.x);
        __stcg(io.llo + x, v.y);
    } else {
        __stcg(io.lp + x, v);
    }
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// x += (hi + lo), x a load pair: both parts by error-free transfers into x.x, errors to x.y
__device__ __forceinline__ void pair_add(float2& x, float hi, float lo) {
    float t, e;
    two_sum(x.x, hi, t, e);
    x.x = t;
    x.y += e + lo;
    two_sum(x.x, x.y, t, e);   // renormalise
    x.x = t;
    x.y = e;
}

// x += y for (hi, lo) pairs (TwoSum of the high parts, low parts added)
__device__ __forceinline__ void pair_acc(float& hi, float& lo, float yh, float yl) {
    float s, e;
    two_sum(hi, yh, s, e);
    hi = s;
    lo += e + yl;
}

// block-wide sums: NP (hi, lo) pairs (TwoSum at every addition), NF floats, NI ints; every
// thread gets the same totals, summed in the same order
template <int NP, int NF, int NI>
__device__ __forceinline__ void block_sum(float2 (&pp)[NP], float (&f)[NF], int (&k)[NI], float* shf, int* shi) {
    constexpr int NW = 2 * NP + NF;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const float h2 = __shfl_xor_sync(0xffffffffu, pp[i].x, o), l2 = __shfl_xor_sync(0xffffffffu, pp[i].y, o);
            pair_acc(pp[i].x, pp[i].y, h2, l2);
        }
#pragma unroll
        for (int i = 0; i < NF; ++i) f[i] += __shfl_xor_sync(0xffffffffu, f[i], o);
#pragma unroll
        for (int i = 0; i < NI; ++i) k[i] += __shfl_xor_sync(0xffffffffu, k[i], o);
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NP; ++i) { shf[NW * wid + 2 * i] = pp[i].x; shf[NW * wid + 2 * i + 1] = pp[i].y; }
#pragma unroll
        for (int i = 0; i < NF; ++i) shf[NW * wid + 2 * NP + i] = f[i];
#pragma unroll
        for (int i = 0; i < NI; ++i) shi[NI * wid + i] = k[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NP; ++i) pp[i] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int i = 0; i < NF; ++i) f[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < NI; ++i) k[i] = 0;
    const int nw = (int)(blockDim.x >> 5);
    for (int w = 0; w < nw; ++w) {
#pragma unroll
        for (int i = 0; i < NP; ++i) pair_acc(pp[i].x, pp[i].y, shf[NW * w + 2 * i], shf[NW * w + 2 * i + 1]);
#pragma unroll
        for (int i = 0; i < NF; ++i) f[i] += shf[NW * w + 2 * NP + i];
#pragma unroll
        for (int i = 0; i < NI; ++i) k[i] += shi[NI * w + i];
    }
}

// piece of g that edge (a, w) is on at d: 0 share clipped at 0, 1 interior, 2 clipped at w
__device__ __forceinline__ int piece(float a, float w, float d) { return d >= a ? 0 : (d <= a - w ? 2 : 1); }

__device__ __forceinline__ float share(float a, float w, float d) { return fminf(fmaxf(a - d, 0.0f), w); }

// the hub's share of an edge from the stored split s = f_e(a)
__device__ __forceinline__ float hub_share(bool ha, float s, float w) { return ha ? s : w - s; }

// the star's edges: registers first (a_j, old split, weight, side bit), then the scratch
// array (a_j, t_j) of large stars
template <bool WEIGHTED, int R>
struct StarEdges {
    const float* ra;
    const float* rs;
    const float* rw;
    unsigned rha;
    const float* cw;
    const float2* Bbuf;
    int32_t pr, p1, bbuf_p0, B;
    template <class F>
    __device__ __forceinline__ void each(F f) const {
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (rw[r] > 0.0f) f(ra[r], hub_share((rha >> r) & 1u, rs[r], rw[r]), rw[r]);
        for (int32_t p = pr + (int32_t)threadIdx.x; p < p1; p += B) {
            const float2 at = Bbuf[p - bbuf_p0];
            f(at.x, at.y, WEIGHTED ? __ldg(cw + p) : 1.0f);
        }
    }
};

// The root search in the frame of a reference hub load: g(d) = sum_j (share_j(d) - t_j) -
// off - d (off = the frame's offset from the hub's current load) is strictly decreasing and
// piecewise linear, with its root inside [lo, hi].  The bracket shrinks at every evaluation.
// The next point is a Newton step from the last point when it falls inside the bracket,
// else the secant of the bracket ends once both have been evaluated (Illinois: the g value
// of an end kept twice in a row is halved), else the midpoint.  Exact stops: a Newton step
// that stays on the piece it started from is the root; a bracket whose ends are on the same
// piece for every edge is linear, and its secant is the root.  Each evaluation is one block
// reduction; sums of the terms are compensated (hi, lo) pairs.
template <class Edges>
__device__ float star_root(const Edges& E, float lo, float hi, float off, float g0, int A0, float* shf, int* shi) {
    float glo = 0.0f, ghi = 0.0f;
    bool klo = false, khi = false;
    float x = 0.0f, gx = g0;
    int Ax = A0;
    if (gx == 0.0f) return 0.0f;
    if (gx > 0.0f) { lo = 0.0f; glo = gx; klo = true; } else { hi = 0.0f; ghi = gx; khi = true; }
    int Xb = 1, side = 0, stuck = 0;
    for (int it = 0; it < kStarNewton; ++it) {
        if (Xb == 0 && klo && khi)   // g is linear on [lo, hi]
            return glo == ghi ? lo : fminf(fmaxf(lo + glo * (hi - lo) / (glo - ghi), lo), hi);
        float y = x + gx / (1.0f + (float)Ax);
        const bool newton = y > lo && y < hi;
        if (!newton) {
            y = 0.5f * (lo + hi);
            if (klo && khi) {
                float a = glo, b = ghi;
                const float damp = ldexpf(1.0f, -stuck);
                if (side == 1) b *= damp;
                if (side == -1) a *= damp;
                const float ys = lo + a * (hi - lo) / (a - b);
                if (ys > lo && ys < hi) y = ys;
            }
            if (!(y > lo && y < hi)) return x;   // the bracket is down to adjacent floats
        }
        float2 G[1] = {make_float2(0.0f, 0.0f)};
        float fz[1] = {0.0f};
        int k[4] = {0, 0, 0, 0};
        E.each([&](float a, float t, float w) {
            float h, l;
            two_sum(share(a, w, y), -t, h, l);
            pair_acc(G[0].x, G[0].y, h, l);
            const int py = piece(a, w, y);
            k[0] += py == 1;
            k[1] += py != piece(a, w, x);
            k[2] += py != piece(a, w, lo);
            k[3] += py != piece(a, w, hi);
        });
        block_sum<1, 1, 4>(G, fz, k, shf, shi);
        const float gy = ((G[0].x - off) + G[0].y) - y;
        if (gy == 0.0f || (newton && k[1] == 0)) return y;
        if (gy > 0.0f) {
            lo = y; glo = gy; klo = true; Xb = k[3];
            stuck = side == 1 ? stuck + 1 : 1;
            side = 1;
        } else {
            hi = y; ghi = gy; khi = true; Xb = k[2];
            stuck = side == -1 ? stuck + 1 : 1;
            side = -1;
        }
        x = y;
        gx = gy;
        Ax = k[0];
    }
    return x;
}

// leaf update and the hub's share of it, for one edge: s_old -> s_new (stored split f_e(a))
template <bool PACKED>
__device__ __forceinline__ void star_apply(const StarIO& io, float* cs, int32_t p, bool ha, int32_t leaf,
                                           float s_old, float s_new, float& hub_hi, float& hub_lo) {
    float d, e;
    two_sum(s_new, -s_old, d, e);   // s_new - s_old = d + e exactly
    __stcg(cs + p, s_new);
    float2 L = star_load<PACKED>(io, leaf);
    // hub = a: the hub's share is s, the leaf's w - s; hub = b: the other way round
    pair_add(L, ha ? -d : d, ha ? -e : e);
    star_store<PACKED>(io, leaf, L);
    pair_acc(hub_hi, hub_lo, ha ? d : -d, ha ? e : -e);
}

// a_j = (l_j - frame) + t_j for a leaf load pair l_j and a frame pair
__device__ __forceinline__ float frame_level(float2 L, float2 F, float t) { return ((L.x - F.x) + (L.y - F.y)) + t; }

template <bool WEIGHTED, bool PACKED, int NT>
__global__ void __launch_bounds__(NT, NT == kStarThreads ? 1 : 4)
k_star_steps(int32_t S, const int32_t* __restrict__ step_seg, const int32_t* __restrict__ seg_beg,
             const int32_t* __restrict__ seg_hub, StarIO io, const float* __restrict__ cw, float* __restrict__ cs,
             float2* __restrict__ Bbuf, int32_t bbuf_p0, unsigned* __restrict__ bar, int32_t* __restrict__ err) {
    __shared__ float shf[6 * kStarWarps];
    __shared__ int shi[4 * kStarWarps];
    constexpr int R = kStarRegs;
    const int32_t B = (int32_t)blockDim.x;
    for (int32_t k = 0; k < S; ++k) {
        const int32_t g0 = __ldg(step_seg + k), g1 = __ldg(step_seg + k + 1);
        for (int32_t sg = g0 + (int32_t)blockIdx.x; sg < g1; sg += (int32_t)gridDim.x) {
            const int32_t h = __ldg(seg_hub + sg);
            const int32_t p0 = __ldg(seg_beg + sg), p1 = __ldg(seg_beg + sg + 1);
            const int32_t pr = p0 + R * B;   // positions from pr on go through the scratch array
            const float2 lh = star_load<PACKED>(io, h);
            // per edge: a_j (frame lh), old split, weight, leaf, side
            float ra[R], rw[R], rs[R];
            int32_t rl[R];
            unsigned rha = 0;
            float2 gp[1] = {make_float2(0.0f, 0.0f)};   // g(0) + 0, compensated
            float f2[2] = {0.0f, 0.0f};                 // T, W
            int k1[1] = {0};                            // interior edges at d = 0
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int32_t p = p0 + (int32_t)threadIdx.x + r * B;
                rw[r] = 0.0f;   // w = 0 marks an empty register slot (weights are > 0)
                ra[r] = 0.0f;
                rs[r] = 0.0f;
                rl[r] = -1;
                if (p < p1) {
                    int32_t a, b;
                    star_ends<PACKED>(io, p, a, b);
                    const float w = WEIGHTED ? __ldg(cw + p) : 1.0f;
                    const float sv = __ldcg(cs + p);
                    const bool ha = a == h;
                    const int32_t leaf = ha ? b : a;
                    const float t = hub_share(ha, sv, w);
                    ra[r] = frame_level(star_load<PACKED>(io, leaf), lh, t);
                    rw[r] = w;
                    rs[r] = sv;
                    rl[r] = leaf;
                    rha |= ha ? (1u << r) : 0u;
                    f2[0] += t;
                    f2[1] += w;
                    float hh, ll;
                    two_sum(share(ra[r], w, 0.0f), -t, hh, ll);
                    pair_acc(gp[0].x, gp[0].y, hh, ll);
                    k1[0] += piece(ra[r], w, 0.0f) == 1;
                }
            }
            for (int32_t p = pr + (int32_t)threadIdx.x; p < p1; p += B) {
                int32_t a, b;
                star_ends<PACKED>(io, p, a, b);
                const float w = WEIGHTED ? __ldg(cw + p) : 1.0f;
                const float sv = __ldcg(cs + p);
                const bool ha = a == h;
                const float t = hub_share(ha, sv, w);
                const float av = frame_level(star_load<PACKED>(io, ha ? b : a), lh, t);
                Bbuf[p - bbuf_p0] = make_float2(av, t);
                f2[0] += t;
                f2[1] += w;
                float hh, ll;
                two_sum(share(av, w, 0.0f), -t, hh, ll);
                pair_acc(gp[0].x, gp[0].y, hh, ll);
                k1[0] += piece(av, w, 0.0f) == 1;
            }
            block_sum<1, 2, 1>(gp, f2, k1, shf, shi);
            const float T = f2[0], W = f2[1];
            const float slack = 4e-6f * (T + W) + 1e-30f;
            const StarEdges<WEIGHTED, R> E{ra, rs, rw, rha, cw, Bbuf, pr, p1, bbuf_p0, B};
            float dl = star_root(E, -T - slack, W - T + slack, 0.0f, gp[0].x + gp[0].y, k1[0], shf, shi);
            // far from the current hub load, FP32 levels in lh's frame are too coarse: recentre
            // at lh + dl (the leaf levels are then small differences) and solve again
            if (fabsf(dl) > ldexpf(fabsf(lh.x), -12)) {
                float2 F = lh;
                pair_add(F, dl, 0.0f);
                gp[0] = make_float2(0.0f, 0.0f);
                k1[0] = 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (rl[r] >= 0) {
                        const float t = hub_share((rha >> r) & 1u, rs[r], rw[r]);
                        ra[r] = frame_level(star_load<PACKED>(io, rl[r]), F, t);
                        float hh, ll;
                        two_sum(share(ra[r], rw[r], 0.0f), -t, hh, ll);
                        pair_acc(gp[0].x, gp[0].y, hh, ll);
                        k1[0] += piece(ra[r], rw[r], 0.0f) == 1;
                    }
                }
                for (int32_t p = pr + (int32_t)threadIdx.x; p < p1; p += B) {
                    int32_t a, b;
                    star_ends<PACKED>(io, p, a, b);
                    const bool ha = a == h;
                    const float w = WEIGHTED ? __ldg(cw + p) : 1.0f;
                    const float t = Bbuf[p - bbuf_p0].y;
                    const float av = frame_level(star_load<PACKED>(io, ha ? b : a), F, t);
                    Bbuf[p - bbuf_p0] = make_float2(av, t);
                    float hh, ll;
                    two_sum(share(av, w, 0.0f), -t, hh, ll);
                    pair_acc(gp[0].x, gp[0].y, hh, ll);
                    k1[0] += piece(av, w, 0.0f) == 1;
                }
                float fz[2] = {0.0f, 0.0f};
                block_sum<1, 2, 1>(gp, fz, k1, shf, shi);
                const float g0 = ((gp[0].x - dl) + gp[0].y);
                const float sl2 = slack + 4e-6f * fabsf(dl);
                dl = star_root(E, -T - dl - sl2, W - T - dl + sl2, dl, g0, k1[0], shf, shi);
            }
            // new splits and the load changes they make
            float hub_hi = 0.0f, hub_lo = 0.0f;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (rl[r] >= 0) {
                    const int32_t p = p0 + (int32_t)threadIdx.x + r * B;
                    const bool ha = (rha >> r) & 1u;
                    const float t = share(ra[r], rw[r], dl);
                    const float s_new = fminf(fmaxf(ha ? t : rw[r] - t, 0.0f), rw[r]);
                    star_apply<PACKED>(io, cs, p, ha, rl[r], rs[r], s_new, hub_hi, hub_lo);
                }
            }
            for (int32_t p = pr + (int32_t)threadIdx.x; p < p1; p += B) {
                int32_t a, b;
                star_ends<PACKED>(io, p, a, b);
                const bool ha = a == h;
                const float w = WEIGHTED ? __ldg(cw + p) : 1.0f;
                const float sv = __ldcg(cs + p);
                const float t = share(Bbuf[p - bbuf_p0].x, w, dl);
                const float s_new = fminf(fmaxf(ha ? t : w - t, 0.0f), w);
                star_apply<PACKED>(io, cs, p, ha, ha ? b : a, sv, s_new, hub_hi, hub_lo);
            }
            float2 dh[1] = {make_float2(hub_hi, hub_lo)};
            float fz[1] = {0.0f};
            int kz[1] = {0};
            block_sum<1, 1, 1>(dh, fz, kz, shf, shi);
            if (threadIdx.x == 0) {
                float2 H = lh;
                pair_add(H, dh[0].x, dh[0].y);
                star_store<PACKED>(io, h, H);
            }
        }
        if (k + 1 < S && !grid_barrier(bar, bar + 1, gridDim.x, err)) return;
    }
}

}  // namespace

void StarSplit::release(lowd_ctx* h) {
    dfree(h, &dfull);
    dfree(h, &pid);
    dfree(h, &sid);
    dfree(h, &gu);
    dfree(h, &gv);
}

// Classify the edges of the current graph for hub stars (hub_tau: 1 automatic, >= 2 the
// threshold) for the given schedule.  With no star edge the split is released and reports all
// edges plain.
lowd_status lowd_star_split(lowd_ctx* h, int32_t hub_tau, int schedule, StarSplit* sp) {
    cudaStream_t st = h->st;
    const int64_t m = h->m;
    const int32_t n = h->n;
    *sp = StarSplit();
    sp->m_plain = m;
    if (hub_tau <= 0 || m == 0) return LOWD_OK;
    int32_t *fl[2] = {nullptr, nullptr}, *fp[2] = {nullptr, nullptr};
    unsigned long long* cnt = nullptr;
    lowd_status s = LOWD_OK;
    do {
        if ((s = h->need_tmp(lowd_sort_tmp_bytes(m + 2)))) break;
        if ((s = dalloc(h, &sp->dfull, n))) break;
        lowd_degrees_i32(h, sp->dfull);
        int32_t tau = hub_tau;
        if (tau == 1 && schedule == 1) {   // the near-universal nodes: degree >= ~max degree / 2
            int64_t p = 2;
            const int64_t dmax = lowd_max_degree(h);
            while (2 * p < dmax && p < (1 << 30)) p *= 2;
            tau = (int32_t)p;
        } else if (tau == 1) {
            if ((s = dalloc(h, &cnt, 32))) break;
            cudaMemsetAsync(cnt, 0, 32 * sizeof(unsigned long long), st);
            LOWD_LAUNCH(k_degree_powers, grid_for(n), kT, 0, st, sp->dfull, n, cnt);
            unsigned long long hc[32];
            cudaError_t e = cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { s = h->fail(e); break; }
            tau = 1 << 30;
            for (int k = 1; k < 31; ++k)
                if (hc[k] <= (1ull << (k - 1))) { tau = 1 << k; break; }
        }
        for (int i = 0; i < 2 && s == LOWD_OK; ++i) {
            if ((s = dalloc(h, &fl[i], m))) break;
            s = dalloc(h, &fp[i], m);
        }
        if (s) break;
        LOWD_LAUNCH(k_star_flags, grid_for(m), kT, 0, st, h->u, h->v, m, sp->dfull, tau, fl[0], fl[1]);
        scan_exclusive<int32_t>(fl[0], fp[0], m, h->d_i32 + 14, h->tmp, st);
        scan_exclusive<int32_t>(fl[1], fp[1], m, h->d_i32 + 15, h->tmp, st);
        int32_t cnts[2];
        cudaError_t e = cudaMemcpyAsync(cnts, h->d_i32 + 14, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { s = h->fail(e); break; }
        if (cnts[1] == 0) {   // no star edge: every edge is plain
            sp->release(h);
            sp->m_plain = m;
            break;
        }
        sp->tau = tau;
        sp->m_plain = cnts[0];
        sp->ms = cnts[1];
        if ((s = dalloc(h, &sp->pid, sp->m_plain))) break;
        if ((s = dalloc(h, &sp->sid, sp->ms))) break;
        if ((s = dalloc(h, &sp->gu, sp->m_plain))) break;
        if ((s = dalloc(h, &sp->gv, sp->m_plain))) break;
        LOWD_LAUNCH(k_select_ids, grid_for(m), kT, 0, st, fl[0], fp[0], m, sp->pid);
        LOWD_LAUNCH(k_select_ids, grid_for(m), kT, 0, st, fl[1], fp[1], m, sp->sid);
        if (sp->m_plain > 0)
            LOWD_LAUNCH(k_gather_ends, grid_for(sp->m_plain), kT, 0, st, sp->pid, sp->m_plain, h->u, h->v, sp->gu,
                        sp->gv);
        if (cudaGetLastError() != cudaSuccess) s = h->fail(cudaGetLastError());
    } while (0);
    for (int i = 0; i < 2; ++i) { dfree(h, &fl[i]); dfree(h, &fp[i]); }
    dfree(h, &cnt);
    if (s) sp->release(h);
    return s;
}

// The star steps of sp, placed at positions [p0, p0 + ms) of the class-major order: writes
// h->perm there (allocated by the caller), builds the step and star tables, and extends the
// exported class offsets (h->coff_real, C_plain + 1 entries over m_real_plain real positions)
// by one block per step.
lowd_status lowd_star_blocks(lowd_ctx* h, const StarSplit& sp, int64_t p0, int32_t C_plain, int64_t m_real_plain) {
    cudaStream_t st = h->st;
    const int64_t ms = sp.ms;
    const int32_t n = h->n;
    if (ms == 0) return LOWD_OK;
    uint32_t *sk0 = nullptr, *sk1 = nullptr;
    int32_t *so0 = nullptr, *so1 = nullptr, *head = nullptr, *hpos = nullptr, *cnew = nullptr;
    uint64_t *q0 = nullptr, *q1 = nullptr;
    lowd_status s = LOWD_OK;
    do {
        if ((s = h->need_tmp(lowd_sort_tmp_bytes(ms + 2)))) break;
        if ((s = dalloc(h, &sk0, ms)) || (s = dalloc(h, &sk1, ms)) || (s = dalloc(h, &so0, ms)) ||
            (s = dalloc(h, &so1, ms)) || (s = dalloc(h, &head, ms)) || (s = dalloc(h, &hpos, ms)) ||
            (s = dalloc(h, &q0, ms)) || (s = dalloc(h, &q1, ms)))
            break;
        cudaMemcpyAsync(so0, sp.sid, sizeof(int32_t) * (size_t)ms, cudaMemcpyDeviceToDevice, st);
        int32_t* cur_o = so0;
        int32_t* oth_o = so1;
        const int nbits = bit_length_u64((uint64_t)(n > 1 ? n - 1 : 1));
        for (int which = 0; which < 3; ++which) {   // hub, then hub degree (descending), then leaf
            LOWD_LAUNCH(k_star_keys, grid_for(ms), kT, 0, st, cur_o, ms, h->u, h->v, sp.dfull, sp.tau, which, sk0);
            const int c = radix_sort_pairs<uint32_t, int32_t>(sk0, cur_o, sk1, oth_o, ms, which == 1 ? 31 : nbits,
                                                             h->tmp, st);
            if (c) { int32_t* t = cur_o; cur_o = oth_o; oth_o = t; }
            if (which == 2 && c) { uint32_t* t = sk0; sk0 = sk1; sk1 = t; }   // leaf keys in sk0
        }
        LOWD_LAUNCH(k_star_step_keys, grid_for(ms), kT, 0, st, sk0, cur_o, ms, h->u, h->v, sp.dfull, sp.tau, q0);
        const int32_t dmax = lowd_max_degree(h);
        const int sbits = 32 + bit_length_u64((uint64_t)(dmax > 0 ? dmax : 1));   // step < max degree
        const int cq = radix_sort_pairs<uint64_t, int32_t>(q0, cur_o, q1, oth_o, ms, sbits, h->tmp, st);
        uint64_t* qk = cq ? q1 : q0;
        int32_t* qo = cq ? oth_o : cur_o;
        LOWD_LAUNCH(k_star_heads, grid_for(ms), kT, 0, st, qk, ms, head);
        scan_exclusive<int32_t>(head, hpos, ms, h->d_i32 + 14, h->tmp, st);
        int32_t NSg = 0;
        uint64_t lastkey = 0;
        cudaError_t e = cudaMemcpyAsync(&NSg, h->d_i32 + 14, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&lastkey, qk + ms - 1, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { s = h->fail(e); break; }
        const int32_t S = (int32_t)(lastkey >> 32) + 1;
        if ((s = dalloc(h, &h->star_seg_beg, (size_t)NSg + 1)) || (s = dalloc(h, &h->star_seg_hub, (size_t)NSg)) ||
            (s = dalloc(h, &h->star_step_seg, (size_t)S + 1)) || (s = dalloc(h, &h->star_bbuf, (size_t)ms)))
            break;
        LOWD_LAUNCH(k_star_segments, grid_for(ms), kT, 0, st, qk, head, hpos, ms, (int32_t)p0, h->star_seg_beg,
                    h->star_seg_hub, h->star_step_seg);
        LOWD_LAUNCH(k_set_i32, 1, 1, 0, st, h->star_seg_beg + NSg, (int32_t)(p0 + ms));
        LOWD_LAUNCH(k_set_i32, 1, 1, 0, st, h->star_step_seg + S, NSg);
        cudaMemcpyAsync(h->perm + p0, qo, sizeof(int32_t) * (size_t)ms, cudaMemcpyDeviceToDevice, st);
        std::vector<int32_t> hs((size_t)S + 1), hb((size_t)NSg + 1);
        e = cudaMemcpyAsync(hs.data(), h->star_step_seg, sizeof(int32_t) * hs.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hb.data(), h->star_seg_beg, sizeof(int32_t) * hb.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { s = h->fail(e); break; }
        int32_t maxseg = 0;
        for (int32_t k = 0; k < S; ++k) maxseg = hs[(size_t)k + 1] - hs[(size_t)k] > maxseg ? hs[(size_t)k + 1] - hs[(size_t)k] : maxseg;
        // exported class offsets: the plain classes, then one block per star step
        if ((s = dalloc(h, &cnew, (size_t)C_plain + S + 1))) break;
        cudaMemcpyAsync(cnew, h->coff_real, sizeof(int32_t) * ((size_t)C_plain + 1), cudaMemcpyDeviceToDevice, st);
        std::vector<int32_t> tail((size_t)S);
        for (int32_t k = 1; k <= S; ++k)
            tail[(size_t)k - 1] = (int32_t)(m_real_plain + (hb[(size_t)hs[(size_t)k]] - p0));
        cudaMemcpyAsync(cnew + C_plain + 1, tail.data(), sizeof(int32_t) * tail.size(), cudaMemcpyHostToDevice, st);
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { s = h->fail(e); break; }
        dfree(h, &h->coff_real);
        h->coff_real = cnew;
        cnew = nullptr;
        h->star_tau = sp.tau;
        h->star_S = S;
        h->star_nseg = NSg;
        h->star_m = ms;
        h->star_p0 = p0;
        h->star_maxseg = maxseg;
        if (cudaGetLastError() != cudaSuccess) s = h->fail(cudaGetLastError());
    } while (0);
    dfree(h, &sk0); dfree(h, &sk1); dfree(h, &so0); dfree(h, &so1); dfree(h, &head); dfree(h, &hpos); dfree(h, &q0); dfree(h, &q1);
    dfree(h, &cnew);
    return s;
}

// One pass's star steps (one cooperative launch).  The grid barrier words (d_i32[12..13])
// must be zero before the first launch of a run.
cudaError_t lowd_star_pass(lowd_ctx* h) {
    if (h->star_S <= 0) return cudaSuccess;
    const bool weighted = h->cw != nullptr;
    const bool packed = h->sched == 1;
    // many stars per step (unpruned graphs): small blocks, several stars at once per SM
    const int sms = lowd_device_sms();
    const bool small = (int64_t)h->star_nseg >= 2LL * sms * (int64_t)h->star_S;
    const int nt = small ? kStarThreadsSmall : kStarThreads;
    auto kern = small ? (weighted ? (packed ? k_star_steps<true, true, kStarThreadsSmall>
                                            : k_star_steps<true, false, kStarThreadsSmall>)
                                  : (packed ? k_star_steps<false, true, kStarThreadsSmall>
                                            : k_star_steps<false, false, kStarThreadsSmall>))
                      : (weighted ? (packed ? k_star_steps<true, true, kStarThreads>
                                            : k_star_steps<true, false, kStarThreads>)
                                  : (packed ? k_star_steps<false, true, kStarThreads>
                                            : k_star_steps<false, false, kStarThreads>));
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    const int cap = small ? 4 : 2;
    int blocks = sms * (per_sm < cap ? per_sm : cap);
    if (h->star_maxseg < blocks) blocks = h->star_maxseg > 0 ? h->star_maxseg : 1;
    StarIO io{};
    if (packed) {
        io.cuv = h->cuv;
        io.lhi = h->l;
        io.llo = h->l_lo;
    } else {
        io.ea = h->s2_ea;
        io.eb = h->s2_eb;
        io.lp = h->s2_lp;
    }
    int32_t S = h->star_S;
    const int32_t* ss = h->star_step_seg;
    const int32_t* sb = h->star_seg_beg;
    const int32_t* shb = h->star_seg_hub;
    const float* pcw = h->cw;
    float* pcs = h->cs;
    float2* pbb = h->star_bbuf;
    int32_t bp0 = (int32_t)h->star_p0;
    unsigned* bar = reinterpret_cast<unsigned*>(h->d_i32 + 12);
    int32_t* errp = h->d_i32 + 8;
    void* args[] = {&S, &ss, &sb, &shb, &io, &pcw, &pcs, &pbb, &bp0, &bar, &errp};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(nt), args, 0, h->st);
    lowd_note_launch();
    return e;
}

// ------------------------------------------------------------------ failure-detection self-test

namespace {

__global__ void k_barrier_selftest(unsigned* bar, unsigned nblocks, uint32_t spins, int32_t* err) {
    grid_barrier(bar, bar + 1, nblocks, err, spins);
}

}  // namespace

extern "C" lowd_status lowd_selftest_barrier_timeout(int32_t* err_bits) {
    if (!err_bits) return LOWD_ERR_INVALID_ARG;
    *err_bits = 0;
    unsigned* d = nullptr;
    if (cudaMalloc((void**)&d, 4 * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return LOWD_ERR_OUT_OF_MEMORY;
    }
    cudaError_t e = cudaMemset(d, 0, 4 * sizeof(unsigned));
    unsigned* bar = d;
    int32_t* err = reinterpret_cast<int32_t*>(d + 2);
    unsigned expected = 3;           // two blocks arrive: the barrier can never open
    uint32_t spins = 1u << 16;       // a short limit: the wait ends in milliseconds
    void* args[] = {&bar, &expected, &spins, &err};
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, dim3(2), dim3(32), args, 0, nullptr);
    lowd_note_launch();
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    int32_t v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, err, sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LOWD_ERR_CUDA;
    }
    *err_bits = v;
    return LOWD_OK;
}
