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
// Execution.  One CTA of 1024 threads keeps every node load in shared memory for all
// passes of a call and streams the edges of each class (packed 16-bit endpoint pairs
// when n <= 65536, the FP32 split and, if weighted, the FP32 weight), prefetching the
// next class's edges into registers while the current class is updated; __syncthreads
// separates classes.  The split of edge e = (lo, hi) is stored once, s_e = f_e(lo);
// f_e(hi) = w_e - s_e (the tighter dual's equality f_e(u) + f_e(v) = w_e, Sec. III-B).
#include "ctx.cuh"
#include "prims.cuh"

using namespace lowd;

namespace {

constexpr int kT = 256;
constexpr int kCtaThreads = 1024;
constexpr int kPre = 2;  // edges per thread prefetched for the next class

inline unsigned grid_for(int64_t n) {
    int64_t b = (n + kT - 1) / kT;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (unsigned)b;
}

__global__ void k_circle_colour(const int32_t* __restrict__ u, const int32_t* __restrict__ v, int64_t m,
                                int32_t n, uint32_t* __restrict__ key, int32_t* __restrict__ val) {
    const uint32_t Np = (uint32_t)(n + (n & 1));
    const uint32_t P = Np - 1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t a = (uint32_t)u[e], b = (uint32_t)v[e];
        uint32_t c = (b == Np - 1) ? (2u * a) % P : (a + b) % P;
        key[e] = c;
        val[e] = (int32_t)e;
    }
}

__global__ void k_class_heads(const uint32_t* __restrict__ key, int64_t m, int32_t* __restrict__ head) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        head[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

__global__ void k_class_offsets(const int32_t* __restrict__ head, const int32_t* __restrict__ hpos,
                                int64_t m, int32_t C, int32_t* __restrict__ coff) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        if (head[i]) coff[hpos[i]] = (int32_t)i;
    if (blockIdx.x == 0 && threadIdx.x == 0) coff[C] = (int32_t)m;
}

// Gather the class-major streams: endpoints (packed or not), weights, initial splits.
__global__ void k_gather_streams(const int32_t* __restrict__ perm, int64_t m,
                                 const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                                 const float* __restrict__ w, const float* __restrict__ s_init,
                                 uint32_t* __restrict__ cuv, int32_t* __restrict__ cu,
                                 int32_t* __restrict__ cv, float* __restrict__ cw,
                                 float* __restrict__ cs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t e = perm[i];
        int32_t a = u[e], b = v[e];
        if (cuv) cuv[i] = (uint32_t)a | ((uint32_t)b << 16);
        else { cu[i] = a; cv[i] = b; }
        float we = w ? w[e] : 1.0f;
        if (cw) cw[i] = we;
        float s = s_init ? fminf(fmaxf(s_init[e], 0.0f), we) : we * 0.5f;  // Alg. 1: w_e / 2
        cs[i] = s;
    }
}

// FP64 loads from the splits: l_x = sum over edges at x of f_e(x).
__global__ void k_rederive(int64_t m, const uint32_t* __restrict__ cuv, const int32_t* __restrict__ cu,
                           const int32_t* __restrict__ cv, const float* __restrict__ cw,
                           const float* __restrict__ cs, double* __restrict__ L64) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t a, b;
        if (cuv) { uint32_t p = cuv[i]; a = (int32_t)(p & 0xffffu); b = (int32_t)(p >> 16); }
        else { a = cu[i]; b = cv[i]; }
        double s = (double)cs[i];
        double w = cw ? (double)cw[i] : 1.0;
        atomicAdd(&L64[a], s);
        atomicAdd(&L64[b], w - s);
    }
}

// l = (float) L64; stats[0] += sum l, stats[1] += sum l^2, stats[2] = max l (FP64)
__global__ void k_load_stats(const double* __restrict__ L64, int32_t n, float* __restrict__ l,
                             double* __restrict__ stats) {
    __shared__ double sh[kT / 32 + 1];
    double s1 = 0.0, s2 = 0.0, mx = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double x = L64[i];
        if (l) l[i] = (float)x;
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

__global__ void k_splits_from_canonical(const int32_t* __restrict__ perm, int64_t m,
                                        const float* __restrict__ in, float* __restrict__ cs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        cs[i] = in[perm[i]];
}

__global__ void k_splits_to_canonical(const int32_t* __restrict__ perm, int64_t m,
                                      const float* __restrict__ cs, float* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        out[perm[i]] = cs[i];
}

struct EdgeReg {
    int32_t a, b;
    float s, w;
};

template <bool PACKED, bool WEIGHTED>
__device__ __forceinline__ EdgeReg load_edge(int64_t i, const uint32_t* __restrict__ cuv,
                                             const int32_t* __restrict__ cu, const int32_t* __restrict__ cv,
                                             const float* __restrict__ cw, const float* __restrict__ cs) {
    EdgeReg r;
    if (PACKED) { uint32_t p = __ldg(cuv + i); r.a = (int32_t)(p & 0xffffu); r.b = (int32_t)(p >> 16); }
    else { r.a = __ldg(cu + i); r.b = __ldg(cv + i); }
    r.w = WEIGHTED ? __ldg(cw + i) : 1.0f;
    r.s = cs[i];
    return r;
}

// The LOWD edge update of Algorithm 1 on e = (a, b) with f_e(a) = s, f_e(b) = w - s.
__device__ __forceinline__ void lowd_edge(float* L, EdgeReg& r) {
    float la = L[r.a], lb = L[r.b];
    float d;
    if (la > lb) {
        d = fminf((la - lb) * 0.5f, r.s);
        la -= d; lb += d;
        r.s -= d;
    } else {
        d = fminf((lb - la) * 0.5f, r.w - r.s);
        la += d; lb -= d;
        r.s = fminf(r.s + d, r.w);
    }
    L[r.a] = la; L[r.b] = lb;
}

template <bool PACKED, bool WEIGHTED>
__global__ void __launch_bounds__(kCtaThreads, 1)
k_sweep_cta(int32_t n, int32_t C, const int32_t* __restrict__ coff,
            const uint32_t* __restrict__ cuv, const int32_t* __restrict__ cu,
            const int32_t* __restrict__ cv, const float* __restrict__ cw,
            float* __restrict__ cs, float* __restrict__ l, int32_t passes) {
    extern __shared__ float L[];
    const int tid = threadIdx.x;
    for (int i = tid; i < n; i += kCtaThreads) L[i] = l[i];
    __syncthreads();
    for (int32_t t = 0; t < passes; ++t) {
        int32_t beg = __ldg(coff);
        int32_t end = C > 0 ? __ldg(coff + 1) : beg;
        // registers for the current class
        EdgeReg cur[kPre];
#pragma unroll
        for (int k = 0; k < kPre; ++k) {
            int64_t i = (int64_t)beg + tid + (int64_t)k * kCtaThreads;
            if (i < end) cur[k] = load_edge<PACKED, WEIGHTED>(i, cuv, cu, cv, cw, cs);
        }
        for (int32_t c = 0; c < C; ++c) {
            // prefetch the next class
            int32_t nb = end, ne = (c + 2 <= C) ? __ldg(coff + c + 2) : end;
            EdgeReg nxt[kPre];
#pragma unroll
            for (int k = 0; k < kPre; ++k) {
                int64_t i = (int64_t)nb + tid + (int64_t)k * kCtaThreads;
                if (c + 1 < C && i < ne) nxt[k] = load_edge<PACKED, WEIGHTED>(i, cuv, cu, cv, cw, cs);
            }
#pragma unroll
            for (int k = 0; k < kPre; ++k) {
                int64_t i = (int64_t)beg + tid + (int64_t)k * kCtaThreads;
                if (i < end) {
                    lowd_edge(L, cur[k]);
                    cs[i] = cur[k].s;
                }
            }
            // classes larger than the prefetch window
            for (int64_t i = (int64_t)beg + tid + (int64_t)kPre * kCtaThreads; i < end; i += kCtaThreads) {
                EdgeReg r = load_edge<PACKED, WEIGHTED>(i, cuv, cu, cv, cw, cs);
                lowd_edge(L, r);
                cs[i] = r.s;
            }
            __syncthreads();
            beg = nb; end = ne;
#pragma unroll
            for (int k = 0; k < kPre; ++k) cur[k] = nxt[k];
        }
    }
    for (int i = tid; i < n; i += kCtaThreads) l[i] = L[i];
}


// Deep-pipelined form of the same sweep.  The classes of all passes form one stream
// q = 0, 1, ... (class q mod C); each thread owns position `tid` of every class and keeps
// the edge data of the next kRing classes of the stream in a register ring, so a global
// load is issued kRing classes (several hundred cycles) before its use.  The class
// offsets live in shared memory when they fit next to the loads.  The load for class
// q + kRing is issued after class q is updated, so when a class comes round again in the
// next pass (C >= kRing) its split was already written by the same thread.  Positions
// past blockDim.x in a class are updated directly from global memory.
constexpr int kRing = 8;

template <bool WEIGHTED>
__device__ __forceinline__ void ring_issue(int32_t cls, bool ok, const int32_t* CO, int tid,
                                           const uint32_t* __restrict__ cuv, const float* __restrict__ cw,
                                           const float* __restrict__ cs, int32_t& si, uint32_t& suv,
                                           float& ss, float& sw) {
    si = -1;
    if (ok) {
        int32_t i = CO[cls] + tid;
        if (i < CO[cls + 1]) {
            si = i;
            suv = __ldg(cuv + i);
            ss = __ldcg(cs + i);
            if (WEIGHTED) sw = __ldg(cw + i);
        }
    }
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(kCtaThreads, 1)
k_sweep_ring(int32_t n, int32_t C, const int32_t* __restrict__ coff, int32_t co_smem,
             const uint32_t* __restrict__ cuv, const float* __restrict__ cw,
             float* __restrict__ cs, float* __restrict__ l, int32_t passes) {
    extern __shared__ float L[];
    int32_t* COs = reinterpret_cast<int32_t*>(L + n);
    const int tid = threadIdx.x;
    const int B = blockDim.x;
    for (int i = tid; i < n; i += B) L[i] = l[i];
    if (co_smem)
        for (int i = tid; i <= C; i += B) COs[i] = coff[i];
    __syncthreads();
    const int32_t* CO = co_smem ? COs : coff;
    const int64_t Q = (int64_t)C * passes;
    int32_t si[kRing];
    uint32_t suv[kRing];
    float ss[kRing], sw[kRing];
    int32_t c_issue = 0;
    int64_t q_issue = 0;
#pragma unroll
    for (int j = 0; j < kRing; ++j) {
        ring_issue<WEIGHTED>(c_issue, q_issue < Q, CO, tid, cuv, cw, cs, si[j], suv[j], ss[j], sw[j]);
        c_issue = (c_issue + 1 == C) ? 0 : c_issue + 1;
        ++q_issue;
    }
    int32_t c = 0;
    for (int64_t q0 = 0; q0 < Q; q0 += kRing) {
#pragma unroll
        for (int j = 0; j < kRing; ++j) {
            if (q0 + j < Q) {
                if (si[j] >= 0) {
                    EdgeReg r;
                    r.a = (int32_t)(suv[j] & 0xffffu);
                    r.b = (int32_t)(suv[j] >> 16);
                    r.s = ss[j];
                    r.w = WEIGHTED ? sw[j] : 1.0f;
                    lowd_edge(L, r);
                    __stcg(cs + si[j], r.s);
                }
                const int32_t end = CO[c + 1];
                for (int32_t i = CO[c] + B + tid; i < end; i += B) {
                    EdgeReg r = load_edge<true, WEIGHTED>(i, cuv, nullptr, nullptr, cw, cs);
                    lowd_edge(L, r);
                    cs[i] = r.s;
                }
                ring_issue<WEIGHTED>(c_issue, q_issue < Q, CO, tid, cuv, cw, cs, si[j], suv[j], ss[j], sw[j]);
                c_issue = (c_issue + 1 == C) ? 0 : c_issue + 1;
                ++q_issue;
                c = (c + 1 == C) ? 0 : c + 1;
                __syncthreads();
            }
        }
    }
    for (int i = tid; i < n; i += B) l[i] = L[i];
}

template <bool WEIGHTED>
cudaError_t launch_ring(lowd_ctx* h, int32_t passes) {
    const size_t lbytes = sizeof(float) * (size_t)h->n;
    const size_t cbytes = sizeof(int32_t) * ((size_t)h->C + 1);
    const size_t budget = 227 * 1024;
    const int co_smem = lbytes + cbytes <= budget ? 1 : 0;
    const size_t smem = lbytes + (co_smem ? cbytes : 0);
    int32_t maxc = 0;
    for (int32_t c = 0; c < h->C; ++c) maxc = max(maxc, h->coff_h[c + 1] - h->coff_h[c]);
    int threads = ((maxc + 31) / 32) * 32;
    if (threads < 128) threads = 128;
    if (threads > kCtaThreads) threads = kCtaThreads;
    auto kern = k_sweep_ring<WEIGHTED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    LOWD_LAUNCH(kern, 1, threads, smem, h->st, h->n, h->C, h->coff, co_smem, h->cuv, h->cw, h->cs, h->l,
                passes);
    return cudaGetLastError();
}

template <bool PACKED, bool WEIGHTED>
cudaError_t launch_cta(lowd_ctx* h, int32_t passes) {
    size_t smem = sizeof(float) * (size_t)(h->n > 0 ? h->n : 1);
    auto kern = k_sweep_cta<PACKED, WEIGHTED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    LOWD_LAUNCH(kern, 1, kCtaThreads, smem, h->st, h->n, h->C, h->coff, h->cuv, h->cu, h->cv, h->cw, h->cs, h->l, passes);
    return cudaGetLastError();
}

cudaError_t run_passes(lowd_ctx* h, int32_t passes) {
    if (passes <= 0 || h->m == 0) return cudaSuccess;
    const bool packed = h->cuv != nullptr;
    const bool weighted = h->cw != nullptr;
    if (packed && h->C >= kRing) return weighted ? launch_ring<true>(h, passes) : launch_ring<false>(h, passes);
    if (packed && weighted) return launch_cta<true, true>(h, passes);
    if (packed) return launch_cta<true, false>(h, passes);
    if (weighted) return launch_cta<false, true>(h, passes);
    return launch_cta<false, false>(h, passes);
}

}  // namespace

// Build the schedule and the class-major streams, then initialise the splits (equal
// split, or the given canonical-order splits) and the loads.
lowd_status lowd_sweep_prepare(lowd_ctx* h, int schedule_req, const float* init_splits_canon) {
    cudaStream_t st = h->st;
    const int64_t m = h->m;
    const int32_t n = h->n;
    if (schedule_req == 2) return LOWD_ERR_TOO_LARGE;  // grid schedule not available in this build
    if (n > LOWD_SMEM_NODES) {
        snprintf(h->err, sizeof(h->err), "current graph has %d nodes; the shared-memory sweep holds at most %d",
                 n, LOWD_SMEM_NODES);
        return LOWD_ERR_TOO_LARGE;
    }
    uint32_t* key[2] = {nullptr, nullptr};
    int32_t* val[2] = {nullptr, nullptr};
    int32_t *head = nullptr, *hpos = nullptr;
    lowd_status s = LOWD_OK;
    auto cleanup = [&]() { dfree(&key[0]); dfree(&key[1]); dfree(&val[0]); dfree(&val[1]); dfree(&head); dfree(&hpos); };
    do {
        if ((s = h->need_tmp(lowd_sort_tmp_bytes(m > n ? m : n)))) break;
        if ((s = dalloc(h, &key[0], m))) break;
        if ((s = dalloc(h, &key[1], m))) break;
        if ((s = dalloc(h, &val[0], m))) break;
        if ((s = dalloc(h, &val[1], m))) break;
        if ((s = dalloc(h, &head, m))) break;
        if ((s = dalloc(h, &hpos, m))) break;
        int32_t C = 0;
        int cur = 0;
        if (m > 0) {
            LOWD_LAUNCH(k_circle_colour, grid_for(m), kT, 0, st, h->u, h->v, m, n, key[0], val[0]);
            const uint32_t P = (uint32_t)(n + (n & 1)) - 1u;
            int bits = bit_length_u64(P > 0 ? P - 1 : 0);
            if (bits < 1) bits = 1;
            cur = radix_sort_pairs<uint32_t, int32_t>(key[0], val[0], key[1], val[1], m, bits, h->tmp, st);
            LOWD_LAUNCH(k_class_heads, grid_for(m), kT, 0, st, key[cur], m, head);
            scan_exclusive<int32_t>(head, hpos, m, h->d_i32 + 5, h->tmp, st);
            if (cudaMemcpyAsync(h->h_pin, h->d_i32 + 5, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
            C = *(int32_t*)h->h_pin;
        }
        h->C = C;
        if ((s = dalloc(h, &h->coff, (size_t)C + 1))) break;
        if (m > 0) LOWD_LAUNCH(k_class_offsets, grid_for(m), kT, 0, st, head, hpos, m, C, h->coff);
        else cudaMemsetAsync(h->coff, 0, sizeof(int32_t), st);
        h->coff_h = (int32_t*)malloc(sizeof(int32_t) * ((size_t)C + 1));
        if (!h->coff_h) { s = LOWD_ERR_OUT_OF_MEMORY; break; }
        if (cudaMemcpyAsync(h->coff_h, h->coff, sizeof(int32_t) * ((size_t)C + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            { s = h->fail(cudaGetLastError()); break; }
        // the class-major permutation
        h->perm = val[cur];
        val[cur] = nullptr;
        if (n <= 65536) { if ((s = dalloc(h, &h->cuv, m))) break; }
        else {
            if ((s = dalloc(h, &h->cu, m))) break;
            if ((s = dalloc(h, &h->cv, m))) break;
        }
        if (h->w && (s = dalloc(h, &h->cw, m))) break;
        if ((s = dalloc(h, &h->cs, m))) break;
        if ((s = dalloc(h, &h->l, n))) break;
        if (m > 0)
            LOWD_LAUNCH(k_gather_streams, grid_for(m), kT, 0, st, h->perm, m, h->u, h->v, h->w, init_splits_canon,
                                                         h->cuv, h->cu, h->cv, h->cw, h->cs);
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
    if (h->m > 0) LOWD_LAUNCH(k_rederive, grid_for(h->m), kT, 0, st, h->m, h->cuv, h->cu, h->cv, h->cw, h->cs, L64);
    LOWD_LAUNCH(k_load_stats, grid_for(h->n), kT, 0, st, L64, h->n, h->l, h->d_stats);
    double tmp3[3];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp3, h->d_stats, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(&L64);
    if (e != cudaSuccess) return h->fail(e);
    if (stats3) { stats3[0] = tmp3[0]; stats3[1] = tmp3[1]; stats3[2] = tmp3[2]; }
    return LOWD_OK;
}

lowd_status lowd_sweep_splits_canonical(lowd_ctx* h, float* out_dev) {
    if (h->m > 0) LOWD_LAUNCH(k_splits_to_canonical, grid_for(h->m), kT, 0, h->st, h->perm, h->m, h->cs, out_dev);
    LOWD_CK_LAUNCH();
    return LOWD_OK;
}

lowd_status lowd_sweep_load_canonical(lowd_ctx* h, const float* splits_dev) {
    if (h->m > 0) LOWD_LAUNCH(k_splits_from_canonical, grid_for(h->m), kT, 0, h->st, h->perm, h->m, splits_dev, h->cs);
    LOWD_CK_LAUNCH();
    return LOWD_OK;
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
    while (done < k) {
        int32_t step = k - done;
        if (o.check_every > 0 && o.check_every < step) step = o.check_every;
        LOWD_CK(run_passes(h, step));
        done += step;
        h->iters += step;
        if (o.check_every > 0) {
            LOWD_TRY(lowd_sweep_rederive(h, st3));
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
