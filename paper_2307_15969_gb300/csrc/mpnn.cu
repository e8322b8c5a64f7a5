// Learned warm start for Algorithm 1: a mean-aggregation message-passing network that
// predicts each edge's initial split.  The paper starts every edge at the equal split
// f_e(u) = f_e(v) = w_e / 2 (Alg. 1, initialisation); any split inside [0, w_e] is a valid
// start and the passes still converge to the same loads (Theorem 2 does not depend on the
// start), so the network only changes how far the first pass is from the optimum.
//
// Network (H = 64, three message-passing layers) on an undirected graph, edges (lo, hi):
//   x_v   = (log(1 + d_v), mean log w over v's edges, log(1 + sum of the neighbours' d))
//   h0    = relu(x W_in + b_in)
//   layer m_v = mean of h over v's neighbours;  h' = relu([h, m] W_l^T + b_l)
//   phi_v = q . h3_v;  sigma_e = 1 / (1 + exp(phi_hi - phi_lo));  f_e(lo) = sigma_e w_e
// Training loss: sum_v (l_v - t_v)^2 / sum_v t_v^2 against target loads t (converged
// LOWD loads), l_v the loads the predicted splits give.
//
// Precision: master parameters, gradients and Adam moments FP32; node states h and means m
// stored BF16; the layer products [h, m] W_l^T (forward) and dA W_l (backward, dA rounded
// to BF16) run on the tensor cores (tcgen05, BF16 operands in shared memory, FP32
// accumulators in tensor memory); every other sum is FP32 on the CUDA cores, reductions
// across blocks in FP64.  Weight gradients are FP32 sums on the CUDA cores.
#include "ctx.cuh"
#include "prims.cuh"
#include "async.cuh"
#include "umma.cuh"

#include <cuda_bf16.h>
#include <math.h>
#include <new>

using namespace lowd;
typedef __nv_bfloat16 bf16;

namespace {

constexpr int kH = 64;
constexpr int kL = 3;
constexpr int kIn = 3;
constexpr int64_t kLayerParams = (int64_t)kH * 2 * kH + kH;
constexpr int64_t kParams = kIn * kH + kH + kL * kLayerParams + kH;
__host__ __device__ constexpr int64_t off_W(int l) { return kIn * kH + kH + (int64_t)l * kLayerParams; }
__host__ __device__ constexpr int64_t off_b(int l) { return off_W(l) + (int64_t)kH * 2 * kH; }
constexpr int64_t kOffQ = kIn * kH + kH + kL * kLayerParams;
constexpr int kT = 256;
constexpr int kWarpsPerBlock = kT / 32;
constexpr uint32_t kUmmaWaitLimit = 1u << 24;
constexpr int kUmmaSmem = 56 * 1024;   // caps residency at 4 CTAs per SM: <= 512 TMEM columns
constexpr int kUmmaCtasPerSm = 4;

inline unsigned blocks_for(int64_t items, int per) { return lowd_grid_for(items, per, 16); }

__device__ __forceinline__ float wt(const float* w, int64_t e) { return w ? w[e] : 1.0f; }

// ------------------------------------------------------------------ graph binding

__global__ void k_mp_check(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                           const float* __restrict__ w, int64_t m, int32_t n, int32_t* __restrict__ err) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = lo[e], b = hi[e];
        bool ok = a >= 0 && a < b && b < n;
        if (w) ok = ok && isfinite(w[e]) && w[e] > 0.0f;
        if (!ok) atomicOr(err, 1);
    }
}

__global__ void k_mp_keys(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, int64_t m,
                          uint32_t* __restrict__ key, int32_t* __restrict__ val, int32_t* __restrict__ cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = lo[e], b = hi[e];
        key[2 * e] = (uint32_t)a;
        val[2 * e] = (int32_t)(2 * e);          // side 0: the node is lo
        key[2 * e + 1] = (uint32_t)b;
        val[2 * e + 1] = (int32_t)(2 * e + 1);  // side 1: the node is hi
        atomicAdd(&cnt[a], 1);
        atomicAdd(&cnt[b], 1);
    }
}

// adjacency entry i of node v: edge adj[i] >> 1, v is its lo end iff (adj[i] & 1) == 0
__global__ void k_mp_nbr(const int32_t* __restrict__ adj, int64_t len, const int32_t* __restrict__ lo,
                         const int32_t* __restrict__ hi, int32_t* __restrict__ nbr) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = adj[i];
        const int64_t e = a >> 1;
        nbr[i] = (a & 1) ? lo[e] : hi[e];
    }
}

// warp-per-node loop helper
#define FOR_NODE_WARP(v, n)                                                                  \
    for (int32_t v = (int32_t)(blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)); v < (n); \
         v += (int32_t)(gridDim.x * kWarpsPerBlock))

__global__ void k_mp_feat1(int32_t n, const int32_t* __restrict__ row, const int32_t* __restrict__ adj,
                           const float* __restrict__ w, float* __restrict__ dw, float* __restrict__ x) {
    const int lane = threadIdx.x & 31;
    FOR_NODE_WARP(v, n) {
        float d = 0.0f, sl = 0.0f;
        const int32_t b = row[v], e = row[v + 1];
        for (int32_t i = b + lane; i < e; i += 32) {
            const float we = wt(w, adj[i] >> 1);
            d += we;
            sl += logf(we);
        }
        d = warp_sum(d);
        sl = warp_sum(sl);
        if (lane == 0) {
            dw[v] = d;
            x[3 * (int64_t)v] = log1pf(d);
            x[3 * (int64_t)v + 1] = e > b ? sl / (float)(e - b) : 0.0f;
        }
    }
}

__global__ void k_mp_feat2(int32_t n, const int32_t* __restrict__ row, const int32_t* __restrict__ nbr,
                           const float* __restrict__ dw, float* __restrict__ x) {
    const int lane = threadIdx.x & 31;
    FOR_NODE_WARP(v, n) {
        float s = 0.0f;
        for (int32_t i = row[v] + lane; i < row[v + 1]; i += 32) s += dw[nbr[i]];
        s = warp_sum(s);
        if (lane == 0) x[3 * (int64_t)v + 2] = log1pf(s);
    }
}

// ------------------------------------------------------------------ forward

__global__ void k_mp_embed(int32_t n, const float* __restrict__ x, const float* __restrict__ p, bf16* __restrict__ h0) {
    const int64_t total = (int64_t)n * kH;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i >> 6;
        const int j = (int)(i & 63);
        float a = p[kIn * kH + j];
#pragma unroll
        for (int k = 0; k < kIn; ++k) a += x[3 * v + k] * p[k * kH + j];
        h0[i] = __float2bfloat16_rn(fmaxf(a, 0.0f));
    }
}

// m_v = mean of h over v's neighbours; lane l owns features 2l, 2l + 1
__global__ void k_mp_mean(int32_t n, const int32_t* __restrict__ row, const int32_t* __restrict__ nbr,
                          const bf16* __restrict__ h, bf16* __restrict__ mo) {
    const int lane = threadIdx.x & 31;
    const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(h);
    FOR_NODE_WARP(v, n) {
        const int32_t b = row[v], e = row[v + 1];
        float ax = 0.0f, ay = 0.0f;
        for (int32_t base = b; base < e; base += 32) {
            const int32_t cntn = min(32, e - base);
            const int32_t mine = lane < cntn ? nbr[base + lane] : 0;
            int32_t j = 0;
            for (; j + 4 <= cntn; j += 4) {
                const int32_t u0 = __shfl_sync(0xffffffffu, mine, j);
                const int32_t u1 = __shfl_sync(0xffffffffu, mine, j + 1);
                const int32_t u2 = __shfl_sync(0xffffffffu, mine, j + 2);
                const int32_t u3 = __shfl_sync(0xffffffffu, mine, j + 3);
                const float2 f0 = __bfloat1622float2(h2[(int64_t)u0 * 32 + lane]);
                const float2 f1 = __bfloat1622float2(h2[(int64_t)u1 * 32 + lane]);
                const float2 f2 = __bfloat1622float2(h2[(int64_t)u2 * 32 + lane]);
                const float2 f3 = __bfloat1622float2(h2[(int64_t)u3 * 32 + lane]);
                ax += f0.x; ay += f0.y;
                ax += f1.x; ay += f1.y;
                ax += f2.x; ay += f2.y;
                ax += f3.x; ay += f3.y;
            }
            for (; j < cntn; ++j) {
                const int32_t u = __shfl_sync(0xffffffffu, mine, j);
                const float2 f = __bfloat1622float2(h2[(int64_t)u * 32 + lane]);
                ax += f.x; ay += f.y;
            }
        }
        const float inv = e > b ? 1.0f / (float)(e - b) : 0.0f;
        reinterpret_cast<__nv_bfloat162*>(mo)[(int64_t)v * 32 + lane] = __floats2bfloat162_rn(ax * inv, ay * inv);
    }
}

enum { EPI_RELU_BF16 = 0, EPI_F32 = 1 };

// Row-tile product on the tensor cores: for every tile of 128 rows, D[128 x N] = A B^T with
// A = the tile's rows of [A0, A1] (K = 128: two 64-column bf16 arrays) or of A0 (K = 64),
// B [N x K] bf16 row-major; FP32 accumulators in tensor memory.  Epilogue: bias + relu to
// bf16 rows of width N, or FP32 rows of width N.  Rows past n read as zero and are not
// stored.  One CTA of 4 warps per tile (grid-stride over tiles); warp w reads tensor-memory
// lanes 32w..32w+31 (rows of the tile).  The wait on the MMA's commit is bounded; on expiry
// the block records an error, waits (bounded) once more and frees its tensor memory.
template <int K, int N, int EPI>
__global__ void __launch_bounds__(128) k_umma_rows(int32_t n, const bf16* __restrict__ A0, const bf16* __restrict__ A1,
                                                   const bf16* __restrict__ B, const float* __restrict__ bias,
                                                   bf16* __restrict__ outb, float* __restrict__ outf,
                                                   int32_t* __restrict__ err) {
    static_assert(K == 64 || K == 128, "K");
    static_assert(N == 64 || N == 128, "N");
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr uint32_t kABytes = 128u * K * 2u;
    unsigned char* sA = smem;
    unsigned char* sB = smem + kABytes;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_taddr;
    __shared__ int32_t s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tmem_alloc(&s_taddr, (uint32_t)N);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    constexpr int kKC = K / 8;  // 16-byte chunks per row
    for (int c = tid; c < N * kKC; c += 128) {
        const int rl = c & 7, kc = (c >> 3) % kKC, rh = (c >> 3) / kKC;
        const int r = rh * 8 + rl;
        const uint4 val = *reinterpret_cast<const uint4*>(B + (size_t)r * K + kc * 8);
        *reinterpret_cast<uint4*>(sB + umma_tile_offset(r, kc * 8, K)) = val;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;
    const int32_t tiles = (n + 127) / 128;
    constexpr uint32_t idesc = umma_idesc_bf16(128, N);
    uint32_t phase = 0;
    bool failed = false;
    for (int32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t row0 = (int64_t)tile * 128;
        for (int c = tid; c < 128 * kKC; c += 128) {
            const int rl = c & 7, kc = (c >> 3) % kKC, rh = (c >> 3) / kKC;
            const int r = rh * 8 + rl;
            const int64_t gr = row0 + r;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (gr < n) {
                const bf16* src = (K == 128 && kc >= 8) ? A1 + gr * 64 + (kc - 8) * 8 : A0 + gr * 64 + kc * 8;
                val = *reinterpret_cast<const uint4*>(src);
            }
            *reinterpret_cast<uint4*>(sA + umma_tile_offset(r, kc * 8, K)) = val;
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int ks = 0; ks < K / 16; ++ks)
                umma_bf16(taddr, umma_desc(a0 + ks * 256, 128, K * 16), umma_desc(b0 + ks * 256, 128, K * 16), idesc,
                          ks > 0 ? 1u : 0u);
            umma_commit(&bar);
            uint32_t spins = 0;
            bool ok = mbar_try_wait(&bar, phase);
            while (!ok && ++spins < kUmmaWaitLimit) ok = mbar_try_wait(&bar, phase);
            s_ok = ok ? 1 : 0;
        }
        __syncthreads();
        if (!s_ok) { failed = true; break; }
        phase ^= 1u;
        tc_fence_after();
        const int r = warp * 32 + lane;
        const int64_t gr = row0 + r;
        const uint32_t trow = taddr + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 16) {
            float vv[16];
            tmem_ld16(trow + (uint32_t)c0, vv);
            if (gr < n) {
                if (EPI == EPI_RELU_BF16) {
                    uint32_t pk[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float a = fmaxf(vv[2 * i] + bias[c0 + 2 * i], 0.0f);
                        const float b = fmaxf(vv[2 * i + 1] + bias[c0 + 2 * i + 1], 0.0f);
                        const __nv_bfloat162 t2 = __floats2bfloat162_rn(a, b);
                        pk[i] = *reinterpret_cast<const uint32_t*>(&t2);
                    }
                    uint4* dst = reinterpret_cast<uint4*>(outb + gr * N + c0);
                    dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                } else {
                    float4* dst = reinterpret_cast<float4*>(outf + gr * N + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) dst[i] = make_float4(vv[4 * i], vv[4 * i + 1], vv[4 * i + 2], vv[4 * i + 3]);
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (failed && tid == 0) {
        atomicOr(err, 2);
        uint32_t spins = 0;   // the MMA may still be running: bounded second wait before freeing
        while (!mbar_try_wait(&bar, phase) && ++spins < kUmmaWaitLimit) {
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, (uint32_t)N);
}

__global__ void k_mp_phi(int32_t n, const bf16* __restrict__ h, const float* __restrict__ q, float* __restrict__ phi) {
    const int lane = threadIdx.x & 31;
    const float2 qq = make_float2(q[2 * lane], q[2 * lane + 1]);
    FOR_NODE_WARP(v, n) {
        const float2 f = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(h)[(int64_t)v * 32 + lane]);
        float s = f.x * qq.x + f.y * qq.y;
        s = warp_sum(s);
        if (lane == 0) phi[v] = s;
    }
}

__global__ void k_mp_sigma(int64_t m, const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                           const float* __restrict__ phi, float* __restrict__ sigma) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const float z = phi[lo[e]] - phi[hi[e]];
        sigma[e] = 1.0f / (1.0f + expf(-z));
    }
}

__global__ void k_mp_loads(int32_t n, const int32_t* __restrict__ row, const int32_t* __restrict__ adj,
                           const float* __restrict__ w, const float* __restrict__ sigma, float* __restrict__ loads) {
    const int lane = threadIdx.x & 31;
    FOR_NODE_WARP(v, n) {
        float s = 0.0f;
        for (int32_t i = row[v] + lane; i < row[v + 1]; i += 32) {
            const int32_t a = adj[i];
            const int64_t e = a >> 1;
            const float sg = sigma[e];
            s += (a & 1) ? (1.0f - sg) * wt(w, e) : sg * wt(w, e);
        }
        s = warp_sum(s);
        if (lane == 0) loads[v] = s;
    }
}

__global__ void k_mp_loss(int32_t n, const float* __restrict__ l, const float* __restrict__ t, double* __restrict__ part) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const double d = (double)l[v] - (double)t[v];
        a += d * d;
        b += (double)t[v] * (double)t[v];
    }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = a; part[2 * blockIdx.x + 1] = b; }
}

__global__ void k_mp_loss_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) { a += part[2 * i]; b += part[2 * i + 1]; }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0) { out[0] = a; out[1] = b; out[2] = b > 0.0 ? a / b : 0.0; }
}

// ------------------------------------------------------------------ backward

__global__ void k_mp_gl(int32_t n, const float* __restrict__ l, const float* __restrict__ t,
                        const double* __restrict__ sc, float* __restrict__ gl) {
    const double Z = sc[1];
    const float s = Z > 0.0 ? (float)(2.0 / Z) : 0.0f;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        gl[v] = s * (l[v] - t[v]);
}

__global__ void k_mp_delta(int64_t m, const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                           const float* __restrict__ w, const float* __restrict__ sigma, const float* __restrict__ gl,
                           float* __restrict__ delta) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const float s = sigma[e];
        delta[e] = wt(w, e) * (gl[lo[e]] - gl[hi[e]]) * s * (1.0f - s);
    }
}

__global__ void k_mp_psi(int32_t n, const int32_t* __restrict__ row, const int32_t* __restrict__ adj,
                         const float* __restrict__ delta, float* __restrict__ psi) {
    const int lane = threadIdx.x & 31;
    FOR_NODE_WARP(v, n) {
        float s = 0.0f;
        for (int32_t i = row[v] + lane; i < row[v + 1]; i += 32) {
            const int32_t a = adj[i];
            const float d = delta[a >> 1];
            s += (a & 1) ? -d : d;
        }
        s = warp_sum(s);
        if (lane == 0) psi[v] = s;
    }
}

// G3 = psi q^T (gradient of the loss in h3) and per-block partials of dq = sum_v psi_v h3_v
__global__ void k_mp_head_bwd(int32_t n, const float* __restrict__ psi, const bf16* __restrict__ h,
                              const float* __restrict__ q, float* __restrict__ G, float* __restrict__ part) {
    __shared__ float2 sh[kWarpsPerBlock][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float2 qq = make_float2(q[2 * lane], q[2 * lane + 1]);
    float2 acc = make_float2(0.0f, 0.0f);
    FOR_NODE_WARP(v, n) {
        const float ps = psi[v];
        reinterpret_cast<float2*>(G)[(int64_t)v * 32 + lane] = make_float2(ps * qq.x, ps * qq.y);
        const float2 f = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(h)[(int64_t)v * 32 + lane]);
        acc.x += ps * f.x;
        acc.y += ps * f.y;
    }
    sh[wid][lane] = acc;
    __syncthreads();
    if (wid == 0) {
        float2 s = make_float2(0.0f, 0.0f);
        for (int k = 0; k < kWarpsPerBlock; ++k) { s.x += sh[k][lane].x; s.y += sh[k][lane].y; }
        part[blockIdx.x * 64 + 2 * lane] = s.x;
        part[blockIdx.x * 64 + 2 * lane + 1] = s.y;
    }
}

// out[c] = sum over blocks of part[b * cols + c], in FP64
__global__ void k_mp_reduce_cols(const float* __restrict__ part, int nb, int cols, float* __restrict__ out) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += (double)part[(size_t)b * cols + c];
        out[c] = (float)s;
    }
}

__global__ void k_mp_dA(int64_t cnt, const float* __restrict__ G, const bf16* __restrict__ h, float* __restrict__ dA,
                        bf16* __restrict__ dAb) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = __bfloat162float(h[i]) > 0.0f ? G[i] : 0.0f;
        dA[i] = d;
        if (dAb) dAb[i] = __float2bfloat16_rn(d);
    }
}

constexpr int kDWCols = 128 * 64 + 64;   // per-block partials: [in][out] weights, then the bias

// Weight gradient of a 128 -> 64 layer on the tensor cores: per CTA, D[128 x 64] = X^T dA
// over its chunks of 64 nodes (X = [h, m] bf16, the product's K = nodes), with dA the bf16
// copy that the backward-data product also uses; FP32 accumulators in tensor memory.  Each
// chunk is staged transposed (rows = X's columns / dA's columns, K-major) into one of two
// shared-memory buffers while the other buffer's four MMAs run; the commit of a buffer is
// awaited (bounded) before the buffer is staged again.  The bias gradient (sum of the FP32
// dA over nodes) is summed on the CUDA cores while staging.  Epilogue: warp w reads tensor
// lanes 32w.. (rows of X^T) and writes the CTA's partials in the layout k_mp_dW_final reduces.
constexpr int kDwChunk = 64;                                  // nodes per staged chunk
constexpr uint32_t kDwABytes = 128u * kDwChunk * 2u;          // X^T tile
constexpr uint32_t kDwBBytes = 64u * kDwChunk * 2u;           // dA^T tile
constexpr int kDwSmem = 56 * 1024;                            // >= 2 (A + B); caps residency at 4 CTAs
__global__ void __launch_bounds__(128) k_umma_dW(int32_t n, const bf16* __restrict__ h, const bf16* __restrict__ mm,
                                                 const bf16* __restrict__ dAb, const float* __restrict__ dA,
                                                 float* __restrict__ part, int32_t* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t s_taddr;
    __shared__ int32_t s_ok;
    __shared__ float s_bias[64];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tmem_alloc(&s_taddr, 64u);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        s_ok = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;
    constexpr uint32_t idesc = umma_idesc_bf16(128, 64);
    const int64_t chunks = ((int64_t)n + kDwChunk - 1) / kDwChunk;
    float bsum = 0.0f;   // column tid & 63 of the bias gradient, nodes of this thread's half
    int32_t it = 0;
    bool failed = false;
    for (int64_t ch = blockIdx.x; ch < chunks; ch += gridDim.x, ++it) {
        const int b = it & 1;
        unsigned char* sA = smem + (uint32_t)b * (kDwABytes + kDwBBytes);
        unsigned char* sB = sA + kDwABytes;
        if (it >= 2) {   // the MMAs that last read this buffer (two chunks ago) must be done
            if (tid == 0) {
                const uint32_t par = (uint32_t)(((it - 2) >> 1) & 1);
                uint32_t spins = 0;
                bool ok = mbar_try_wait(&bar[b], par);
                while (!ok && ++spins < kUmmaWaitLimit) ok = mbar_try_wait(&bar[b], par);
                s_ok = ok ? 1 : 0;
            }
            __syncthreads();
            if (!s_ok) { failed = true; break; }
        }
        const int64_t v0 = ch * kDwChunk;
        // X^T: row f (feature 0..127), K = node; 16-byte global loads of 8 features
        for (int idx = tid; idx < kDwChunk * 16; idx += 128) {
            const int node = idx & (kDwChunk - 1), fc = idx >> 6;
            const int64_t v = v0 + node;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (v < n) val = *reinterpret_cast<const uint4*>((fc < 8 ? h + v * 64 + fc * 8 : mm + v * 64 + (fc - 8) * 8));
            const uint16_t* e8 = reinterpret_cast<const uint16_t*>(&val);
#pragma unroll
            for (int e = 0; e < 8; ++e)
                *reinterpret_cast<uint16_t*>(sA + umma_tile_offset(fc * 8 + e, node, kDwChunk)) = e8[e];
        }
        // dA^T: row j (output column 0..63), K = node; the bias gradient from the FP32 dA
        for (int idx = tid; idx < kDwChunk * 64; idx += 128) {
            const int node = idx >> 6, j = idx & 63;
            const int64_t v = v0 + node;
            uint16_t bits = 0;
            if (v < n) {
                bits = *reinterpret_cast<const uint16_t*>(dAb + v * 64 + j);
                bsum += dA[v * 64 + j];
            }
            *reinterpret_cast<uint16_t*>(sB + umma_tile_offset(j, node, kDwChunk)) = bits;
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int ks = 0; ks < kDwChunk / 16; ++ks)
                umma_bf16(taddr, umma_desc(a0 + ks * 256, 128, kDwChunk * 16), umma_desc(b0 + ks * 256, 128, kDwChunk * 16),
                          idesc, (it > 0 || ks > 0) ? 1u : 0u);
            umma_commit(&bar[b]);
        }
    }
    // wait for the last chunk's MMAs (a commit covers every earlier MMA of the thread)
    if (it > 0 && tid == 0) {
        const int last = it - 1;
        const uint32_t par = (uint32_t)((last >> 1) & 1);
        uint32_t spins = 0;
        bool ok = mbar_try_wait(&bar[last & 1], par);
        while (!ok && ++spins < kUmmaWaitLimit) ok = mbar_try_wait(&bar[last & 1], par);
        if (!ok) failed = true;
        s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_ok) failed = true;
    tc_fence_after();
    float* out = part + (size_t)blockIdx.x * kDWCols;
    const int r = warp * 32 + lane;   // row of X^T = input feature
    if (!failed) {
#pragma unroll 1
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float vv[16];
            if (it > 0) tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, vv);
#pragma unroll
            for (int i = 0; i < 16; ++i) out[r * 64 + c0 + i] = it > 0 ? vv[i] : 0.0f;
        }
    } else if (tid == 0) {
        atomicOr(err, 2);
    }
    if (tid >= 64) s_bias[tid - 64] = bsum;
    __syncthreads();
    if (tid < 64) out[128 * 64 + tid] = bsum + s_bias[tid];
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, 64u);
}

// reduce the dW partials: grad W_l [out][in] and grad b_l
__global__ void k_mp_dW_final(const float* __restrict__ part, int nb, float* __restrict__ gW, float* __restrict__ gb) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < kDWCols; c += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += (double)part[(size_t)b * kDWCols + c];
        if (c < 128 * 64) {
            const int in = c >> 6, o = c & 63;
            gW[o * 128 + in] = (float)s;
        } else {
            gb[c - 128 * 64] = (float)s;
        }
    }
}

// embedding layer: per-block partials of dW_in = x^T dA0 (3 x 64) and db_in
constexpr int kDWinCols = kIn * 64 + 64;
__global__ void __launch_bounds__(256) k_mp_dWin(int32_t n, const float* __restrict__ x, const float* __restrict__ dA,
                                                 float* __restrict__ part) {
    __shared__ float sh[4][kDWinCols];
    const int t = threadIdx.x, j = t & 63, g = t >> 6;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, ab = 0.0f;
    for (int64_t v = (int64_t)blockIdx.x * 4 + g; v < n; v += (int64_t)gridDim.x * 4) {
        const float d = dA[v * 64 + j];
        a0 += x[3 * v] * d;
        a1 += x[3 * v + 1] * d;
        a2 += x[3 * v + 2] * d;
        ab += d;
    }
    sh[g][j] = a0; sh[g][64 + j] = a1; sh[g][128 + j] = a2; sh[g][192 + j] = ab;
    __syncthreads();
    if (g == 0) {
        for (int c = j; c < kDWinCols; c += 64) {
            part[(size_t)blockIdx.x * kDWinCols + c] = sh[0][c] + sh[1][c] + sh[2][c] + sh[3][c];
        }
    }
}

// gradient in the previous layer's h: dX[u, :64] + sum over neighbours v of dX[v, 64:] / deg(v)
__global__ void k_mp_prevG(int32_t n, const int32_t* __restrict__ row, const int32_t* __restrict__ nbr,
                           const float* __restrict__ dX, float* __restrict__ Gp) {
    const int lane = threadIdx.x & 31;
    const float2* d2 = reinterpret_cast<const float2*>(dX);
    FOR_NODE_WARP(u, n) {
        float2 acc = d2[(int64_t)u * 64 + lane];
        const int32_t b = row[u], e = row[u + 1];
        for (int32_t base = b; base < e; base += 32) {
            const int32_t cntn = min(32, e - base);
            int32_t mine = 0;
            float inv = 0.0f;
            if (lane < cntn) {
                mine = nbr[base + lane];
                inv = 1.0f / (float)(row[mine + 1] - row[mine]);
            }
            for (int32_t j = 0; j < cntn; ++j) {
                const int32_t v = __shfl_sync(0xffffffffu, mine, j);
                const float iv = __shfl_sync(0xffffffffu, inv, j);
                const float2 f = d2[(int64_t)v * 64 + 32 + lane];
                acc.x += f.x * iv;
                acc.y += f.y * iv;
            }
        }
        reinterpret_cast<float2*>(Gp)[(int64_t)u * 32 + lane] = acc;
    }
}

__global__ void k_mp_adam(int64_t P, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                          float* __restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// bf16 copies of the layer weights: wb[l] = W_l [out][in] (forward B operand, K = in),
// wtb[l] = W_l^T [in][out] (backward B operand, K = out)
__global__ void k_mp_cast(const float* __restrict__ p, bf16* __restrict__ wb, bf16* __restrict__ wtb) {
    const int total = kL * kH * 2 * kH;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int l = i / (kH * 2 * kH), r = i % (kH * 2 * kH);
        const int o = r / (2 * kH), in = r % (2 * kH);
        const bf16 b = __float2bfloat16_rn(p[off_W(l) + r]);
        wb[i] = b;
        wtb[(size_t)l * kH * 2 * kH + (size_t)in * kH + o] = b;
    }
}

__global__ void k_mp_splits(int64_t m, const float* __restrict__ sigma, const float* __restrict__ w, float* __restrict__ s) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        s[e] = sigma[e] * wt(w, e);
}

}  // namespace

struct lowd_mpnn_ctx {
    cudaStream_t st = nullptr;
    bool own_stream = false;
    char err[256] = {0};
    int dev_sms = 152;
    // parameters
    float *p = nullptr, *g = nullptr, *am = nullptr, *av = nullptr;
    bf16 *wb = nullptr, *wtb = nullptr;
    int32_t adam_t = 0;
    // bound graph
    int32_t n = 0;
    int64_t m = 0;
    int bound = 0, has_target = 0, forward_done = 0, weighted = 0;
    int64_t cap_n = -1, cap_m = -1;
    int32_t *lo = nullptr, *hi = nullptr, *row = nullptr, *adj = nullptr, *nbr = nullptr;
    uint32_t *key0 = nullptr, *key1 = nullptr;   // [2m] sort keys (ping, pong)
    float *w = nullptr, *target = nullptr, *x = nullptr, *dw = nullptr;
    bf16* h[kL + 1] = {nullptr};
    bf16* mm[kL] = {nullptr};
    bf16* dAb = nullptr;
    float *phi = nullptr, *sigma = nullptr, *loads = nullptr, *gl = nullptr, *delta = nullptr, *psi = nullptr;
    float *G = nullptr, *G2 = nullptr, *dA = nullptr, *dX = nullptr, *part = nullptr;
    double* sc = nullptr;      // [0] sum (l - t)^2, [1] sum t^2, [2] loss
    double* lpart = nullptr;   // loss partials
    int32_t* d_err = nullptr;
    double* h_sc = nullptr;    // pinned
    void* tmp = nullptr;
    size_t tmp_cap = 0;

    lowd_status fail(cudaError_t e) {
        snprintf(err, sizeof(err), "%s", cudaGetErrorString(e));
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LOWD_ERR_OUT_OF_MEMORY : LOWD_ERR_CUDA;
    }
};

namespace {

constexpr int kPartBlocks = 152 * 2;   // blocks of the reduction kernels

template <class T>
cudaError_t mp_alloc(T** p, size_t count) {
    *p = nullptr;
    return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

template <class T>
void mp_free(T** p) {
    if (*p) cudaFree(*p);
    *p = nullptr;
}

void free_graph(lowd_mpnn_ctx* c) {
    mp_free(&c->lo); mp_free(&c->hi); mp_free(&c->row); mp_free(&c->adj); mp_free(&c->nbr);
    mp_free(&c->key0); mp_free(&c->key1);
    mp_free(&c->w); mp_free(&c->target); mp_free(&c->x); mp_free(&c->dw);
    for (auto& p : c->h) mp_free(&p);
    for (auto& p : c->mm) mp_free(&p);
    mp_free(&c->dAb); mp_free(&c->phi); mp_free(&c->sigma); mp_free(&c->loads); mp_free(&c->gl);
    mp_free(&c->delta); mp_free(&c->psi); mp_free(&c->G); mp_free(&c->G2); mp_free(&c->dA); mp_free(&c->dX);
    mp_free(&c->tmp);
    c->tmp_cap = 0;
    c->cap_n = c->cap_m = -1;
    c->bound = 0;
}

cudaError_t ensure_graph(lowd_mpnn_ctx* c, int64_t n, int64_t m) {
    if (n <= c->cap_n && m <= c->cap_m) return cudaSuccess;
    free_graph(c);
    const size_t N = (size_t)n, M = (size_t)m;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = mp_alloc(&c->lo, M);
    if (e == cudaSuccess) e = mp_alloc(&c->hi, M);
    if (e == cudaSuccess) e = mp_alloc(&c->w, M);
    if (e == cudaSuccess) e = mp_alloc(&c->row, N + 1);
    if (e == cudaSuccess) e = mp_alloc(&c->adj, 2 * M);
    if (e == cudaSuccess) e = mp_alloc(&c->nbr, 2 * M);
    if (e == cudaSuccess) e = mp_alloc(&c->key0, 2 * M);
    if (e == cudaSuccess) e = mp_alloc(&c->key1, 2 * M);
    if (e == cudaSuccess) e = mp_alloc(&c->target, N);
    if (e == cudaSuccess) e = mp_alloc(&c->x, 3 * N);
    if (e == cudaSuccess) e = mp_alloc(&c->dw, N);
    for (int l = 0; l <= kL && e == cudaSuccess; ++l) e = mp_alloc(&c->h[l], N * kH);
    for (int l = 0; l < kL && e == cudaSuccess; ++l) e = mp_alloc(&c->mm[l], N * kH);
    if (e == cudaSuccess) e = mp_alloc(&c->dAb, N * kH);
    if (e == cudaSuccess) e = mp_alloc(&c->phi, N);
    if (e == cudaSuccess) e = mp_alloc(&c->sigma, M);
    if (e == cudaSuccess) e = mp_alloc(&c->loads, N);
    if (e == cudaSuccess) e = mp_alloc(&c->gl, N);
    if (e == cudaSuccess) e = mp_alloc(&c->delta, M);
    if (e == cudaSuccess) e = mp_alloc(&c->psi, N);
    if (e == cudaSuccess) e = mp_alloc(&c->G, N * kH);
    if (e == cudaSuccess) e = mp_alloc(&c->G2, N * kH);
    if (e == cudaSuccess) e = mp_alloc(&c->dA, N * kH);
    if (e == cudaSuccess) e = mp_alloc(&c->dX, N * 2 * kH);
    if (e == cudaSuccess) {
        c->tmp_cap = lowd_sort_tmp_bytes(2 * m > n + 1 ? 2 * m : n + 1);
        e = cudaMalloc(&c->tmp, c->tmp_cap);
    }
    if (e != cudaSuccess) { free_graph(c); return e; }
    c->cap_n = n;
    c->cap_m = m;
    return cudaSuccess;
}

template <int K, int N, int EPI>
cudaError_t launch_umma(lowd_mpnn_ctx* c, const bf16* A0, const bf16* A1, const bf16* B, const float* bias, bf16* ob,
                        float* of) {
    if (c->n == 0) return cudaSuccess;
    auto kern = k_umma_rows<K, N, EPI>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kUmmaSmem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = ((int64_t)c->n + 127) / 128;
    int64_t grid = (int64_t)c->dev_sms * kUmmaCtasPerSm;
    if (grid > tiles) grid = tiles;
    LOWD_LAUNCH(kern, (unsigned)grid, 128, kUmmaSmem, c->st, c->n, A0, A1, B, bias, ob, of, c->d_err);
    return cudaGetLastError();
}

lowd_status read_err(lowd_mpnn_ctx* c, const char* what) {
    int32_t e = 0;
    cudaError_t ce = cudaMemcpyAsync(&e, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->st);
    if (ce != cudaSuccess) return c->fail(ce);
    if (e & 2) {
        snprintf(c->err, sizeof(c->err), "%s: a bounded wait on a tensor-core commit expired", what);
        cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), c->st);
        return LOWD_ERR_CUDA;
    }
    return LOWD_OK;
}

#define MP_CK(call)                                  \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return c->fail(e_);   \
    } while (0)

lowd_status mp_bind_dev(lowd_mpnn_ctx* c, int32_t n, int64_t m, const int32_t* lo, const int32_t* hi, const float* w,
                        const float* target, cudaMemcpyKind kind) {
    MP_CK(ensure_graph(c, n, m));
    c->n = n;
    c->m = m;
    c->bound = 0;
    c->forward_done = 0;
    c->weighted = w != nullptr;
    c->has_target = target != nullptr;
    if (m > 0) {
        MP_CK(cudaMemcpyAsync(c->lo, lo, sizeof(int32_t) * (size_t)m, kind, c->st));
        MP_CK(cudaMemcpyAsync(c->hi, hi, sizeof(int32_t) * (size_t)m, kind, c->st));
        if (w) MP_CK(cudaMemcpyAsync(c->w, w, sizeof(float) * (size_t)m, kind, c->st));
    }
    if (target && n > 0) MP_CK(cudaMemcpyAsync(c->target, target, sizeof(float) * (size_t)n, kind, c->st));
    const float* wp = w ? c->w : nullptr;
    MP_CK(cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), c->st));
    int32_t* cnt = reinterpret_cast<int32_t*>(c->G);   // scratch: n + 1 counters
    MP_CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)n + 1), c->st));
    if (m > 0) {
        LOWD_LAUNCH(k_mp_check, blocks_for(m, kT), kT, 0, c->st, c->lo, c->hi, wp, m, n, c->d_err);
        uint32_t* k0 = c->key0;
        uint32_t* k1 = c->key1;
        int32_t* v0 = c->nbr;   // sort values ping / pong; nbr is rebuilt from adj below
        int32_t* v1 = c->adj;
        LOWD_LAUNCH(k_mp_keys, blocks_for(m, kT), kT, 0, c->st, c->lo, c->hi, m, k0, v0, cnt);
        const int bits = bit_length_u64(n > 1 ? (uint64_t)(n - 1) : 1);
        const int r = radix_sort_pairs<uint32_t, int32_t>(k0, v0, k1, v1, 2 * m, bits, c->tmp, c->st);
        if (r == 0) MP_CK(cudaMemcpyAsync(c->adj, v0, sizeof(int32_t) * 2 * (size_t)m, cudaMemcpyDeviceToDevice, c->st));
        LOWD_LAUNCH(k_mp_nbr, blocks_for(2 * m, kT), kT, 0, c->st, c->adj, 2 * m, c->lo, c->hi, c->nbr);
    }
    scan_exclusive<int32_t>(cnt, c->row, (int64_t)n + 1, nullptr, c->tmp, c->st);
    MP_CK(cudaGetLastError());
    int32_t bad = 0;
    MP_CK(cudaMemcpyAsync(&bad, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
    MP_CK(cudaStreamSynchronize(c->st));
    if (bad) {
        snprintf(c->err, sizeof(c->err), "edges must satisfy 0 <= lo < hi < n with finite weights > 0");
        return LOWD_ERR_INVALID_ARG;
    }
    if (n > 0) {
        const unsigned gw = blocks_for(n, kWarpsPerBlock);
        LOWD_LAUNCH(k_mp_feat1, gw, kT, 0, c->st, n, c->row, c->adj, wp, c->dw, c->x);
        LOWD_LAUNCH(k_mp_feat2, gw, kT, 0, c->st, n, c->row, c->nbr, c->dw, c->x);
    }
    MP_CK(cudaGetLastError());
    c->bound = 1;
    return LOWD_OK;
}

lowd_status mp_forward(lowd_mpnn_ctx* c) {
    const int32_t n = c->n;
    const int64_t m = c->m;
    const float* wp = c->weighted ? c->w : nullptr;
    if (n > 0) {
        LOWD_LAUNCH(k_mp_embed, blocks_for((int64_t)n * kH, kT), kT, 0, c->st, n, c->x, c->p, c->h[0]);
        const unsigned gw = blocks_for(n, kWarpsPerBlock);
        for (int l = 0; l < kL; ++l) {
            LOWD_LAUNCH(k_mp_mean, gw, kT, 0, c->st, n, c->row, c->nbr, c->h[l], c->mm[l]);
            MP_CK((launch_umma<128, 64, EPI_RELU_BF16>(c, c->h[l], c->mm[l], c->wb + (size_t)l * kH * 2 * kH,
                                                        c->p + off_b(l), c->h[l + 1], nullptr)));
        }
        LOWD_LAUNCH(k_mp_phi, gw, kT, 0, c->st, n, c->h[kL], c->p + kOffQ, c->phi);
    }
    if (m > 0) LOWD_LAUNCH(k_mp_sigma, blocks_for(m, kT), kT, 0, c->st, m, c->lo, c->hi, c->phi, c->sigma);
    if (n > 0)
        LOWD_LAUNCH(k_mp_loads, blocks_for(n, kWarpsPerBlock), kT, 0, c->st, n, c->row, c->adj, wp, c->sigma, c->loads);
    MP_CK(cudaGetLastError());
    if (c->has_target) {
        const int nb = (int)blocks_for(n > 0 ? n : 1, kT) > kPartBlocks ? kPartBlocks : (int)blocks_for(n > 0 ? n : 1, kT);
        LOWD_LAUNCH(k_mp_loss, nb, kT, 0, c->st, n, c->loads, c->target, c->lpart);
        LOWD_LAUNCH(k_mp_loss_final, 1, kT, 0, c->st, c->lpart, nb, c->sc);
        MP_CK(cudaGetLastError());
    }
    LOWD_TRY(read_err(c, "forward"));
    c->forward_done = 1;
    return LOWD_OK;
}

lowd_status mp_backward(lowd_mpnn_ctx* c) {
    const int32_t n = c->n;
    const int64_t m = c->m;
    const float* wp = c->weighted ? c->w : nullptr;
    MP_CK(cudaMemsetAsync(c->g, 0, sizeof(float) * kParams, c->st));
    if (n == 0) return LOWD_OK;
    const unsigned gw = blocks_for(n, kWarpsPerBlock);
    LOWD_LAUNCH(k_mp_gl, blocks_for(n, kT), kT, 0, c->st, n, c->loads, c->target, c->sc, c->gl);
    if (m > 0) LOWD_LAUNCH(k_mp_delta, blocks_for(m, kT), kT, 0, c->st, m, c->lo, c->hi, wp, c->sigma, c->gl, c->delta);
    else MP_CK(cudaMemsetAsync(c->delta, 0, sizeof(float), c->st));
    LOWD_LAUNCH(k_mp_psi, gw, kT, 0, c->st, n, c->row, c->adj, c->delta, c->psi);
    const unsigned gh = gw > (unsigned)kPartBlocks ? (unsigned)kPartBlocks : gw;
    LOWD_LAUNCH(k_mp_head_bwd, gh, kT, 0, c->st, n, c->psi, c->h[kL], c->p + kOffQ, c->G, c->part);
    LOWD_LAUNCH(k_mp_reduce_cols, 1, 64, 0, c->st, c->part, (int)gh, 64, c->g + kOffQ);
    float* G = c->G;
    float* Gn = c->G2;
    const int64_t dw_chunks = ((int64_t)n + kDwChunk - 1) / kDwChunk;
    const unsigned gdw = dw_chunks > kPartBlocks ? (unsigned)kPartBlocks : (unsigned)dw_chunks;
    MP_CK(cudaFuncSetAttribute(k_umma_dW, cudaFuncAttributeMaxDynamicSharedMemorySize, kDwSmem));
    for (int l = kL - 1; l >= 0; --l) {
        LOWD_LAUNCH(k_mp_dA, blocks_for((int64_t)n * kH, kT), kT, 0, c->st, (int64_t)n * kH, G, c->h[l + 1], c->dA, c->dAb);
        LOWD_LAUNCH(k_umma_dW, gdw, 128, kDwSmem, c->st, n, c->h[l], c->mm[l], c->dAb, c->dA, c->part, c->d_err);
        LOWD_LAUNCH(k_mp_dW_final, blocks_for(kDWCols, kT), kT, 0, c->st, c->part, (int)gdw, c->g + off_W(l), c->g + off_b(l));
        MP_CK((launch_umma<64, 128, EPI_F32>(c, c->dAb, nullptr, c->wtb + (size_t)l * kH * 2 * kH, nullptr, nullptr,
                                              c->dX)));
        LOWD_LAUNCH(k_mp_prevG, gw, kT, 0, c->st, n, c->row, c->nbr, c->dX, Gn);
        float* t = G; G = Gn; Gn = t;
    }
    LOWD_LAUNCH(k_mp_dA, blocks_for((int64_t)n * kH, kT), kT, 0, c->st, (int64_t)n * kH, G, c->h[0], c->dA,
                (bf16*)nullptr);
    const unsigned gi = blocks_for((n + 3) / 4, 1) > (unsigned)kPartBlocks ? (unsigned)kPartBlocks : blocks_for((n + 3) / 4, 1);
    LOWD_LAUNCH(k_mp_dWin, gi, 256, 0, c->st, n, c->x, c->dA, c->part);
    LOWD_LAUNCH(k_mp_reduce_cols, 1, 256, 0, c->st, c->part, (int)gi, kDWinCols, c->g);   // W_in then b_in
    MP_CK(cudaGetLastError());
    return read_err(c, "backward");
}

lowd_status cast_weights(lowd_mpnn_ctx* c) {
    LOWD_LAUNCH(k_mp_cast, blocks_for(kL * kH * 2 * kH, kT), kT, 0, c->st, c->p, c->wb, c->wtb);
    MP_CK(cudaGetLastError());
    return LOWD_OK;
}

}  // namespace

extern "C" {

int64_t lowd_mpnn_param_count(void) { return kParams; }

lowd_status lowd_mpnn_create(void* stream, lowd_mpnn* out) {
    if (!out) return LOWD_ERR_INVALID_ARG;
    *out = nullptr;
    lowd_mpnn_ctx* c = new (std::nothrow) lowd_mpnn_ctx();
    if (!c) return LOWD_ERR_OUT_OF_MEMORY;
    c->st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!c->st) {
        e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
        c->own_stream = e == cudaSuccess;
    }
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->dev_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = mp_alloc(&c->p, kParams);
    if (e == cudaSuccess) e = mp_alloc(&c->g, kParams);
    if (e == cudaSuccess) e = mp_alloc(&c->am, kParams);
    if (e == cudaSuccess) e = mp_alloc(&c->av, kParams);
    if (e == cudaSuccess) e = mp_alloc(&c->wb, (size_t)kL * kH * 2 * kH);
    if (e == cudaSuccess) e = mp_alloc(&c->wtb, (size_t)kL * kH * 2 * kH);
    if (e == cudaSuccess) e = mp_alloc(&c->part, (size_t)kPartBlocks * kDWCols);
    if (e == cudaSuccess) e = mp_alloc(&c->sc, 4);
    if (e == cudaSuccess) e = mp_alloc(&c->lpart, 2 * (size_t)kPartBlocks);
    if (e == cudaSuccess) e = mp_alloc(&c->d_err, 4);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_sc, 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->p, 0, sizeof(float) * kParams, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->am, 0, sizeof(float) * kParams, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->av, 0, sizeof(float) * kParams, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), c->st);
    if (e == cudaSuccess && cast_weights(c) != LOWD_OK) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        lowd_mpnn_free(c);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LOWD_ERR_OUT_OF_MEMORY : LOWD_ERR_CUDA;
    }
    *out = c;
    return LOWD_OK;
}

lowd_status lowd_mpnn_set_params(lowd_mpnn c, const float* params, int32_t mem) {
    if (!c || !params || (mem != LOWD_MEM_HOST && mem != LOWD_MEM_DEVICE)) return LOWD_ERR_INVALID_ARG;
    const cudaMemcpyKind k = mem == LOWD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    MP_CK(cudaMemcpyAsync(c->p, params, sizeof(float) * kParams, k, c->st));
    MP_CK(cudaMemsetAsync(c->am, 0, sizeof(float) * kParams, c->st));
    MP_CK(cudaMemsetAsync(c->av, 0, sizeof(float) * kParams, c->st));
    c->adam_t = 0;
    c->forward_done = 0;
    LOWD_TRY(cast_weights(c));
    MP_CK(cudaStreamSynchronize(c->st));
    return LOWD_OK;
}

lowd_status lowd_mpnn_get_params(lowd_mpnn c, float* params, int32_t mem) {
    if (!c || !params || (mem != LOWD_MEM_HOST && mem != LOWD_MEM_DEVICE)) return LOWD_ERR_INVALID_ARG;
    const cudaMemcpyKind k = mem == LOWD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    MP_CK(cudaMemcpyAsync(params, c->p, sizeof(float) * kParams, k, c->st));
    MP_CK(cudaStreamSynchronize(c->st));
    return LOWD_OK;
}

lowd_status lowd_mpnn_bind(lowd_mpnn c, int32_t n, int64_t m, const int32_t* lo, const int32_t* hi, const float* w,
                           const float* target, int32_t mem) {
    if (!c || n < 0 || m < 0 || (m > 0 && (!lo || !hi)) || (mem != LOWD_MEM_HOST && mem != LOWD_MEM_DEVICE))
        return LOWD_ERR_INVALID_ARG;
    if (m >= ((int64_t)1 << 30) || n > (1 << 30)) return LOWD_ERR_TOO_LARGE;
    return mp_bind_dev(c, n, m, lo, hi, w, target,
                       mem == LOWD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
}

lowd_status lowd_mpnn_set_features(lowd_mpnn c, const float* x, int32_t mem) {
    if (!c || !x || (mem != LOWD_MEM_HOST && mem != LOWD_MEM_DEVICE)) return LOWD_ERR_INVALID_ARG;
    if (!c->bound) return LOWD_ERR_BAD_STATE;
    const cudaMemcpyKind k = mem == LOWD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (c->n > 0) MP_CK(cudaMemcpyAsync(c->x, x, sizeof(float) * 3 * (size_t)c->n, k, c->st));
    MP_CK(cudaStreamSynchronize(c->st));
    c->forward_done = 0;
    return LOWD_OK;
}

lowd_status lowd_mpnn_forward(lowd_mpnn c, double* loss) {
    if (!c) return LOWD_ERR_INVALID_ARG;
    if (!c->bound) return LOWD_ERR_BAD_STATE;
    LOWD_TRY(mp_forward(c));
    if (loss) {
        if (!c->has_target) return LOWD_ERR_BAD_STATE;
        MP_CK(cudaMemcpyAsync(c->h_sc, c->sc, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
        MP_CK(cudaStreamSynchronize(c->st));
        *loss = c->h_sc[2];
    }
    return LOWD_OK;
}

lowd_status lowd_mpnn_backward(lowd_mpnn c) {
    if (!c) return LOWD_ERR_INVALID_ARG;
    if (!c->bound || !c->forward_done || !c->has_target) return LOWD_ERR_BAD_STATE;
    return mp_backward(c);
}

lowd_status lowd_mpnn_adam(lowd_mpnn c, float lr, float beta1, float beta2, float eps) {
    if (!c || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return LOWD_ERR_INVALID_ARG;
    c->adam_t += 1;
    const float bc1 = (float)(1.0 - pow((double)beta1, (double)c->adam_t));
    const float bc2 = (float)(1.0 - pow((double)beta2, (double)c->adam_t));
    LOWD_LAUNCH(k_mp_adam, blocks_for(kParams, kT), kT, 0, c->st, (int64_t)kParams, c->p, c->g, c->am, c->av, lr, beta1,
                beta2, eps, bc1, bc2);
    LOWD_TRY(cast_weights(c));
    c->forward_done = 0;
    MP_CK(cudaStreamSynchronize(c->st));
    return LOWD_OK;
}

lowd_status lowd_mpnn_read(lowd_mpnn c, int32_t what, float* out, int32_t mem) {
    if (!c || !out || (mem != LOWD_MEM_HOST && mem != LOWD_MEM_DEVICE)) return LOWD_ERR_INVALID_ARG;
    const float* src = nullptr;
    size_t count = 0;
    switch (what) {
        case LOWD_MPNN_SIGMA: src = c->sigma; count = (size_t)c->m; break;
        case LOWD_MPNN_LOADS: src = c->loads; count = (size_t)c->n; break;
        case LOWD_MPNN_GRAD: src = c->g; count = (size_t)kParams; break;
        case LOWD_MPNN_FEATURES: src = c->x; count = 3 * (size_t)c->n; break;
        case LOWD_MPNN_PHI: src = c->phi; count = (size_t)c->n; break;
        default: return LOWD_ERR_INVALID_ARG;
    }
    if (what != LOWD_MPNN_GRAD && !c->bound) return LOWD_ERR_BAD_STATE;
    if ((what == LOWD_MPNN_SIGMA || what == LOWD_MPNN_LOADS || what == LOWD_MPNN_PHI) && !c->forward_done)
        return LOWD_ERR_BAD_STATE;
    const cudaMemcpyKind k = mem == LOWD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (count) MP_CK(cudaMemcpyAsync(out, src, sizeof(float) * count, k, c->st));
    MP_CK(cudaStreamSynchronize(c->st));
    return LOWD_OK;
}

lowd_status lowd_warm_start(lowd_handle h, lowd_mpnn c) {
    if (!h || !c) return LOWD_ERR_INVALID_ARG;
    if (h->m >= ((int64_t)1 << 30)) return LOWD_ERR_TOO_LARGE;
    cudaError_t e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return h->fail(e);
    lowd_status s = mp_bind_dev(c, h->n, h->m, h->u, h->v, h->w, nullptr, cudaMemcpyDeviceToDevice);
    if (s == LOWD_OK) s = mp_forward(c);
    if (s != LOWD_OK) {
        snprintf(h->err, sizeof(h->err), "warm start: %.200s", c->err);
        return s;
    }
    float* d = nullptr;
    LOWD_TRY(dalloc(h, &d, h->m));
    if (h->m > 0) LOWD_LAUNCH(k_mp_splits, blocks_for(h->m, kT), kT, 0, c->st, h->m, c->sigma, c->weighted ? c->w : nullptr, d);
    e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) { dfree(h, &d); return h->fail(e); }
    s = lowd_apply_splits_dev(h, d);
    cudaStreamSynchronize(h->st);
    dfree(h, &d);
    return s;
}

const char* lowd_mpnn_last_error(lowd_mpnn c) { return c ? c->err : ""; }

void lowd_mpnn_free(lowd_mpnn c) {
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    free_graph(c);
    mp_free(&c->p); mp_free(&c->g); mp_free(&c->am); mp_free(&c->av);
    mp_free(&c->wb); mp_free(&c->wtb); mp_free(&c->part); mp_free(&c->sc); mp_free(&c->lpart); mp_free(&c->d_err);
    if (c->h_sc) cudaFreeHost(c->h_sc);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    delete c;
}

}  // extern "C"
