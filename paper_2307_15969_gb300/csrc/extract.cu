// Algorithm 1's extraction on the GPU: order nodes by load, peel from the lowest, keep
// the densest set seen.  Peeling from the lowest load visits exactly the prefixes
// S_k = {the k highest nodes in (load, id) order}, k = n..1, and replaces the best set
// only on a strictly higher density, so the answer is the largest k maximising
// W(S_k)/k.  W(S_k) is computed for every k at once: each edge contributes its weight to
// the prefix that first contains both of its ends, bucket max(pos_a, pos_b) of the
// descending order, and an inclusive scan of the buckets gives W(S_k).  All weights
// are integer 2^-20 units, so the sums are exact and the comparison
// W_a * k_b > W_b * k_a is done exactly in 128 bits.
#include "ctx.cuh"
#include "prims.cuh"

using namespace lowd;

namespace {

constexpr int kT = 256;

inline unsigned grid_for(int64_t n) { return lowd_grid_for(n, kT); }

// descending-load key: larger load -> smaller key; values start as n-1..0 so that the
// stable sort leaves equal loads in descending id order
__global__ void k_load_keys(const float* __restrict__ l, int32_t n, uint32_t* __restrict__ key,
                            int32_t* __restrict__ val) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = n - 1 - (int32_t)i;
        float f = l[x] + 0.0f;  // -0 -> +0
        uint32_t b = __float_as_uint(f);
        uint32_t ord = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // ascending order of floats
        key[i] = ~ord;
        val[i] = x;
    }
}

__global__ void k_positions(const int32_t* __restrict__ order, int32_t n, int32_t* __restrict__ pos) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        pos[order[i]] = (int32_t)i;
}

__global__ void k_edge_buckets(const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                               const int64_t* __restrict__ wu, int64_t m,
                               const int32_t* __restrict__ pos, unsigned long long* __restrict__ bucket) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t p = max(pos[u[e]], pos[v[e]]);
        atomicAdd(&bucket[p], wu ? (unsigned long long)wu[e] : 1ull);
    }
}

struct Best {
    int64_t W;  // W(S_k) in units
    int64_t k;  // |S_k|
};

// a better than b: W_a/k_a > W_b/k_b, ties to the larger set
__device__ __forceinline__ bool better(const Best& a, const Best& b) {
    __int128 l = (__int128)a.W * (__int128)b.k;
    __int128 r = (__int128)b.W * (__int128)a.k;
    if (l != r) return l > r;
    return a.k > b.k;
}

__device__ __forceinline__ Best shfl_best(const Best& x, int o) {
    Best y;
    y.W = __shfl_xor_sync(0xffffffffu, x.W, o);
    y.k = __shfl_xor_sync(0xffffffffu, x.k, o);
    return y;
}

// prefix weights W(S_k) = scan[k-1] + bucket[k-1] (inclusive); per-block best
__global__ void k_best_prefix(const int64_t* __restrict__ excl, const unsigned long long* __restrict__ bucket,
                              int32_t n, Best* __restrict__ part) {
    Best b{0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        Best c{excl[i] + (int64_t)bucket[i], i + 1};
        if (b.k == 0 || better(c, b)) b = c;
    }
    for (int o = 16; o > 0; o >>= 1) {
        Best y = shfl_best(b, o);
        if (y.k != 0 && (b.k == 0 || better(y, b))) b = y;
    }
    __shared__ Best sh[kT / 32];
    if (lane_id() == 0) sh[warp_id()] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        Best r = sh[0];
        for (int wv = 1; wv < (int)(blockDim.x >> 5); ++wv)
            if (sh[wv].k != 0 && (r.k == 0 || better(sh[wv], r))) r = sh[wv];
        part[blockIdx.x] = r;
    }
}

__global__ void k_best_final(const Best* __restrict__ part, int32_t np, Best* __restrict__ out) {
    if (threadIdx.x != 0) return;
    Best r{0, 0};
    for (int i = 0; i < np; ++i)
        if (part[i].k != 0 && (r.k == 0 || better(part[i], r))) r = part[i];
    *out = r;
}

__global__ void k_in_best(const int32_t* __restrict__ pos, int32_t n, const Best* __restrict__ best,
                          int32_t* __restrict__ flag) {
    int64_t k = best->k;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = pos[i] < k ? 1 : 0;
}

__global__ void k_emit_members(const int32_t* __restrict__ flag, const int32_t* __restrict__ fpos,
                               int32_t n, const int32_t* __restrict__ map, int32_t* __restrict__ S) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) S[fpos[i]] = map ? map[i] : (int32_t)i;
}

}  // namespace

// Best prefix of the load order on the current graph.  S_dev (device, may be null)
// receives the members in ascending ORIGINAL ids.  *S_size and *W_best are host values.
lowd_status lowd_extract_best(lowd_ctx* h, const float* loads_dev, int32_t* S_dev,
                              int32_t* S_size, int64_t* W_best) {
    cudaStream_t st = h->st;
    const int32_t n = h->n;
    const int64_t m = h->m;
    uint32_t* key[2] = {nullptr, nullptr};
    int32_t* val[2] = {nullptr, nullptr};
    int32_t *pos = nullptr, *flag = nullptr, *fpos = nullptr;
    unsigned long long* bucket = nullptr;
    int64_t* excl = nullptr;
    Best* part = nullptr;
    lowd_status s = LOWD_OK;
    auto cleanup = [&]() {
        dfree(h, &key[0]); dfree(h, &key[1]); dfree(h, &val[0]); dfree(h, &val[1]); dfree(h, &pos);
        dfree(h, &flag); dfree(h, &fpos); dfree(h, &bucket); dfree(h, &excl); dfree(h, &part);
    };
    do {
        if ((s = h->need_tmp(lowd_sort_tmp_bytes(m > n ? m : n)))) break;
        if ((s = dalloc(h, &key[0], n))) break;
        if ((s = dalloc(h, &key[1], n))) break;
        if ((s = dalloc(h, &val[0], n))) break;
        if ((s = dalloc(h, &val[1], n))) break;
        if ((s = dalloc(h, &pos, n))) break;
        if ((s = dalloc(h, &bucket, n))) break;
        if ((s = dalloc(h, &excl, n))) break;
        const unsigned nb = grid_for(n);
        if ((s = dalloc(h, &part, nb + 1))) break;
        LOWD_LAUNCH(k_load_keys, grid_for(n), kT, 0, st, loads_dev, n, key[0], val[0]);
        int cur = radix_sort_pairs<uint32_t, int32_t>(key[0], val[0], key[1], val[1], n, 32, h->tmp, st);
        LOWD_LAUNCH(k_positions, grid_for(n), kT, 0, st, val[cur], n, pos);
        cudaMemsetAsync(bucket, 0, sizeof(unsigned long long) * (size_t)n, st);
        if (m > 0) LOWD_LAUNCH(k_edge_buckets, grid_for(m), kT, 0, st, h->u, h->v, h->wu, m, pos, bucket);
        scan_exclusive<int64_t>((const int64_t*)bucket, excl, n, nullptr, h->tmp, st);
        LOWD_LAUNCH(k_best_prefix, nb, kT, 0, st, excl, bucket, n, part);
        LOWD_LAUNCH(k_best_final, 1, 32, 0, st, part, (int32_t)nb, part + nb);
        if (S_dev) {
            if ((s = dalloc(h, &flag, n))) break;
            if ((s = dalloc(h, &fpos, n))) break;
            LOWD_LAUNCH(k_in_best, grid_for(n), kT, 0, st, pos, n, part + nb, flag);
            scan_exclusive<int32_t>(flag, fpos, n, nullptr, h->tmp, st);
            LOWD_LAUNCH(k_emit_members, grid_for(n), kT, 0, st, flag, fpos, n, h->map, S_dev);
        }
        Best b;
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&b, part + nb, sizeof(Best), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { s = h->fail(e); break; }
        if (S_size) *S_size = (int32_t)b.k;
        if (W_best) *W_best = b.W;
    } while (0);
    cleanup();
    return s;
}

// ------------------------------------------------------------------ allocation-free variant
//
// lowd_extract_noalloc runs the same extraction kernels as lowd_extract on arrays the
// caller passes, taking every intermediate buffer from one statically sized device array
// instead of cudaMalloc.  It serves callers that must not allocate device memory
// themselves or through the library: a process whose device memory is owned by its own
// pool allocator, or a loop with a fixed memory budget that cannot afford the implicit
// device synchronisation of cudaMalloc/cudaFree.  The array lives for the life of the
// process on every device that loads this library, so its size is kept small: graphs of
// at most LOWD_NOALLOC_MAX_NODES nodes.

namespace {

constexpr int32_t kNoallocMaxNodes = LOWD_NOALLOC_MAX_NODES;

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// carve-up of the scratch array for n nodes (byte offsets, each 256-aligned)
struct NoallocLayout {
    size_t bad, key0, key1, val0, val1, pos, bucket, excl, flag, fpos, part, tmp, total;
};

constexpr size_t noalloc_part_entries() {
    return (size_t)((kNoallocMaxNodes + 255) / 256) + 1;
}

inline NoallocLayout noalloc_layout(int32_t n) {
    NoallocLayout L{};
    size_t o = 0;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    L.bad = o; o = al256(o + 4);
    L.key0 = o; o = al256(o + 4 * nn);
    L.key1 = o; o = al256(o + 4 * nn);
    L.val0 = o; o = al256(o + 4 * nn);
    L.val1 = o; o = al256(o + 4 * nn);
    L.pos = o; o = al256(o + 4 * nn);
    L.bucket = o; o = al256(o + 8 * nn);
    L.excl = o; o = al256(o + 8 * nn);
    L.flag = o; o = al256(o + 4 * nn);
    L.fpos = o; o = al256(o + 4 * nn);
    L.part = o; o = al256(o + sizeof(Best) * noalloc_part_entries());
    L.tmp = o; o = al256(o + lowd_sort_tmp_bytes(n));
    L.total = o;
    return L;
}

// The scratch, sized for the largest graph accepted: for LOWD_NOALLOC_MAX_NODES nodes the
// carve-up needs about 2.8 MiB; each call checks the carve-up against this size.
constexpr size_t kNoallocScratchBytes = (size_t)4 << 20;  // 4 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of the scratch on the current device.  It is looked up on every call:
// after cudaDeviceReset the module is loaded again and the array may sit elsewhere, so a
// cached address could be stale.
cudaError_t noalloc_scratch(void** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

// Bits of the input-check word of the allocation-free extraction.
enum { NA_RANGE = 1, NA_LOOP = 2, NA_WEIGHT = 4 };

// Each edge's weight in 2^-20 units, rounded as lowd_load_graph rounds it, added to the
// bucket of the later of its ends.  The caller's arrays are not trusted: an edge with an end
// outside [0, n), a self-loop, or a weight that is not positive and finite or that would let
// the int64 prefix sums overflow (2^-20 units >= wmax_units) is skipped and flagged in *bad.
__global__ void k_edge_buckets_f32(const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                                   const float* __restrict__ w, int64_t m, int32_t n, double wmax_units,
                                   const int32_t* __restrict__ pos, unsigned long long* __restrict__ bucket,
                                   int32_t* __restrict__ bad) {
    int flags = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = u[e], b = v[e];
        if (a < 0 || a >= n || b < 0 || b >= n) { flags |= NA_RANGE; continue; }
        if (a == b) { flags |= NA_LOOP; continue; }
        unsigned long long x = 1ull;
        if (w) {
            const float wf = w[e];
            if (!(wf > 0.0f) || !isfinite(wf)) { flags |= NA_WEIGHT; continue; }
            const double y = rint((double)wf * 1048576.0);
            if (!(y < wmax_units)) { flags |= NA_WEIGHT; continue; }
            x = y < 1.0 ? 1ull : (unsigned long long)y;
        }
        atomicAdd(&bucket[max(pos[a], pos[b])], x);
    }
    flags = __reduce_or_sync(0xffffffffu, flags);
    if (flags && lane_id() == 0) atomicOr(bad, flags);
}

}  // namespace

extern "C" lowd_status lowd_extract_noalloc(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                                            const float* w, const float* loads, int32_t* S, int32_t* S_size,
                                            double* rho, void* stream) {
    if (n < 1 || m < 0 || m >= ((int64_t)1 << 31) || !loads || (m > 0 && (!u || !v)) || !S_size || !rho)
        return LOWD_ERR_INVALID_ARG;
    if (n > kNoallocMaxNodes) return LOWD_ERR_TOO_LARGE;
    const NoallocLayout lay = noalloc_layout(n);
    if (lay.total > kNoallocScratchBytes) return LOWD_ERR_TOO_LARGE;
    void* base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) {
        cudaGetLastError();
        return LOWD_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* b = (unsigned char*)base;
    uint32_t* key0 = (uint32_t*)(b + lay.key0);
    uint32_t* key1 = (uint32_t*)(b + lay.key1);
    int32_t* val0 = (int32_t*)(b + lay.val0);
    int32_t* val1 = (int32_t*)(b + lay.val1);
    int32_t* pos = (int32_t*)(b + lay.pos);
    unsigned long long* bucket = (unsigned long long*)(b + lay.bucket);
    int64_t* excl = (int64_t*)(b + lay.excl);
    int32_t* flag = (int32_t*)(b + lay.flag);
    int32_t* fpos = (int32_t*)(b + lay.fpos);
    Best* part = (Best*)(b + lay.part);
    void* tmp = b + lay.tmp;
    int32_t* bad = (int32_t*)(b + lay.bad);
    const unsigned nb = grid_for(n);
    // the array keeps the previous call's contents: the buckets and the check word must
    // start at zero
    cudaMemsetAsync(bucket, 0, sizeof(unsigned long long) * (size_t)n, st);
    cudaMemsetAsync(bad, 0, sizeof(int32_t), st);
    // per-edge weight bound: m edges of < 2^62 / m units each keep every prefix sum and the
    // 128-bit density products exact
    const double wmax_units = m > 0 ? 4611686018427387904.0 / (double)m : 0.0;
    LOWD_LAUNCH(k_load_keys, grid_for(n), kT, 0, st, loads, n, key0, val0);
    const int cur = radix_sort_pairs<uint32_t, int32_t>(key0, val0, key1, val1, n, 32, tmp, st);
    LOWD_LAUNCH(k_positions, grid_for(n), kT, 0, st, cur ? val1 : val0, n, pos);
    if (m > 0) LOWD_LAUNCH(k_edge_buckets_f32, grid_for(m), kT, 0, st, u, v, w, m, n, wmax_units, pos, bucket, bad);
    scan_exclusive<int64_t>((const int64_t*)bucket, excl, n, nullptr, tmp, st);
    LOWD_LAUNCH(k_best_prefix, nb, kT, 0, st, excl, bucket, n, part);
    LOWD_LAUNCH(k_best_final, 1, 32, 0, st, part, (int32_t)nb, part + nb);
    LOWD_LAUNCH(k_in_best, grid_for(n), kT, 0, st, pos, n, part + nb, flag);
    scan_exclusive<int32_t>(flag, fpos, n, nullptr, tmp, st);
    if (S) LOWD_LAUNCH(k_emit_members, grid_for(n), kT, 0, st, flag, fpos, n, nullptr, S);
    Best best;
    int32_t badw = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&best, part + nb, sizeof(Best), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&badw, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LOWD_ERR_CUDA;
    }
    if (badw) return LOWD_ERR_INVALID_ARG;   // S (if given) holds a result of the valid edges only
    *S_size = (int32_t)best.k;
    const double scale = w ? 1048576.0 : 1.0;
    *rho = best.k > 0 ? (double)best.W / scale / (double)best.k : 0.0;
    return LOWD_OK;
}

// ------------------------------------------------------------------ LDD export
//
// The locally-dense decomposition read off converged loads (Sec. II, Definition of LDD;
// Properties 1-2: every node of B_i \ B_{i-1} carries the load lambda_i and
// lambda_1 > lambda_2 > ...).  Nodes in descending (load, id) order; a shell ends where the
// next load is lower by more than rel_tol of the current one; lambda_i is then computed
// exactly from the integer prefix weights: (W(B_i) - W(B_{i-1})) / |B_i \ B_{i-1}|.

namespace {

__global__ void k_ldd_cuts(const float* __restrict__ l, const int32_t* __restrict__ order, int32_t n,
                           double rel_tol, int32_t* __restrict__ cut) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i == n - 1) { cut[i] = 1; continue; }
        const double a = (double)l[order[i]], b = (double)l[order[i + 1]];
        cut[i] = (a - b) > rel_tol * fabs(a) ? 1 : 0;
    }
}

// shell of sorted position i = cuts before i; position i closing shell j records its end
__global__ void k_ldd_emit(const int32_t* __restrict__ order, const int32_t* __restrict__ cut,
                           const int32_t* __restrict__ cpos, int32_t n, const int32_t* __restrict__ map,
                           int32_t* __restrict__ shell_orig, int32_t* __restrict__ shell_end) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = order[i];
        shell_orig[map ? map[x] : x] = cpos[i] + 1;   // 1-based shell index
        if (cut[i]) shell_end[cpos[i]] = (int32_t)i + 1;
    }
}

// lambda_j from the prefix weights W(S_k) = excl[k] (k < n), W(S_n) = excl[n-1] + bucket[n-1]
__global__ void k_ldd_lambda(const int32_t* __restrict__ shell_end, int32_t ns, const int64_t* __restrict__ excl,
                             const unsigned long long* __restrict__ bucket, int32_t n, double scale,
                             double* __restrict__ lam) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ns;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = shell_end[j];
        const int32_t b = j > 0 ? shell_end[j - 1] : 0;
        const int64_t We = e < n ? excl[e] : excl[n - 1] + (int64_t)bucket[n - 1];
        const int64_t Wb = b == 0 ? 0 : (b < n ? excl[b] : excl[n - 1] + (int64_t)bucket[n - 1]);
        lam[j] = (double)(We - Wb) / scale / (double)(e - b);
    }
}

__global__ void k_fill_i32_x(int32_t* __restrict__ x, int64_t n, int32_t val) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = val;
}

}  // namespace

// shell_orig [n0] (device), shell_end [n] (device), lam [n] (device); *ns host
lowd_status lowd_ldd_export(lowd_ctx* h, const float* loads_dev, double rel_tol, int32_t* shell_orig,
                            int32_t* shell_end, double* lam, int32_t* ns_out) {
    cudaStream_t st = h->st;
    const int32_t n = h->n;
    const int64_t m = h->m;
    uint32_t* key[2] = {nullptr, nullptr};
    int32_t* val[2] = {nullptr, nullptr};
    int32_t *pos = nullptr, *cut = nullptr, *cpos = nullptr;
    unsigned long long* bucket = nullptr;
    int64_t* excl = nullptr;
    lowd_status s = LOWD_OK;
    auto cleanup = [&]() {
        dfree(h, &key[0]); dfree(h, &key[1]); dfree(h, &val[0]); dfree(h, &val[1]); dfree(h, &pos);
        dfree(h, &cut); dfree(h, &cpos); dfree(h, &bucket); dfree(h, &excl);
    };
    do {
        if ((s = h->need_tmp(lowd_sort_tmp_bytes(m > n ? m : n)))) break;
        if ((s = dalloc(h, &key[0], n))) break;
        if ((s = dalloc(h, &key[1], n))) break;
        if ((s = dalloc(h, &val[0], n))) break;
        if ((s = dalloc(h, &val[1], n))) break;
        if ((s = dalloc(h, &pos, n))) break;
        if ((s = dalloc(h, &cut, n))) break;
        if ((s = dalloc(h, &cpos, n))) break;
        if ((s = dalloc(h, &bucket, n))) break;
        if ((s = dalloc(h, &excl, n))) break;
        LOWD_LAUNCH(k_load_keys, grid_for(n), kT, 0, st, loads_dev, n, key[0], val[0]);
        const int cur = radix_sort_pairs<uint32_t, int32_t>(key[0], val[0], key[1], val[1], n, 32, h->tmp, st);
        int32_t* order = val[cur];
        LOWD_LAUNCH(k_positions, grid_for(n), kT, 0, st, order, n, pos);
        cudaMemsetAsync(bucket, 0, sizeof(unsigned long long) * (size_t)n, st);
        if (m > 0) LOWD_LAUNCH(k_edge_buckets, grid_for(m), kT, 0, st, h->u, h->v, h->wu, m, pos, bucket);
        scan_exclusive<int64_t>((const int64_t*)bucket, excl, n, nullptr, h->tmp, st);
        LOWD_LAUNCH(k_ldd_cuts, grid_for(n), kT, 0, st, loads_dev, order, n, rel_tol, cut);
        scan_exclusive<int32_t>(cut, cpos, n, h->d_i32 + 9, h->tmp, st);
        LOWD_LAUNCH(k_fill_i32_x, grid_for(h->n0), kT, 0, st, shell_orig, (int64_t)h->n0, 0);
        LOWD_LAUNCH(k_ldd_emit, grid_for(n), kT, 0, st, order, cut, cpos, n, h->map, shell_orig, shell_end);
        int32_t ns = 0;
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ns, h->d_i32 + 9, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { s = h->fail(e); break; }
        const double scale = h->wu ? 1048576.0 : 1.0;
        LOWD_LAUNCH(k_ldd_lambda, grid_for(ns), kT, 0, st, shell_end, ns, excl, bucket, n, scale, lam);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { s = h->fail(e); break; }
        *ns_out = ns;
    } while (0);
    cleanup();
    return s;
}
