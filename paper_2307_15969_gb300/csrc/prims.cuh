// Device primitives shared by the LOWD kernels: warp/block scans, a device-wide
// exclusive scan, and a stable least-significant-digit radix sort whose passes are
// counting sorts (per-tile digit histogram with warp-level match/ballot ranks,
// exclusive scan of the histograms, stable scatter).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// Host-side count of kernel launches made by this library (all threads, all handles).
void lowd_note_launch();

// Streaming multiprocessors of the current device (queried once per device ordinal).
int lowd_device_sms();

// Blocks for a grid-stride loop over n items at `threads` per block: enough to cover n,
// at most `per_sm` blocks per SM of the current device.
inline unsigned lowd_grid_for(int64_t n, int threads, int per_sm = 32) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)lowd_device_sms() * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// Launch a kernel and count it.
#define LOWD_LAUNCH(kern, grid, block, smem, stream, ...)              \
    do {                                                               \
        kern<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);      \
        lowd_note_launch();                                            \
    } while (0)

namespace lowd {

constexpr int kWarp = 32;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned warp_id() { return threadIdx.x >> 5; }

template <class T>
__device__ __forceinline__ T warp_incl_scan(T x) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane_id() >= o) x += y;
    }
    return x;
}

template <class T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive prefix and
// writes the block total.  `sh` needs blockDim.x/32 + 1 elements.
template <class T>
__device__ __forceinline__ T block_excl_scan(T x, T* sh, T* total) {
    T inc = warp_incl_scan(x);
    if (lane_id() == 31) sh[warp_id()] = inc;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (warp_id() == 0) {
        T t = (int)lane_id() < nw ? sh[lane_id()] : T(0);
        T ti = warp_incl_scan(t);
        if ((int)lane_id() < nw) sh[lane_id()] = ti - t;
        if ((int)lane_id() == nw - 1) sh[nw] = ti;
    }
    __syncthreads();
    T r = inc - x + sh[warp_id()];
    *total = sh[nw];
    __syncthreads();
    return r;
}

template <class T>
__device__ __forceinline__ T block_sum(T x, T* sh) {
    x = warp_sum(x);
    if (lane_id() == 0) sh[warp_id()] = x;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    T r = T(0);
    if (warp_id() == 0) {
        r = (int)lane_id() < nw ? sh[lane_id()] : T(0);
        r = warp_sum(r);
    }
    __syncthreads();
    return r;  // valid in thread 0
}

// ------------------------------------------------------------------ device-wide scan

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

template <class T>
__global__ void scan_reduce_kernel(const T* __restrict__ in, int64_t n, T* __restrict__ part) {
    __shared__ T sh[kScanThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t j = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (j < n) acc += in[j];
    }
    T s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// single block: exclusive scan of the per-tile partial sums, total to part[nb]
template <class T>
__global__ void scan_partials_kernel(T* __restrict__ part, int64_t nb) {
    __shared__ T sh[kScanThreads / 32 + 1];
    T carry = T(0);
    for (int64_t base = 0; base < nb; base += kScanThreads) {
        int64_t j = base + threadIdx.x;
        T x = j < nb ? part[j] : T(0);
        T tot;
        T e = block_excl_scan(x, sh, &tot);
        if (j < nb) part[j] = e + carry;
        carry += tot;
    }
    if (threadIdx.x == 0) part[nb] = carry;
}

template <class T>
__global__ void scan_apply_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t n,
                                  const T* __restrict__ part) {
    __shared__ T sh[kScanThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    // blocked arrangement: thread t owns items [base + t*I, base + t*I + I)
    T v[kScanItems];
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t j = base + (int64_t)threadIdx.x * kScanItems + i;
        v[i] = j < n ? in[j] : T(0);
        acc += v[i];
    }
    T tot;
    T pre = block_excl_scan(acc, sh, &tot) + part[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t j = base + (int64_t)threadIdx.x * kScanItems + i;
        if (j < n) out[j] = pre;
        pre += v[i];
    }
}

inline int64_t scan_num_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }
// bytes of scratch a scan of n elements of type T needs
template <class T>
inline size_t scan_tmp_bytes(int64_t n) { return sizeof(T) * (size_t)(scan_num_tiles(n) + 2); }

// out[i] = sum(in[0..i)), and *total_dev (device pointer, may be null) = sum(in).
// in and out may alias.  tmp: scan_tmp_bytes<T>(n) bytes.
template <class T>
inline void scan_exclusive(const T* in, T* out, int64_t n, T* total_dev, void* tmp,
                           cudaStream_t st) {
    int64_t nb = scan_num_tiles(n);
    T* part = (T*)tmp;
    if (n > 0) {
        LOWD_LAUNCH(scan_reduce_kernel<T>, (unsigned)nb, kScanThreads, 0, st, in, n, part);
        LOWD_LAUNCH(scan_partials_kernel<T>, 1, kScanThreads, 0, st, part, nb);
        LOWD_LAUNCH(scan_apply_kernel<T>, (unsigned)nb, kScanThreads, 0, st, in, out, n, part);
        if (total_dev) cudaMemcpyAsync(total_dev, part + nb, sizeof(T), cudaMemcpyDeviceToDevice, st);
    } else if (total_dev) {
        cudaMemsetAsync(total_dev, 0, sizeof(T), st);
    }
}

// ------------------------------------------------------------------ stable LSD radix sort

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per tile
constexpr int kRadix = 256;                           // 8-bit digits

template <class K>
__device__ __forceinline__ unsigned digit_of(K k, int shift) { return (unsigned)((k >> shift) & 0xffu); }

// Per-tile digit histogram, digit-major: hist[d * ntiles + tile].
template <class K>
__global__ void radix_hist_kernel(const K* __restrict__ keys, int64_t n, int shift,
                                  uint32_t* __restrict__ hist, int64_t ntiles) {
    __shared__ uint32_t h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int i = 0; i < kSortItems; ++i) {
        int64_t j = base + (int64_t)i * kSortThreads + threadIdx.x;
        bool ok = j < n;
        unsigned d = ok ? digit_of(keys[j], shift) : 0u;
        // warp-aggregate equal digits before touching shared memory
        unsigned peers = __match_any_sync(0xffffffffu, ok ? d : 0x100u);
        int leader = __ffs(peers) - 1;
        if (ok && (int)lane_id() == leader) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x)
        hist[(int64_t)i * ntiles + blockIdx.x] = h[i];
}

// Stable scatter: key at position j of its tile goes to offset[digit, tile] plus the
// number of earlier keys of the same tile with the same digit.  Keys are taken in
// rounds of kSortThreads consecutive positions; inside a round the rank among equal
// digits comes from __match_any_sync (within a warp) plus per-warp counts (across
// warps), so the order of equal keys is preserved.
template <class K, class V>
__global__ void radix_scatter_kernel(const K* __restrict__ kin, const V* __restrict__ vin,
                                     K* __restrict__ kout, V* __restrict__ vout, int64_t n,
                                     int shift, const uint32_t* __restrict__ offs, int64_t ntiles) {
    constexpr int NW = kSortThreads / 32;
    __shared__ uint32_t base_d[kRadix];
    __shared__ uint32_t wcnt[NW][kRadix];
    const int64_t tile = blockIdx.x;
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) base_d[i] = offs[(int64_t)i * ntiles + tile];
    const int64_t base = tile * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        for (int i = threadIdx.x; i < NW * kRadix; i += blockDim.x) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        int64_t j = base + (int64_t)r * kSortThreads + threadIdx.x;
        bool ok = j < n;
        K k = ok ? kin[j] : K(0);
        unsigned d = ok ? digit_of(k, shift) : 0x100u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned lt = (1u << lane_id()) - 1u;
        unsigned rank_in_warp = __popc(peers & lt);
        if (ok && rank_in_warp == 0) wcnt[warp_id()][d] = __popc(peers);
        __syncthreads();
        // exclusive prefix over warps, per digit; then advance the digit base
        for (int dd = threadIdx.x; dd < kRadix; dd += blockDim.x) {
            uint32_t run = 0;
            const uint32_t b = base_d[dd];
#pragma unroll
            for (int w = 0; w < NW; ++w) { uint32_t c = wcnt[w][dd]; wcnt[w][dd] = b + run; run += c; }
            base_d[dd] = b + run;
        }
        __syncthreads();
        if (ok) {
            uint32_t pos = wcnt[warp_id()][d] + rank_in_warp;
            kout[pos] = k;
            if (vin) vout[pos] = vin[j];
        }
        __syncthreads();
    }
}

inline int64_t radix_num_tiles(int64_t n) { return (n + kSortTile - 1) / kSortTile; }
inline size_t radix_tmp_bytes(int64_t n) {
    int64_t nt = radix_num_tiles(n);
    size_t h = sizeof(uint32_t) * (size_t)(kRadix * nt + 2);
    return h + scan_tmp_bytes<uint32_t>(kRadix * nt) + 256;
}

// Stable sort of (key, value) pairs by the low `bits` bits of the key.  Ping-pongs
// between (k0, v0) and (k1, v1); returns 0 if the result is in (k0, v0), 1 if in
// (k1, v1).  v0/v1 may be null (keys only).  n < 2^32.
template <class K, class V>
inline int radix_sort_pairs(K* k0, V* v0, K* k1, V* v1, int64_t n, int bits, void* tmp,
                            cudaStream_t st) {
    if (n <= 1 || bits <= 0) return 0;
    int64_t nt = radix_num_tiles(n);
    uint32_t* hist = (uint32_t*)tmp;
    void* stmp = (char*)tmp + (((sizeof(uint32_t) * (size_t)(kRadix * nt + 2)) + 255) & ~(size_t)255);
    int cur = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        K* ki = cur ? k1 : k0; V* vi = cur ? v1 : v0;
        K* ko = cur ? k0 : k1; V* vo = cur ? v0 : v1;
        LOWD_LAUNCH(radix_hist_kernel<K>, (unsigned)nt, kSortThreads, 0, st, ki, n, shift, hist, nt);
        scan_exclusive<uint32_t>(hist, hist, kRadix * nt, nullptr, stmp, st);
        auto scatter = radix_scatter_kernel<K, V>;
        LOWD_LAUNCH(scatter, (unsigned)nt, kSortThreads, 0, st, ki, vi, ko, vo, n, shift, hist, nt);
        cur ^= 1;
    }
    return cur;
}

inline int bit_length_u64(uint64_t x) { int b = 0; while (x) { ++b; x >>= 1; } return b; }

}  // namespace lowd
