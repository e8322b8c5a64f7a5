// Handle state and host-side helpers shared by the LOWD translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "../../include/lowd.h"
#include "prims.cuh"

// Shared-memory budget of the one-CTA sweep: loads of up to this many nodes are kept
// in shared memory (4 bytes each) for the whole sweep.
#define LOWD_SMEM_NODES 53248

// Largest graph (nodes) lowd_extract_noalloc accepts.
#define LOWD_NOALLOC_MAX_NODES 65536

struct lowd_ctx {
    cudaStream_t st = nullptr;
    int mem = LOWD_MEM_HOST;
    int flags = 0;
    char err[256] = {0};

    // loaded graph G
    int32_t n0 = 0;
    int64_t m0 = 0;
    int64_t dup = 0;
    int weighted = 0;
    int inexact = 0;  // some input weight was off the 2^-20 grid (allowed by flag)

    // current graph (G, or H after pruning): canonical order, lo < hi
    int32_t n = 0;
    int64_t m = 0;
    int32_t* u = nullptr;
    int32_t* v = nullptr;
    float* w = nullptr;     // [m] weights, null for unit weights
    int64_t* wu = nullptr;  // [m] weight units of 2^-20, null for unit weights
    int32_t* map = nullptr; // [n] current id -> original id; null while current == G
    int32_t max_deg = -1;      // maximum unweighted degree of the current graph; -1: not computed yet

    // pruning record (original numbering)
    int pruned = 0;
    int32_t prune_rounds = 0;
    int32_t* sort_perm = nullptr;      // [n0]
    int32_t* removal_round = nullptr;  // [n0]

    // LOWD state, kept in schedule (class-major) order
    int inited = 0;
    int32_t iters = 0;
    int sched = 0;             // 1 one-CTA shared memory, 2 grid matchings
    int sweep_kernel = 0;      // kernel of the last pass (lowd_info.sweep_kernel)
    int sweep_E = 0;           // edges per consumer thread of the staged sweep
    int32_t C = 0;             // number of classes
    int64_t m_pad = 0;         // class-major length, each class padded to a multiple of 4
    int32_t* perm = nullptr;   // [m_pad] class-major position -> canonical edge id, -1 = padding
    int32_t* coff = nullptr;   // [C+1] padded class offsets (multiples of 4)
    int32_t* coff_real = nullptr; // [C+1] class offsets without padding
    int32_t* coff_h = nullptr; // [C+1] host copy of coff
    uint32_t* cuv = nullptr;   // [m_pad] packed ends (lo | hi << 16); padding: (n | n << 16)
    uint32_t* crk = nullptr;   // [m_pad] rank of each end among its node's updates per pass
                               // (16 bits per end, bit 15 = the node's last update)
    int use_versions = 0;      // 1: the staged sweep uses per-node versions (kernel 5)
    float* cw = nullptr;       // [m_pad] weights (weighted only); padding 0
    float* cs = nullptr;       // [m_pad] splits f_e(lo); padding 0
    float* l = nullptr;        // [n + 1] loads; slot n is the padding sentinel
    float* l_lo = nullptr;     // [n + 1] low parts: the load is l + l_lo (pair arithmetic in the sweep)

    // streamed schedule (2): chunked class-major stream, loads in global memory
    int32_t s2_NC = 0, s2_E = 0, s2_S = 0, s2_D = 0;   // chunks, edges per stage, stages, lead
    int32_t s2_K = 0;             // leading classes run as grid-wide steps
    int32_t s2_tail = 0;          // 1 if classes remain for the chunked stream
    int32_t* s2_ctab = nullptr;   // [NC][20] chunk headers
    int32_t* s2_beg = nullptr;    // [NC + 1] padded chunk begins
    int32_t* s2_ea = nullptr;     // [m_pad] ends (node n for padding)
    int32_t* s2_eb = nullptr;
    uint32_t* s2_srcA = nullptr;  // [m_pad] read descriptors of the two ends
    uint32_t* s2_srcB = nullptr;
    float2* s2_lp = nullptr;      // [n + 1] loads as (hi, lo) pairs during the passes
    uint32_t* s2_blob = nullptr;  // per chunk: header, ends, read descriptors (, weights)
    int64_t* s2_blobo = nullptr;  // [NC + 1] word offsets of the chunk blobs
    // hub stars (block updates of the edges with exactly one end of degree >= tau), both
    // schedules: the star edges follow the plain ones, at positions [star_p0, star_p0 + star_m)
    int32_t hub_tau = 0;              // asked for: 0 off, 1 automatic threshold, >= 2 the threshold
    int32_t star_tau = 0;             // threshold in use (0: no star edges)
    int32_t star_S = 0;               // star steps per pass
    int32_t star_nseg = 0;            // stars over all steps
    int32_t star_maxseg = 0;          // most stars in one step
    int64_t star_m = 0;               // star edges
    int64_t star_p0 = 0;              // position of the first star edge
    int32_t* star_step_seg = nullptr; // [star_S + 1] first star of each step
    int32_t* star_seg_beg = nullptr;  // [star_nseg + 1] position of each star's first edge
    int32_t* star_seg_hub = nullptr;  // [star_nseg] hub of each star
    float2* star_bbuf = nullptr;      // [star_m] (a_j, t_j) of stars too large for registers

    // scratch
    void* tmp = nullptr;
    size_t tmp_cap = 0;
    double* d_stats = nullptr;  // FP64 accumulators for checks
    int64_t* d_i64 = nullptr;   // small int64 scratch (16 entries)
    int32_t* d_i32 = nullptr;   // small int32 scratch (16 entries)
    int64_t* h_pin = nullptr;   // pinned host mirror of small scalars (16 entries)

    lowd_status fail(cudaError_t e) {
        snprintf(err, sizeof(err), "%s", cudaGetErrorString(e));
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LOWD_ERR_OUT_OF_MEMORY : LOWD_ERR_CUDA;
    }
    lowd_status need_tmp(size_t bytes) {
        if (bytes <= tmp_cap) return LOWD_OK;
        if (tmp) cudaFree(tmp);
        tmp = nullptr;
        tmp_cap = 0;
        size_t b = bytes + (bytes >> 3) + 4096;
        cudaError_t e = cudaMalloc(&tmp, b);
        if (e != cudaSuccess) return fail(e);
        tmp_cap = b;
        return LOWD_OK;
    }
};

#define LOWD_CK(call)                                             \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return h->fail(e_);                \
    } while (0)

#define LOWD_CK_LAUNCH() LOWD_CK(cudaGetLastError())

#define LOWD_TRY(call)                        \
    do {                                      \
        lowd_status s_ = (call);              \
        if (s_ != LOWD_OK) return s_;         \
    } while (0)

// Device buffers of a handle come from the library's stream-ordered memory pool (one per
// device): allocated and freed in the handle's stream order, so a call's temporaries cost no
// device-wide synchronisation, and freed memory stays reserved in the pool for the next call
// (up to lowd_pool's threshold) instead of being unmapped and mapped again.
cudaMemPool_t lowd_pool();

template <class T>
inline lowd_status dalloc(lowd_ctx* h, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaMemPool_t pool = lowd_pool();
    if (!pool) return h->fail(cudaErrorMemoryAllocation);
    cudaError_t e = cudaMallocFromPoolAsync((void**)p, sizeof(T) * count, pool, h->st);
    if (e != cudaSuccess) { *p = nullptr; return h->fail(e); }
    return LOWD_OK;
}

template <class T>
inline void dfree(lowd_ctx* h, T** p) {
    if (*p) cudaFreeAsync(*p, h->st);
    *p = nullptr;
}

// bytes to allocate for a radix sort + scans over n elements
size_t lowd_sort_tmp_bytes(int64_t n);

// graph.cu
lowd_status lowd_graph_load(lowd_ctx* h, const int32_t* du, const int32_t* dv, const float* dw,
                            int64_t m_in);
lowd_status lowd_graph_prune(lowd_ctx* h, int32_t* rounds);
lowd_status lowd_graph_max_degree(lowd_ctx* h);
int32_t lowd_max_degree(lowd_ctx* h);   // h->max_deg, computed on first use
void lowd_degrees_i32(lowd_ctx* h, int32_t* deg);   // unweighted degrees of the current graph

// sweep.cu
lowd_status lowd_sweep_prepare(lowd_ctx* h, int schedule_req, const float* init_splits_canon);
lowd_status lowd_sweep_run(lowd_ctx* h, int32_t k, const lowd_options* opt, lowd_stats* st);
lowd_status lowd_sweep_rederive(lowd_ctx* h, double* stats3);
lowd_status lowd_sweep_splits_canonical(lowd_ctx* h, float* out_dev);
lowd_status lowd_sweep_load_canonical(lowd_ctx* h, const float* splits_dev);
lowd_status lowd_sweep_edge_order(lowd_ctx* h, int32_t* out_dev);

// stars.cu
struct StarSplit {
    int32_t tau = 0;              // threshold in use (0: all edges plain)
    int64_t m_plain = 0, ms = 0;  // plain and star edges
    int32_t* dfull = nullptr;     // [n] unweighted degrees
    int32_t* pid = nullptr;       // [m_plain] plain edge ids (null: every edge is plain)
    int32_t* sid = nullptr;       // [ms] star edge ids
    int32_t* gu = nullptr;        // [m_plain] ends of the plain edges
    int32_t* gv = nullptr;
    void release(lowd_ctx* h);
};
lowd_status lowd_star_split(lowd_ctx* h, int32_t hub_tau, int schedule, StarSplit* sp);
lowd_status lowd_star_blocks(lowd_ctx* h, const StarSplit& sp, int64_t p0, int32_t C_plain, int64_t m_real_plain);
cudaError_t lowd_star_pass(lowd_ctx* h);

// stream.cu
lowd_status lowd_stream_prepare(lowd_ctx* h, const float* init_splits_canon);
lowd_status lowd_stream_rederive(lowd_ctx* h, double* L64);
cudaError_t lowd_stream_passes(lowd_ctx* h, int32_t passes);

// api.cu
lowd_status lowd_apply_splits_dev(lowd_ctx* h, const float* splits_canon_dev);

// extract.cu
lowd_status lowd_extract_best(lowd_ctx* h, const float* loads_dev, int32_t* S_dev_current,
                              int32_t* S_size, int64_t* W_best);
lowd_status lowd_ldd_export(lowd_ctx* h, const float* loads_dev, double rel_tol, int32_t* shell_orig,
                            int32_t* shell_end, double* lam, int32_t* ns_out);
