// C ABI entry points (include/lowd.h): argument checks, host/device marshalling, call
// order, and dispatch to the graph, sweep and extraction units.
#include <atomic>
#include <mutex>
#include <new>

#include "ctx.cuh"

static std::atomic<unsigned long long> g_launches{0};

void lowd_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int lowd_device_sms() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];   // 0 = not yet queried
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return 148;   // a conservative count if the device cannot be queried
    }
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
        cudaGetLastError();
        return 148;
    }
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

// The library's memory pool on the current device, created on first use.  Up to
// kPoolKeepBytes of freed memory stay reserved in it between calls; beyond that, freed memory
// goes back to the device at the next synchronisation.
cudaMemPool_t lowd_pool() {
    constexpr int kMaxDev = 64;
    constexpr uint64_t kPoolKeepBytes = 8ull << 30;
    static cudaMemPool_t pools[kMaxDev] = {};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = kPoolKeepBytes;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = p;
    }
    return pools[dev];
}

namespace {

lowd_status check_handle(lowd_handle h) { return h ? LOWD_OK : LOWD_ERR_INVALID_ARG; }

// Copy n elements between caller memory (host or device per handle) and device memory.
template <class T>
lowd_status to_caller(lowd_ctx* h, T* dst, const T* src_dev, size_t n) {
    if (!dst || n == 0) return LOWD_OK;
    cudaMemcpyKind k = h->mem == LOWD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    LOWD_CK(cudaMemcpyAsync(dst, src_dev, sizeof(T) * n, k, h->st));
    if (h->mem != LOWD_MEM_DEVICE) LOWD_CK(cudaStreamSynchronize(h->st));
    return LOWD_OK;
}

void free_all(lowd_ctx* h) {
    dfree(h, &h->u); dfree(h, &h->v); dfree(h, &h->w); dfree(h, &h->wu); dfree(h, &h->map);
    dfree(h, &h->sort_perm); dfree(h, &h->removal_round);
    dfree(h, &h->perm); dfree(h, &h->coff); dfree(h, &h->coff_real); dfree(h, &h->cuv); dfree(h, &h->crk);
    dfree(h, &h->cw); dfree(h, &h->cs); dfree(h, &h->l); dfree(h, &h->l_lo);
    dfree(h, &h->s2_ctab); dfree(h, &h->s2_beg); dfree(h, &h->s2_ea); dfree(h, &h->s2_eb);
    dfree(h, &h->s2_srcA); dfree(h, &h->s2_srcB); dfree(h, &h->s2_lp); dfree(h, &h->s2_blob); dfree(h, &h->s2_blobo);
    dfree(h, &h->star_step_seg); dfree(h, &h->star_seg_beg); dfree(h, &h->star_seg_hub); dfree(h, &h->star_bbuf);
    if (h->tmp) cudaFree(h->tmp);   // the sort scratch is a plain allocation (need_tmp)
    h->tmp = nullptr;
    h->tmp_cap = 0;
    dfree(h, &h->d_stats); dfree(h, &h->d_i64); dfree(h, &h->d_i32);
    if (h->h_pin) cudaFreeHost(h->h_pin);
    h->h_pin = nullptr;
    free(h->coff_h);
    h->coff_h = nullptr;
}

__global__ void k_init_loads(const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                             const float* __restrict__ w, int64_t m, double* __restrict__ L64) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        double x = w ? 0.5 * (double)w[e] : 0.5;
        atomicAdd(&L64[u[e]], x);
        atomicAdd(&L64[v[e]], x);
    }
}

__global__ void k_to_float(const double* __restrict__ x, int32_t n, float* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

__global__ void k_scatter_loads(const float* __restrict__ l, int32_t n, const int32_t* __restrict__ map,
                                float* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[map ? map[i] : (int32_t)i] = l[i];
}

__global__ void k_clamp_splits(const float* __restrict__ s, const float* __restrict__ w, int64_t m,
                               float* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        float we = w ? w[e] : 1.0f;
        out[e] = fminf(fmaxf(s[e], 0.0f), we);
    }
}

__global__ void k_fill_f32(float* __restrict__ x, int64_t n, float val) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = val;
}

__global__ void k_half_weights(const float* __restrict__ w, int64_t m, float* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = w ? 0.5f * w[e] : 0.5f;
}

inline unsigned grid_for(int64_t n) { return lowd_grid_for(n, 256); }

// loads of the current graph into a fresh device buffer (equal-split loads before any pass)
lowd_status current_loads(lowd_ctx* h, float** out) {
    LOWD_TRY(dalloc(h, out, h->n));
    if (h->inited) {
        LOWD_CK(cudaMemcpyAsync(*out, h->l, sizeof(float) * (size_t)h->n, cudaMemcpyDeviceToDevice, h->st));
        return LOWD_OK;
    }
    double* L64 = nullptr;
    LOWD_TRY(dalloc(h, &L64, h->n));
    cudaMemsetAsync(L64, 0, sizeof(double) * (size_t)h->n, h->st);
    if (h->m > 0) LOWD_LAUNCH(k_init_loads, grid_for(h->m), 256, 0, h->st, h->u, h->v, h->w, h->m, L64);
    LOWD_LAUNCH(k_to_float, grid_for(h->n), 256, 0, h->st, L64, h->n, *out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    dfree(h, &L64);
    if (e != cudaSuccess) return h->fail(e);
    return LOWD_OK;
}

}  // namespace

extern "C" {

const char* lowd_status_string(lowd_status s) {
    switch (s) {
        case LOWD_OK: return "ok";
        case LOWD_ERR_INVALID_ARG: return "invalid argument";
        case LOWD_ERR_OUT_OF_MEMORY: return "out of device memory";
        case LOWD_ERR_CUDA: return "CUDA error";
        case LOWD_ERR_BAD_STATE: return "call out of order";
        case LOWD_ERR_NOT_CONVERGED: return "tolerance not met";
        case LOWD_ERR_INEXACT_WEIGHTS: return "weight not a multiple of 2^-20";
        case LOWD_ERR_TOO_LARGE: return "size beyond a documented limit";
    }
    return "unknown status";
}

const char* lowd_last_error(lowd_handle h) { return h ? h->err : ""; }

uint64_t lowd_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

lowd_status lowd_load_graph(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const float* w,
                            int32_t mem, int32_t flags, void* stream, lowd_handle* out) {
    if (!out) return LOWD_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || m < 0 || m >= ((int64_t)1 << 31)) return LOWD_ERR_INVALID_ARG;
    if (m > 0 && (!u || !v)) return LOWD_ERR_INVALID_ARG;
    if (mem != LOWD_MEM_HOST && mem != LOWD_MEM_DEVICE) return LOWD_ERR_INVALID_ARG;
    if (flags & ~LOWD_LOAD_ALLOW_INEXACT) return LOWD_ERR_INVALID_ARG;
    lowd_ctx* h = new (std::nothrow) lowd_ctx();
    if (!h) return LOWD_ERR_OUT_OF_MEMORY;
    h->st = (cudaStream_t)stream;
    h->mem = mem;
    h->flags = flags;
    h->n0 = n;
    const int32_t* du = u;
    const int32_t* dv = v;
    const float* dw = w;
    int32_t *cu = nullptr, *cv = nullptr;
    float* cw = nullptr;
    lowd_status s = LOWD_OK;
    if (mem == LOWD_MEM_HOST && m > 0) {
        if ((s = dalloc(h, &cu, m)) || (s = dalloc(h, &cv, m)) || (w && (s = dalloc(h, &cw, m)))) {
            dfree(h, &cu); dfree(h, &cv); dfree(h, &cw);
            free_all(h); delete h;
            return s;
        }
        cudaMemcpyAsync(cu, u, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, h->st);
        cudaMemcpyAsync(cv, v, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, h->st);
        if (w) cudaMemcpyAsync(cw, w, sizeof(float) * (size_t)m, cudaMemcpyHostToDevice, h->st);
        du = cu; dv = cv; dw = w ? cw : nullptr;
    }
    s = lowd_graph_load(h, du, dv, dw, m);
    if (s == LOWD_OK) {
        cudaError_t e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) s = h->fail(e);
    } else {
        cudaStreamSynchronize(h->st);
    }
    dfree(h, &cu); dfree(h, &cv); dfree(h, &cw);
    if (s != LOWD_OK) {
        free_all(h);
        delete h;
        return s;
    }
    *out = h;
    return LOWD_OK;
}

lowd_status lowd_prune(lowd_handle h, int32_t* n_kept, int64_t* m_kept, int32_t* rounds) {
    LOWD_TRY(check_handle(h));
    if (h->pruned || h->inited) return LOWD_ERR_BAD_STATE;
    int32_t r = 0;
    LOWD_TRY(lowd_graph_prune(h, &r));
    if (n_kept) *n_kept = h->n;
    if (m_kept) *m_kept = h->m;
    if (rounds) *rounds = r;
    return LOWD_OK;
}

lowd_status lowd_iterate(lowd_handle h, int32_t k, const lowd_options* opt, lowd_stats* st) {
    LOWD_TRY(check_handle(h));
    if (k < 0) return LOWD_ERR_INVALID_ARG;
    if (opt && (opt->check_every < 0 || opt->rel_tol < 0 || opt->schedule < 0 || opt->schedule > 2 ||
                opt->node_versions < 0 || opt->node_versions > 1 || opt->hub_stars < 0))
        return LOWD_ERR_INVALID_ARG;
    h->use_versions = opt ? opt->node_versions : 0;
    if (!h->inited) h->hub_tau = opt ? opt->hub_stars : 0;
    if (!h->inited) LOWD_TRY(lowd_sweep_prepare(h, opt ? opt->schedule : 0, nullptr));
    return lowd_sweep_run(h, k, opt, st);
}

lowd_status lowd_extract(lowd_handle h, int32_t* S, int32_t* S_size, double* rho, float* loads) {
    LOWD_TRY(check_handle(h));
    float* l = nullptr;
    int32_t* Sdev = nullptr;
    lowd_status s = LOWD_OK;
    do {
        if ((s = current_loads(h, &l))) break;
        if (S) {
            if (h->mem == LOWD_MEM_DEVICE) Sdev = S;
            else if ((s = dalloc(h, &Sdev, h->n))) break;
        }
        int32_t k = 0;
        int64_t Wb = 0;
        if ((s = lowd_extract_best(h, l, Sdev, &k, &Wb))) break;
        if (S && h->mem != LOWD_MEM_DEVICE) {
            if ((s = to_caller(h, S, Sdev, (size_t)k))) break;
        }
        if (S_size) *S_size = k;
        double scale = h->wu ? 1048576.0 : 1.0;
        if (rho) *rho = k > 0 ? (double)Wb / scale / (double)k : 0.0;
        if (loads) {
            float* full = nullptr;
            if (h->mem == LOWD_MEM_DEVICE) full = loads;
            else if ((s = dalloc(h, &full, h->n0))) break;
            cudaMemsetAsync(full, 0, sizeof(float) * (size_t)h->n0, h->st);
            LOWD_LAUNCH(k_scatter_loads, grid_for(h->n), 256, 0, h->st, l, h->n, h->map, full);
            if (h->mem != LOWD_MEM_DEVICE) {
                s = to_caller(h, loads, full, (size_t)h->n0);
                dfree(h, &full);
                if (s) break;
            }
        }
        if (cudaGetLastError() != cudaSuccess) { s = h->fail(cudaGetLastError()); break; }
        if (h->mem != LOWD_MEM_DEVICE) {
            cudaError_t e = cudaStreamSynchronize(h->st);
            if (e != cudaSuccess) { s = h->fail(e); break; }
        }
    } while (0);
    if (h->mem != LOWD_MEM_DEVICE) dfree(h, &Sdev);
    dfree(h, &l);
    return s;
}

lowd_status lowd_ldd_dks_bound(int32_t n_shells, const int32_t* shell_end, const double* lambda, int32_t k,
                               double* bound, int32_t* exact) {
    if (n_shells < 1 || !shell_end || !lambda || !bound || k < 1 || k > shell_end[n_shells - 1])
        return LOWD_ERR_INVALID_ARG;
    double prefix = 0.0;   // W(B_{j-1})
    int32_t prev = 0;      // |B_{j-1}|
    for (int32_t j = 0; j < n_shells; ++j) {
        if (shell_end[j] <= prev) return LOWD_ERR_INVALID_ARG;   // sizes must grow
        if (k <= shell_end[j]) {
            *bound = (prefix + (double)(k - prev) * lambda[j]) / (double)k;
            if (exact) *exact = k == shell_end[j] ? 1 : 0;
            return LOWD_OK;
        }
        prefix += lambda[j] * (double)(shell_end[j] - prev);
        prev = shell_end[j];
    }
    return LOWD_ERR_INVALID_ARG;
}

lowd_status lowd_get_ldd(lowd_handle h, double rel_tol, int32_t* shell, double* lambda, int32_t* shell_end,
                         int32_t* n_shells) {
    LOWD_TRY(check_handle(h));
    if (!n_shells || !(rel_tol >= 0.0)) return LOWD_ERR_INVALID_ARG;
    float* l = nullptr;
    int32_t *sh = nullptr, *se = nullptr;
    double* lam = nullptr;
    lowd_status s = LOWD_OK;
    do {
        if ((s = current_loads(h, &l))) break;
        if ((s = dalloc(h, &sh, h->n0))) break;
        if ((s = dalloc(h, &se, h->n))) break;
        if ((s = dalloc(h, &lam, h->n))) break;
        int32_t ns = 0;
        if ((s = lowd_ldd_export(h, l, rel_tol, sh, se, lam, &ns))) break;
        if ((s = to_caller(h, shell, sh, (size_t)h->n0))) break;
        if ((s = to_caller(h, shell_end, se, (size_t)ns))) break;
        if ((s = to_caller(h, lambda, lam, (size_t)ns))) break;
        cudaError_t e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) { s = h->fail(e); break; }
        *n_shells = ns;
    } while (0);
    dfree(h, &l); dfree(h, &sh); dfree(h, &se); dfree(h, &lam);
    return s;
}

lowd_status lowd_get_info(lowd_handle h, lowd_info* info) {
    LOWD_TRY(check_handle(h));
    if (!info) return LOWD_ERR_INVALID_ARG;
    lowd_info x;
    memset(&x, 0, sizeof(x));
    x.n_orig = h->n0;
    x.n = h->n;
    x.m_orig = h->m0;
    x.m = h->m;
    x.duplicates = h->dup;
    x.weighted = h->weighted;
    x.pruned = h->pruned;
    x.classes = h->C + h->star_S;
    x.schedule = h->sched;
    x.max_degree = lowd_max_degree(h);
    x.prune_rounds = h->prune_rounds;
    x.sweep_kernel = h->sweep_kernel;
    x.sweep_edges_per_thread = h->sweep_E;
    x.star_threshold = h->star_tau;
    x.star_steps = h->star_S;
    x.stars = h->star_nseg;
    x.star_edges = h->star_m;
    *info = x;
    return LOWD_OK;
}

lowd_status lowd_get_graph(lowd_handle h, int32_t* u, int32_t* v, float* w) {
    LOWD_TRY(check_handle(h));
    LOWD_TRY(to_caller(h, u, h->u, (size_t)h->m));
    LOWD_TRY(to_caller(h, v, h->v, (size_t)h->m));
    if (w) {
        if (h->w) {
            LOWD_TRY(to_caller(h, w, h->w, (size_t)h->m));
        } else {
            float* ones = nullptr;
            LOWD_TRY(dalloc(h, &ones, h->m));
            if (h->m > 0) LOWD_LAUNCH(k_fill_f32, grid_for(h->m), 256, 0, h->st, ones, h->m, 1.0f);
            lowd_status r = LOWD_OK;
            if (cudaGetLastError() != cudaSuccess) r = h->fail(cudaGetLastError());
            if (r == LOWD_OK) r = to_caller(h, w, ones, (size_t)h->m);
            cudaStreamSynchronize(h->st);
            dfree(h, &ones);
            LOWD_TRY(r);
        }
    }
    return LOWD_OK;
}

lowd_status lowd_get_splits(lowd_handle h, float* s) {
    LOWD_TRY(check_handle(h));
    if (!s) return LOWD_ERR_INVALID_ARG;
    float* d = nullptr;
    LOWD_TRY(dalloc(h, &d, h->m));
    lowd_status r = LOWD_OK;
    if (h->inited) r = lowd_sweep_splits_canonical(h, d);
    else if (h->m > 0) LOWD_LAUNCH(k_half_weights, grid_for(h->m), 256, 0, h->st, h->w, h->m, d);
    if (r == LOWD_OK && cudaGetLastError() != cudaSuccess) r = h->fail(cudaGetLastError());
    if (r == LOWD_OK) r = to_caller(h, s, d, (size_t)h->m);
    if (r == LOWD_OK) {
        cudaError_t e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) r = h->fail(e);
    }
    dfree(h, &d);
    return r;
}

}  // extern "C"

// Splits (canonical order, device) become the state: the first time they initialise the
// schedule, later they replace the splits (clamped to [0, w_e]) and the loads are
// re-derived from them.
lowd_status lowd_apply_splits_dev(lowd_ctx* h, const float* d) {
    if (!h->inited) return lowd_sweep_prepare(h, 0, d);
    float* c = nullptr;
    LOWD_TRY(dalloc(h, &c, h->m));
    if (h->m > 0) LOWD_LAUNCH(k_clamp_splits, grid_for(h->m), 256, 0, h->st, d, h->w, h->m, c);
    lowd_status r = lowd_sweep_load_canonical(h, c);
    cudaStreamSynchronize(h->st);
    dfree(h, &c);
    if (r) return r;
    double st3[3];
    return lowd_sweep_rederive(h, st3);
}

extern "C" {

lowd_status lowd_set_splits(lowd_handle h, const float* s) {
    LOWD_TRY(check_handle(h));
    if (!s) return LOWD_ERR_INVALID_ARG;
    float* d = nullptr;
    LOWD_TRY(dalloc(h, &d, h->m));
    lowd_status r = LOWD_OK;
    cudaMemcpyKind k = h->mem == LOWD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (h->m > 0 && cudaMemcpyAsync(d, s, sizeof(float) * (size_t)h->m, k, h->st) != cudaSuccess)
        r = h->fail(cudaGetLastError());
    if (r == LOWD_OK) r = lowd_apply_splits_dev(h, d);
    cudaStreamSynchronize(h->st);
    dfree(h, &d);
    return r;
}

lowd_status lowd_get_loads(lowd_handle h, float* loads) {
    LOWD_TRY(check_handle(h));
    if (!loads) return LOWD_ERR_INVALID_ARG;
    float* l = nullptr;
    LOWD_TRY(current_loads(h, &l));
    lowd_status r = to_caller(h, loads, l, (size_t)h->n);
    if (r == LOWD_OK) {
        cudaError_t e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) r = h->fail(e);
    }
    dfree(h, &l);
    return r;
}

lowd_status lowd_get_prune_info(lowd_handle h, int32_t* sort_perm, int32_t* removal_round) {
    LOWD_TRY(check_handle(h));
    if (!h->pruned) return LOWD_ERR_BAD_STATE;
    LOWD_TRY(to_caller(h, sort_perm, h->sort_perm, (size_t)h->n0));
    LOWD_TRY(to_caller(h, removal_round, h->removal_round, (size_t)h->n0));
    return LOWD_OK;
}

lowd_status lowd_get_edge_order(lowd_handle h, int32_t* perm, int32_t* class_offsets, int32_t* classes) {
    LOWD_TRY(check_handle(h));
    if (!h->inited) return LOWD_ERR_BAD_STATE;
    if (perm) {
        int32_t* d = nullptr;
        LOWD_TRY(dalloc(h, &d, h->m));
        lowd_status r = lowd_sweep_edge_order(h, d);
        if (r == LOWD_OK) r = to_caller(h, perm, d, (size_t)h->m);
        cudaStreamSynchronize(h->st);
        dfree(h, &d);
        LOWD_TRY(r);
    }
    LOWD_TRY(to_caller(h, class_offsets, h->coff_real, (size_t)h->C + h->star_S + 1));
    if (classes) *classes = h->C + h->star_S;
    return LOWD_OK;
}

void lowd_free(lowd_handle h) {
    if (!h) return;
    cudaStreamSynchronize(h->st);
    free_all(h);
    delete h;
}

}  // extern "C"
