/*
 * Timing variant of the oracle's LOWD passes on all host cores.
 *
 * TEST INFRASTRUCTURE ONLY (the CPU baseline of the benchmark and its test); it is kept apart
 * from the checker functions of lowd_oracle.c and shares no code with the CUDA library.
 *
 * A pass visits colour classes in order (each class a matching: no two of its edges share
 * a node).  The edges of one class are split into equal ranges over the threads, each
 * thread applies Algorithm 1's loop body to its range, and all threads meet at a barrier
 * before the next class.  Updates inside a class touch disjoint node pairs, so the result
 * is exactly the sequential pass in the same order, in double precision.
 */
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    atomic_int count;
    atomic_int gen;
    int parties;
} spin_barrier;

static void barrier_wait(spin_barrier* b) {
    const int g = atomic_load_explicit(&b->gen, memory_order_acquire);
    if (atomic_fetch_add_explicit(&b->count, 1, memory_order_acq_rel) == b->parties - 1) {
        atomic_store_explicit(&b->count, 0, memory_order_relaxed);
        atomic_fetch_add_explicit(&b->gen, 1, memory_order_release);
    } else {
        while (atomic_load_explicit(&b->gen, memory_order_acquire) == g) {
        }
    }
}

/* Algorithm 1's loop body on edge (u, v): move weight from the heavier end to the lighter
 * one, d = min(|l_u - l_v| / 2, split held by the heavier end). */
static void update(double* lu, double* lv, double* fu, double* fv) {
    double d;
    if (*lu > *lv) {
        d = (*lu - *lv) / 2.0;
        if (*fu < d) d = *fu;
        *lu -= d; *fu -= d; *lv += d; *fv += d;
    } else {
        d = (*lv - *lu) / 2.0;
        if (*fv < d) d = *fv;
        *lu += d; *fu += d; *lv -= d; *fv -= d;
    }
}

typedef struct {
    int id, threads;
    int32_t T, C;
    const int32_t *u, *v, *order;
    const int64_t* off;
    double *fu, *fv, *l;
    spin_barrier* bar;
    atomic_int* go;   /* 0 wait, 1 run, -1 leave without work */
} job;

static void* worker(void* arg) {
    job* j = (job*)arg;
    int g;
    while ((g = atomic_load_explicit(j->go, memory_order_acquire)) == 0) {
    }
    if (g < 0) return NULL;
    for (int32_t t = 0; t < j->T; ++t) {
        for (int32_t c = 0; c < j->C; ++c) {
            const int64_t b = j->off[c], e = j->off[c + 1];
            const int64_t len = e - b;
            const int64_t lo = b + len * j->id / j->threads;
            const int64_t hi = b + len * (j->id + 1) / j->threads;
            for (int64_t i = lo; i < hi; ++i) {
                const int32_t x = j->order[i];
                update(&j->l[j->u[x]], &j->l[j->v[x]], &j->fu[x], &j->fv[x]);
            }
            barrier_wait(j->bar);
        }
    }
    return NULL;
}

/* T passes over the classes order[off[c] .. off[c+1]), c = 0..C-1, on `threads` threads.
 * Returns 0, or -1 (nothing done) if the threads could not be started. */
int orc_lowd_iterate_threads(int32_t n, int64_t m, const int32_t* u, const int32_t* v, const int32_t* order,
                             const int64_t* off, int32_t C, int32_t T, int32_t threads, double* fu, double* fv,
                             double* l) {
    (void)n; (void)m;
    if (threads < 1) threads = 1;
    spin_barrier bar;
    atomic_init(&bar.count, 0);
    atomic_init(&bar.gen, 0);
    bar.parties = threads;
    atomic_int go;
    atomic_init(&go, 0);
    job* jobs = (job*)calloc((size_t)threads, sizeof(job));
    pthread_t* tid = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tid) { free(jobs); free(tid); return -1; }
    for (int i = 0; i < threads; ++i) jobs[i] = (job){i, threads, T, C, u, v, order, off, fu, fv, l, &bar, &go};
    int started = 0;
    for (int i = 1; i < threads; ++i) {
        if (pthread_create(&tid[i], NULL, worker, &jobs[i]) != 0) break;
        ++started;
    }
    const int ok = started == threads - 1;
    atomic_store_explicit(&go, ok ? 1 : -1, memory_order_release);
    if (ok) worker(&jobs[0]);
    for (int i = 1; i <= started; ++i) pthread_join(tid[i], NULL);
    free(jobs);
    free(tid);
    return ok ? 0 : -1;
}
