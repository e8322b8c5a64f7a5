/*
 * lowd.h - C ABI of a GB300 (sm_103a) implementation of LOWD, the Locally Optimal
 * Weight Distribution method for the edge-density densest subgraph problem
 * (arXiv 2307.15969), with its pruning pre-process and its extraction step.
 *
 * The method (paper notation): an undirected graph G(V, E, W) with positive edge
 * weights w_e.  Every edge e = (u, v) splits its weight between its ends,
 * f_e(u) + f_e(v) = w_e, f >= 0; a node's load is l_u = sum of f_e(u) over its edges
 * (tighter dual, Sec. III-B).  LOWD (Algorithm 1) starts from the equal split and
 * repeatedly moves weight across each edge from the more loaded end to the less loaded
 * one, as far as the split allows; the loads converge to the locally-dense
 * decomposition (Theorem 2), and peeling nodes by load recovers the densest subgraph.
 * Pruning (Algorithm 2) first removes every node whose degree is below the current
 * density, in rounds, which keeps the densest subgraph (Theorem 3).
 *
 * Calls, in the order of the method:
 *   lowd_load_graph   graph in, canonicalised on the GPU           (Sec. II, Sec. IV data)
 *   lowd_prune        Algorithm 2's pruning loop                   (Sec. III-D, Alg. 2)
 *   lowd_iterate      k passes of Algorithm 1's edge loop          (Alg. 1, Sec. III-A)
 *   lowd_extract      sort by load, best prefix density            (Alg. 1 extraction)
 *
 * Conventions (all calls):
 *   - Every call returns a lowd_status; nothing is thrown or aborted across the ABI.
 *     After an error the handle stays valid and can still be freed.
 *   - All GPU work runs on the CUDA stream given to lowd_load_graph (NULL = legacy
 *     default stream).  A call that writes host memory synchronises that stream before
 *     it returns; calls that write only device memory return without synchronising.
 *   - Pointer arguments are host pointers unless the handle was created with
 *     LOWD_MEM_DEVICE, in which case array arguments (inputs and outputs, never the
 *     scalar out-parameters such as n_kept or stats) are device pointers.
 *   - The handle owns all its device memory (allocated by load_graph and freed by
 *     lowd_free).  The caller owns every array it passes.
 *   - Edge ids, node ids and sizes are 32-bit: n < 2^31 and m < 2^31.
 *   - One handle must not be used by two host threads at once.
 */
#ifndef LOWD_H
#define LOWD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lowd_ctx* lowd_handle;

typedef enum {
    LOWD_OK = 0,
    LOWD_ERR_INVALID_ARG = 1,     /* bad size, null pointer, self-loop, id out of range,
                                     non-positive / non-finite weight */
    LOWD_ERR_OUT_OF_MEMORY = 2,   /* device allocation failed */
    LOWD_ERR_CUDA = 3,            /* any other CUDA runtime error (message kept per handle) */
    LOWD_ERR_BAD_STATE = 4,       /* call out of order, e.g. lowd_prune after lowd_iterate */
    LOWD_ERR_NOT_CONVERGED = 5,   /* rel_tol > 0 was not met within k passes (state valid) */
    LOWD_ERR_INEXACT_WEIGHTS = 6, /* a weight is not a multiple of 2^-20 (see lowd_load_graph) */
    LOWD_ERR_TOO_LARGE = 7        /* a size exceeds a documented limit of the call */
} lowd_status;

enum { LOWD_MEM_HOST = 0, LOWD_MEM_DEVICE = 1 };

/* Load-time flags (bit set). */
enum {
    LOWD_LOAD_ALLOW_INEXACT = 1   /* accept weights off the 2^-20 grid: they are rounded to it
                                     for pruning and extraction sums, kept as given for LOWD */
};

/* Options of lowd_iterate; a zero-initialised struct gives the defaults. */
typedef struct {
    int32_t check_every;  /* >0: every check_every passes, re-derive the loads from the
                             splits in FP64 and evaluate the stop test (default 0: no checks) */
    double  rel_tol;      /* >0: stop once (D - rho(S))/rho(S) <= rel_tol at a check, where
                             D = max load (an upper bound on rho*, Sec. III-B) and S the
                             best prefix of the load order (default 0: run all k passes) */
    int32_t schedule;     /* 0 = automatic; 1 = one-CTA shared-memory sweep (node count
                             must fit shared memory); 2 = grid sweep over matchings */
    int32_t rederive_every; /* re-derive the FP32 loads from the splits (FP64 sums) after at
                             most this many passes, bounding the drift of the running FP32
                             loads: 0 = default 50, < 0 = only at the end of the call */
    int32_t node_versions; /* 1: the one-CTA staged sweep replaces its barrier after every
                             colour class by per-node versions (kernel 5: an update waits only
                             for the previous updates of its two nodes); same pass as kernel 1.
                             Default 0 (kernel 1: on dense cores whose hubs appear in every
                             class it is faster, as waiting warps sleep at the barrier) */
    int32_t hub_stars;    /* hub-star block updates (read when the schedule is built, i.e. by
                             the first lowd_iterate of a graph; a schedule built earlier by
                             lowd_set_splits or lowd_warm_start has none): 0 = off (default); 1 =
                             automatic threshold; t >= 2 = threshold.  Nodes of (unweighted)
                             degree >= t are hubs; an edge with exactly one hub end is a star
                             edge.  A pass runs Algorithm 1 over the other edges in the
                             schedule's own order of their subgraph (circle colouring or
                             level order), then the star steps: the star edges of each leaf
                             are ranked by hub degree (descending) then hub id, and step k
                             holds every leaf's k-th star edge, grouped by hub into
                             vertex-disjoint stars.  Each star's splits become the exact
                             minimiser of the sum of squared loads over them, all else fixed
                             (Sec. III-C's local optimality over a block of edges; a one-leaf
                             star is Algorithm 1's update), so sum l^2 still never rises and
                             the loads converge to the same optimum.  The automatic threshold:
                             schedule 1, the smallest power of two >= half the maximum degree
                             (the near-universal nodes: the fewest steps for the stars' faster
                             descent); schedule 2, the smallest power of two 2^k (k >= 1) with
                             at most 2^(k-1) nodes of degree >= 2^k (also takes the hubs' edges
                             out of the level order).  lowd_get_edge_order then lists the plain
                             classes, then one block per star step; lowd_info reports the
                             threshold, steps, stars and star edges */
} lowd_options;

/* Statistics of the state after lowd_iterate (FP64, from loads re-derived from the
 * splits when a check ran, else from the FP32 loads). */
typedef struct {
    int32_t iters_done;   /* total passes run on this handle so far */
    int32_t checks_done;  /* checks evaluated by this call */
    double  sum_load;     /* sum of l (equals the total edge weight, Sec. III-B) */
    double  sum_load_sq;  /* sum of l^2, the QP objective of Sec. III-C */
    double  max_load;     /* D = max l, an upper bound on rho* (Sec. III-B) */
    double  rho_best;     /* density of the best load-ordered prefix at the last check */
    int32_t best_size;    /* its size */
    int32_t converged;    /* 1 if rel_tol was met */
} lowd_stats;

/* Sizes of the current graph and of its conflict-free schedule. */
typedef struct {
    int32_t n_orig;       /* nodes of the loaded graph G */
    int32_t n;            /* nodes of the current graph (G, or H after lowd_prune) */
    int64_t m_orig;       /* edges of G after canonicalisation */
    int64_t m;            /* edges of the current graph */
    int64_t duplicates;   /* input pairs dropped as repeats by lowd_load_graph */
    int32_t weighted;     /* 1 if weights were given */
    int32_t pruned;       /* 1 after lowd_prune */
    int32_t classes;      /* colour classes of the schedule (0 before lowd_iterate) */
    int32_t schedule;     /* schedule in use: 1 one-CTA shared memory, 2 grid matchings */
    int32_t max_degree;   /* maximum (unweighted) degree of the current graph */
    int32_t prune_rounds; /* rounds lowd_prune ran */
    int32_t sweep_kernel; /* kernel of the last pass: 0 none yet, 1 staged one-CTA sweep with
                             pair loads and a barrier per class, 2 one-CTA register-ring sweep,
                             3 one-CTA simple sweep, 4 streamed sweep (schedule 2, loads in
                             global memory), 5 staged one-CTA sweep with pair loads and
                             per-node versions instead of class barriers */
    int32_t sweep_edges_per_thread; /* edges per consumer thread per class of kernel 1 */
    int32_t star_threshold; /* hub degree threshold of the hub stars in use (0: none) */
    int32_t star_steps;     /* star steps per pass (the last star_steps entries of classes) */
    int32_t stars;          /* stars over all steps */
    int64_t star_edges;     /* star edges (the rest, m - star_edges, run Algorithm 1) */
} lowd_info;

/*
 * lowd_load_graph - build a handle on the undirected graph G(V, E, W) of Sec. II.
 *   n        number of nodes, ids 0..n-1 (1 <= n < 2^31)
 *   m        number of input pairs (0 <= m < 2^31)
 *   u, v     endpoint arrays [m]; direction is ignored, repeated pairs are merged
 *            keeping the first occurrence's weight (the paper removes multiple edges
 *            and self-loops from its datasets, Sec. IV); a self-loop (u == v) or an id
 *            outside [0, n) is rejected with LOWD_ERR_INVALID_ARG
 *   w        weights [m] (> 0, finite), or NULL for unit weights (unweighted graph)
 *   mem      LOWD_MEM_HOST or LOWD_MEM_DEVICE: where u, v, w and every later array
 *            argument of this handle live
 *   flags    0 or LOWD_LOAD_ALLOW_INEXACT
 *   stream   cudaStream_t (as void*) on which all work of this handle runs
 *   out      receives the handle (NULL on error)
 * Weights must be multiples of 2^-20 (they are then exact FP32 values and every
 * degree, W(H) and prefix weight is an exact 64-bit integer), else
 * LOWD_ERR_INEXACT_WEIGHTS unless LOWD_LOAD_ALLOW_INEXACT is set.
 * Inputs are copied; the caller may free them when the call returns.
 */
lowd_status lowd_load_graph(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                            const float* w, int32_t mem, int32_t flags, void* stream,
                            lowd_handle* out);

/*
 * lowd_prune - Algorithm 2's pruning loop (Sec. III-D): delta = rho(H) = W(H)/|H|;
 * remove, all at once, every node u of H with d_H(u) < delta (strict, exact integer
 * test d_H(u)*|H| < W(H)) and its edges; repeat until no node is removed.  d_H is the
 * weighted degree for weighted graphs.  The nodes are first ordered by degree with a
 * counting sort (Sec. III-D); lowd_get_prune_info returns that order.  Afterwards the
 * handle's current graph is H: survivors renumbered by ascending original id, edges
 * kept in their original order.  Must be called before lowd_iterate (else
 * LOWD_ERR_BAD_STATE); may be called once.
 *   n_kept, m_kept, rounds   host out-parameters (may be NULL)
 */
lowd_status lowd_prune(lowd_handle h, int32_t* n_kept, int64_t* m_kept, int32_t* rounds);

/*
 * lowd_iterate - k passes of Algorithm 1's edge loop (its lines after the
 * initialisation) over the current graph.  The first call initialises
 * f_e(u) = f_e(v) = w_e/2 and the loads (Algorithm 1's first loops) and builds the
 * conflict-free schedule: a proper edge colouring, so every colour class is a matching
 * and updating its edges in parallel equals updating them one after another.  A pass
 * visits the classes in order; lowd_get_edge_order gives the resulting edge order.
 *   k     number of passes (>= 0)
 *   opt   options (NULL = defaults)
 *   st    host out-parameter (may be NULL)
 * Returns LOWD_ERR_NOT_CONVERGED only when opt->rel_tol > 0 and it was not met; the
 * state is valid and a further call continues the run.
 */
lowd_status lowd_iterate(lowd_handle h, int32_t k, const lowd_options* opt, lowd_stats* st);

/*
 * lowd_extract - Algorithm 1's extraction: order the current graph's nodes by load
 * (ascending, ties by id), peel them from the lowest, and keep the densest set seen,
 * replacing it only on a strictly higher density (so ties keep the larger set); the
 * empty set is not a candidate.  Prefix weights are exact integers (2^-20 units), the
 * comparison is exact.  Valid at any time after lowd_load_graph (before any pass the
 * loads are the equal-split loads).
 *   S        out: ids of S* in ORIGINAL numbering, ascending; capacity >= n_orig; may be NULL
 *   S_size   host out: |S*|
 *   rho      host out: W(S*)/|S*| as a double
 *   loads    out [n_orig]: FP32 load of every original node; nodes removed by pruning
 *            get 0; may be NULL
 */
lowd_status lowd_extract(lowd_handle h, int32_t* S, int32_t* S_size, double* rho, float* loads);

/* ------------------------------------------------------------------ state and parity hooks */

/*
 * lowd_get_ldd - the locally-dense decomposition read off the current loads (Sec. II,
 * Definition of LDD; Properties 1-2: the nodes of B_i \ B_{i-1} all carry load lambda_i,
 * lambda_1 > lambda_2 > ...).  Nodes of the current graph are ordered by load descending
 * (ties by id descending); a shell ends where the next load is lower by more than
 * rel_tol times the current one.  lambda_i = (W(B_i) - W(B_{i-1})) / |B_i \ B_{i-1}| is
 * computed exactly from integer prefix weights, so on converged loads it is the exact shell
 * density whenever the shells are separated by more than the loads' error.  B_1 with
 * lambda_1 is the maximal densest subgraph; Corollary 1's bounds for the densest
 * k-subgraph follow from (shell_end, lambda).
 *   shell      out [n_orig]: 1-based shell of each original node; 0 for pruned nodes
 *   lambda     out [capacity n]: lambda_i per shell
 *   shell_end  out [capacity n]: |B_i| (shell i covers sorted positions shell_end[i-1]..)
 *   n_shells   host out: number of shells
 * Any of shell / lambda / shell_end may be NULL.
 */
lowd_status lowd_get_ldd(lowd_handle h, double rel_tol, int32_t* shell, double* lambda,
                         int32_t* shell_end, int32_t* n_shells);

/*
 * lowd_ldd_dks_bound - Corollary 1 on an exported decomposition: the upper bound on the
 * density of any k-node subgraph (DkS) and of any subgraph with at least k nodes (DalkS)
 * of the graph the decomposition was taken on.  With |B_{j-1}| < k <= |B_j|,
 *     bound = (W(B_{j-1}) + (k - |B_{j-1}|) * lambda_j) / k,
 * W(B_{j-1}) = sum_{i<j} lambda_i * |B_i \ B_{i-1}|: the mean of the k largest loads (the
 * corollary's proof bounds W(S) by the loads of S; its sum over lambda_i * |B_i| counts
 * each shell's own nodes, |B_i \ B_{i-1}|).  For k = |B_j| the bound is attained by B_j
 * (Corollary 1, item 1) and *exact is set to 1.  Host arithmetic, no GPU work.
 *   n_shells, shell_end, lambda   host arrays as returned by lowd_get_ldd
 *   k          1 <= k <= shell_end[n_shells - 1], else LOWD_ERR_INVALID_ARG
 *   bound      host out; exact: host out (may be NULL)
 * Taken after lowd_prune, the decomposition and the bound are those of the pruned graph.
 */
lowd_status lowd_ldd_dks_bound(int32_t n_shells, const int32_t* shell_end, const double* lambda, int32_t k,
                               double* bound, int32_t* exact);

/* Current graph sizes and schedule.  info: host pointer. */
lowd_status lowd_get_info(lowd_handle h, lowd_info* info);

/* Current graph's edges in the handle's canonical order (lo < hi; sorted by (lo, hi)
 * for G, original order for H), ids in the current numbering.  u, v: [m]; w: [m] or
 * NULL (unit weights give 1). */
lowd_status lowd_get_graph(lowd_handle h, int32_t* u, int32_t* v, float* w);

/* Splits s_e = f_e(lo) of every current edge (f_e(hi) = w_e - s_e), in the canonical
 * edge order: get [m] out, set [m] in (values are clamped to [0, w_e] and the loads are
 * recomputed from them; used for checkpoints and warm starts).  Before the first
 * lowd_iterate, get returns the equal split and set initialises from the given split. */
lowd_status lowd_get_splits(lowd_handle h, float* s);
lowd_status lowd_set_splits(lowd_handle h, const float* s);

/* Current loads [n] (current numbering). */
lowd_status lowd_get_loads(lowd_handle h, float* loads);

/* Pruning details, original numbering: sort_perm [n_orig] = nodes ordered by degree
 * ascending, ties by id (the counting sort); removal_round [n_orig] = 1-based round in
 * which the node was removed, -1 if kept.  Either may be NULL.  LOWD_ERR_BAD_STATE
 * before lowd_prune. */
lowd_status lowd_get_prune_info(lowd_handle h, int32_t* sort_perm, int32_t* removal_round);

/* The schedule: perm [m] lists the canonical edge ids in the order a pass updates them
 * (class by class; inside a class by edge id); class_offsets [classes + 1].  Either may
 * be NULL.  *classes (host) receives the class count.  LOWD_ERR_BAD_STATE before the
 * first lowd_iterate. */
lowd_status lowd_get_edge_order(lowd_handle h, int32_t* perm, int32_t* class_offsets,
                                int32_t* classes);

/*
 * lowd_extract_noalloc - the extraction of lowd_extract on caller-provided DEVICE arrays,
 * without any device allocation.  The paper has no counterpart: this is a service for
 * callers that cannot let a library allocate device memory - for example a process whose
 * device memory belongs to its own pool allocator, or a loop with a fixed memory budget
 * that cannot absorb the device-wide synchronisation cudaMalloc/cudaFree may cause.
 *   n, m       nodes (1 <= n <= 65536) and edges (0 <= m < 2^31)
 *   u, v       device int32 [m]: edge ends, each pair listed once, ids in [0, n), u != v
 *   w          device float [m] weights, or NULL for unit weights; each weight must be
 *              positive and finite and counts as its nearest multiple of 2^-20 (at least
 *              2^-20), as in lowd_load_graph; it must also stay below 2^62 / m units of
 *              2^-20 so that the prefix sums are exact 64-bit integers
 *   loads      device float [n]: node loads (e.g. from lowd_get_loads)
 *   S          device int32 [n] out: ids of S* ascending, or NULL
 *   S_size     host out: |S*|;   rho   host out: W(S*)/|S*|
 *   stream     cudaStream_t (as void*); the call synchronises it before returning
 * Returns LOWD_ERR_TOO_LARGE when n > 65536 and LOWD_ERR_INVALID_ARG on bad arguments.
 * The arrays are checked on the GPU: an edge with an id outside [0, n), a self-loop or a
 * weight outside the rules above is skipped (never read past the arrays) and the call
 * returns LOWD_ERR_INVALID_ARG; S, S_size and rho are then not valid.
 * All intermediate buffers come from one static device array of 4 MiB that every GPU
 * which loads this library holds until the process exits.  Its device address is looked
 * up (cudaGetSymbolAddress) on the first call made on each device, with that device
 * current; make that first call before capturing any stream.  The array is shared by all
 * calls and keeps the previous call's contents, so calls that overlap on the GPU (other
 * streams, other host threads) race with each other: serialise them.
 */
lowd_status lowd_extract_noalloc(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                                 const float* w, const float* loads, int32_t* S, int32_t* S_size,
                                 double* rho, void* stream);

/* ------------------------------------------------------------------ batched graphs
 *
 * Many independent graphs through the whole method (Algorithm 2, colouring, Algorithm 1
 * passes, extraction) in one persistent kernel launch, replayed from a captured CUDA
 * graph.  Each CTA takes graphs from a work queue and runs one graph at a time with its
 * node state in shared memory.  Unit weights only.
 */
typedef struct lowd_batch_ctx* lowd_batch;

enum { LOWD_BATCH_ORDER_AS_GIVEN = 1, LOWD_BATCH_ORDER_LARGEST_FIRST = 2 };

/* Launch schedule of lowd_batch_run; zero fields take the autotuned (or default) value. */
typedef struct {
    int32_t passes;       /* LOWD passes per graph (>= 0) */
    int32_t ctas_per_sm;  /* 1 to 4 (shared memory is split between them) */
    int32_t threads;      /* threads per CTA: multiple of 32 in [64, 1024] */
    int32_t order;        /* LOWD_BATCH_ORDER_* : order in which graphs enter the queue */
} lowd_batch_options;

/*
 * lowd_batch_create - copy a batch of B graphs and check it.
 *   node_off [B+1], edge_off [B+1]  prefix offsets (node_off[0] = edge_off[0] = 0), host
 *                                   or device per `mem`; every graph has >= 1 node
 *   u, v [edge_off[B]]             local node ids of each graph's edges: u < v < n_g and
 *                                   strictly increasing (u, v) inside a graph (the canonical
 *                                   form of Sec. IV: no loops, no repeats)
 * Graphs whose node count exceeds the kernel's shared-memory budget (about 45,000 nodes
 * at one CTA per SM) are reported with status 1 by lowd_batch_results instead of a result.
 *   stream    cudaStream_t (as void*) for all work of the batch; NULL makes the batch use a
 *             non-blocking stream of its own (the launch is captured into a CUDA graph, which
 *             the legacy default stream does not allow)
 */
lowd_status lowd_batch_create(int32_t B, const int64_t* node_off, const int64_t* edge_off,
                              const int32_t* u, const int32_t* v, int32_t mem, void* stream,
                              lowd_batch* out);

/* Run the method on every graph (Algorithm 2, then Algorithm 1 with opt->passes passes,
 * then the extraction).  The first run with a given schedule captures it in a CUDA graph;
 * later runs replay it.  Synchronises the stream. */
lowd_status lowd_batch_run(lowd_batch b, const lowd_batch_options* opt);

/* Time every schedule (graph order x CTAs per SM x threads) on a spread sample of `sample`
 * graphs (0 = all) at `passes` passes; keep the fastest as the default and return it. */
lowd_status lowd_batch_autotune(lowd_batch b, int32_t passes, int32_t sample, lowd_batch_options* best);

/* Per-graph results of the last run, all arrays optional, host or device per `mem`:
 * rho [B] (W(S*)/|S*|), S_size [B], in_S [node_off[B]] (1 if the node is in S*, by local
 * id), n_core / m_core [B] (size of the pruned graph), rounds [B] (pruning rounds),
 * status [B] (0 ok, 1 too many nodes, 2 pruned core too large for the extraction, 3 an
 * internal edge-id check failed, 4 a bounded wait of the staged passes expired; 3 and 4
 * mark a defect, the graph's result is not valid). */
lowd_status lowd_batch_results(lowd_batch b, double* rho, int32_t* S_size, uint8_t* in_S,
                               int32_t* n_core, int32_t* m_core, int32_t* rounds, int32_t* status);

/* FP32 load of every node after the last run's passes, by local id, host or device per
 * `mem`: loads [node_off[B]]; 0 for nodes removed by Algorithm 2 and for graphs with a
 * nonzero status.  Inside each graph the passes visit the core's colour classes (the
 * circle colouring of the core, ids renumbered ascending) in ascending colour. */
lowd_status lowd_batch_loads(lowd_batch b, float* loads);

/* Core membership after the last run, by local id, host or device per `mem`: in_core
 * [node_off[B]] = 1 if the node survived Algorithm 2 (0 as well for graphs with a nonzero
 * status).  With lowd_batch_loads this gives each graph's pruned core and its loads. */
lowd_status lowd_batch_core(lowd_batch b, uint8_t* in_core);

/* Text of the last CUDA error seen by this batch ("" if none). */
const char* lowd_batch_last_error(lowd_batch b);

void lowd_batch_free(lowd_batch b);

/* ------------------------------------------------------------------ learned warm start
 *
 * Not in the paper: the paper starts every edge at the equal split f_e(u) = f_e(v) = w_e/2
 * (Algorithm 1's initialisation).  Any split inside [0, w_e] is a valid start - the
 * convergence argument of Theorem 2 does not depend on it - so a start closer to the
 * optimum only saves passes; the passes, the stop test and the extraction are unchanged.
 * The predictor is a mean-aggregation message-passing network (hidden width 64, three
 * layers; BF16 node states and layer weights, FP32 accumulation, the layer products on the
 * tensor cores) on the graph the passes run on:
 *   x_v   = (log(1 + d_v), mean of log w_e over v's edges, log(1 + sum of the neighbours'
 *            d)), d_v = weighted degree
 *   h0    = relu(x W_in + b_in);  per layer: m_v = mean of h over v's neighbours,
 *           h' = relu([h, m] W_l^T + b_l)
 *   phi_v = q . h3_v;  sigma_e = 1 / (1 + exp(phi_hi - phi_lo));  f_e(lo) = sigma_e w_e
 * Training loss (lowd_mpnn_forward with a target): sum_v (l_v - t_v)^2 / sum_v t_v^2,
 * l_v the loads of the predicted splits, t_v target loads (converged LOWD loads).
 * Flat FP32 parameter vector of lowd_mpnn_param_count() entries: W_in [3][64] (row-major
 * [in][out]), b_in [64], then per layer W_l [64][128] ([out][in]) and b_l [64], then q [64].
 */
typedef struct lowd_mpnn_ctx* lowd_mpnn;

enum { LOWD_MPNN_SIGMA = 1, LOWD_MPNN_LOADS = 2, LOWD_MPNN_GRAD = 3, LOWD_MPNN_FEATURES = 4, LOWD_MPNN_PHI = 5 };

int64_t lowd_mpnn_param_count(void);

/* A network with all parameters 0 (every predicted split is the equal split) and its own
 * device state; stream as in lowd_batch_create (NULL: a non-blocking stream of its own). */
lowd_status lowd_mpnn_create(void* stream, lowd_mpnn* out);

/* Copy the FP32 parameters in (host or device per mem); resets the Adam state. */
lowd_status lowd_mpnn_set_params(lowd_mpnn net, const float* params, int32_t mem);
lowd_status lowd_mpnn_get_params(lowd_mpnn net, float* params, int32_t mem);

/* Bind a graph (copied): n nodes, m edges lo[e] < hi[e] < n, each pair once; w [m] > 0 or
 * NULL for unit weights; target [n] loads or NULL.  Builds the adjacency and the input
 * features.  m < 2^30.  LOWD_ERR_INVALID_ARG on an edge or weight outside these rules. */
lowd_status lowd_mpnn_bind(lowd_mpnn net, int32_t n, int64_t m, const int32_t* lo, const int32_t* hi,
                           const float* w, const float* target, int32_t mem);

/* Replace the bound graph's input features by caller-provided ones, x [3n] (node-major,
 * three per node), host or device per mem; kept until the next bind. */
lowd_status lowd_mpnn_set_features(lowd_mpnn net, const float* x, int32_t mem);

/* Forward pass on the bound graph: splits sigma, their loads and, with a target, the loss
 * (loss may be NULL; a non-NULL loss without a target is LOWD_ERR_BAD_STATE). */
lowd_status lowd_mpnn_forward(lowd_mpnn net, double* loss);

/* Gradient of the loss of the last forward pass with respect to every parameter. */
lowd_status lowd_mpnn_backward(lowd_mpnn net);

/* One Adam step (bias-corrected, step counter kept by the network) with the last gradient. */
lowd_status lowd_mpnn_adam(lowd_mpnn net, float lr, float beta1, float beta2, float eps);

/* Read LOWD_MPNN_SIGMA [m], LOADS [n], PHI [n] (after a forward pass), FEATURES [3n] (after
 * bind) or GRAD [param_count] into out (host or device per mem). */
lowd_status lowd_mpnn_read(lowd_mpnn net, int32_t what, float* out, int32_t mem);

/* Warm start of a handle: the network's splits on the handle's current graph (G, or H
 * after lowd_prune) become the LOWD state, s_e = sigma_e w_e; before the first lowd_iterate
 * this replaces the equal split, later it replaces the current splits (loads re-derived). */
lowd_status lowd_warm_start(lowd_handle h, lowd_mpnn net);

const char* lowd_mpnn_last_error(lowd_mpnn net);
void lowd_mpnn_free(lowd_mpnn net);

/* Release the handle and all its device memory.  NULL is ignored. */
void lowd_free(lowd_handle h);

/* Static text for a status code. */
const char* lowd_status_string(lowd_status s);

/* Text of the last CUDA error seen by this handle ("" if none). */
const char* lowd_last_error(lowd_handle h);

/* Number of CUDA kernels this library has launched in this process so far (all handles,
 * all threads).  A diagnostic for benchmarks; it has no counterpart in the paper. */
uint64_t lowd_launch_count(void);

/* Failure-detection self-test of the bounded grid barrier that the cooperative kernels (grid
 * steps of the streamed schedule, star steps, level colouring) meet at between steps: two
 * blocks are launched on a barrier that expects three, so nothing opens it; with a short spin
 * limit the wait must expire, set bit 1 (value 2) of the kernel's error word and end the
 * kernel.  *err_bits receives that word; returns LOWD_OK once the kernel has ended (the
 * context stays usable), LOWD_ERR_INVALID_ARG for a NULL err_bits, LOWD_ERR_OUT_OF_MEMORY or
 * LOWD_ERR_CUDA if it could not run.  Uses the default stream.  No counterpart in the paper. */
lowd_status lowd_selftest_barrier_timeout(int32_t* err_bits);

#ifdef __cplusplus
}
#endif
#endif /* LOWD_H */
