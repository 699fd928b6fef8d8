/*
 * qqa.h -- C ABI of libqqa, the GB300 (sm_103a) implementation of the
 * per-step replica update of Parallel Quasi-Quantum Annealing (PQQA;
 * Ichikawa & Arai, arXiv 2409.02135).
 *
 * What one annealing step computes, for every node i and replica s of every
 * instance (Sec. 3.2-3.4, Sec. 5 "Implementation", App. C.2-C.3, App. D.1):
 *   g   = d l^/dp  (MIS Eq. 22, max-clique Eq. 24, max-cut Eq. 26; A p by CSR SpMM)
 *       + gamma_t * d s/dp           alpha-entropy, Eq. 7; gamma_t linear (App. C.2)
 *       - alpha (p - mean_i)/STD_i   communication term of Eq. 10
 *   p  <- AdamW(p, g) + sqrt(2 lr T) xi,  then clamp to [0, 1]   (Eq. 11, Sec. 3.4)
 * and every `round_every` steps (and at the end) the projection rounding
 * x = [p > 1/2] with the exact integer cost and feasibility of every replica
 * (Sec. 5 "Implementation").
 *
 * Conventions shared by every entry point:
 *   - Return value: QQA_OK (0) or a negative QQA_E* code; qqa_last_error()
 *     then holds a message for the calling thread.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Calls are
 *     stream-ordered; entry points that return host data synchronise it.
 *   - Host arrays passed in are copied; the caller keeps ownership. Host
 *     output arrays are allocated by the caller. Device memory is owned by
 *     the library and comes from `alloc` when given, else cudaMalloc.
 *   - Replica state is node-major: element (i, s) at i*S + s.
 *   - Objective convention: maximisation units (independent-set size, cut
 *     weight, clique size). `energy` is the penalised minimisation energy
 *     l(x) of Eq. 2 with penalty lambda.
 *   - Nothing here falls back to the CPU: without a usable CUDA device every
 *     call that touches the GPU returns QQA_ECUDA.
 */
#ifndef QQA_H
#define QQA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QQA_OK 0
#define QQA_EINVAL (-1)     /* bad argument or malformed graph */
#define QQA_ENOMEM (-2)     /* device or host allocation failed, or over budget */
#define QQA_ECUDA (-3)      /* a CUDA call failed (message in qqa_last_error) */
#define QQA_ETIMEOUT (-4)   /* a bounded device wait ran out */
#define QQA_ENONFINITE (-5) /* a non-finite gradient or state value was produced */
#define QQA_EBUSY (-6)      /* no free slot / request not finished */

typedef enum { QQA_MIS = 0, QQA_MAXCUT = 1, QQA_MAXCLIQUE = 2 } qqa_kind;
typedef enum { QQA_FP32 = 0, QQA_BF16 = 1 } qqa_precision;

/* Optional device allocator (e.g. a framework's caching allocator). It must
 * return memory aligned to at least 16 bytes (cudaMalloc and PyTorch's caching
 * allocator give 256 / 512); qqa_run_add fails with QQA_EINVAL otherwise. */
typedef struct qqa_allocator {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, void *stream, void *ctx);
    void *ctx;
} qqa_allocator;

/*
 * Hyper-parameters of one instance. Paper values (Sec. 5, App. C.2, C.3,
 * App. D.1): a_ent = 4, gamma_min = -2 (max-cut: -5, or -20 on large graphs),
 * gamma_max = 0.1, weight_decay = 0.01, temperature = 1e-3, lambda = 2,
 * lr in {1, 0.1, 0.01}. beta1/beta2/adam_eps and alpha_comm are not printed
 * in the paper; qqa_default_params fills 0.9/0.999/1e-8 and 0.1.
 */
typedef struct qqa_params {
    int32_t S;            /* replicas, 1..1024 */
    int32_t steps;        /* K: annealing steps; gamma sweeps over all K */
    int32_t round_every;  /* periodic rounding period for the history (0 = final only) */
    int32_t a_ent;        /* alpha-entropy exponent: 2, 4, 6 or 8 */
    float lr, weight_decay, beta1, beta2, adam_eps;
    float gamma_min, gamma_max;
    float alpha_comm;     /* communication strength alpha of Eq. 10 */
    float comm_eps;       /* STD_i = sqrt(var_i + comm_eps) */
    float temperature;    /* Langevin temperature T */
    float lambda;         /* penalty coefficient (MIS, clique) */
    uint64_t seed;        /* Philox key for init and noise */
    int32_t precision;    /* qqa_precision */
    int32_t reserved;
} qqa_params;

/*
 * Launch shape of the fused step kernel. Zero fields are chosen
 * automatically from the replica count, the precision and (qqa_run_create)
 * the graphs.
 *   group_lanes : lanes that share one node row (1, 2, 4, 8, 16, 32)
 *   vec_per_lane: 16-byte vectors of replicas per lane (1, 2, 4, 8)
 *     group_lanes * vec_per_lane * (4 FP32 | 8 BF16 replicas) >= S
 *   block_threads: 32..256, multiple of 32 (the staged kernel uses 256)
 *   grid_blocks : persistent grid size (tiles are walked with a stride)
 *   use_graphs  : capture chunks of steps as CUDA graphs and replay them
 *   kernel      : QQA_KERNEL_AUTO, QQA_KERNEL_DIRECT (every neighbour row
 *                 gathered from global memory), QQA_KERNEL_STAGED (chunks of
 *                 the state staged in shared memory by TMA bulk copies and
 *                 reused by all rows of a block; for dense graphs) or
 *                 QQA_KERNEL_STREAM (each thread prefetches the next row's
 *                 slices with cp.async into private shared memory; for
 *                 sparse, memory-bound graphs)
 *                 QQA_KERNEL_DENSE (S <= 256, dense graphs: the
 *                 product A.p runs on the tensor cores - tcgen05.mma on an
 *                 fp16 adjacency and two fp16 planes of p (formed from the
 *                 FP32 state, the master in BF16 runs), FP32 accumulation
 *                 in tensor memory - followed by an update kernel for the
 *                 rest of the step; needs an n_pad^2 fp16 adjacency per
 *                 instance, n_pad = n rounded up to 128; edge weights must be
 *                 exact in fp16, |w| <= 2048. A run of several instances
 *                 without long rows or max-clique instances steps them as up
 *                 to four chains of whole instances, each on a stream the run
 *                 owns, forked from the caller's stream and joined back to it
 *                 before qqa_run_steps returns its work to that stream; the
 *                 results equal those of each instance run alone)
 *                 or QQA_KERNEL_PIPE (sparse graphs: every warp bulk-copies
 *                 the next rows it owns of p, m and v into its own shared-
 *                 memory double buffer while it updates the current ones)
 *                 QQA_KERNEL_SCALAR: runs whose instances all have S = 1 (the
 *                 paper's setting for random regular graphs, Sec. 5.1) always
 *                 use it, and no other kernel: the state is one value per node,
 *                 without padding, and kernel_param lanes (4, 8, 16, 32) share
 *                 one node's neighbour list in the sparse product
 *   Rows whose degree exceeds max(64, 8 x the graph's mean degree) are updated
 *   by a separate long-row kernel launched with the gather kernels (the
 *   pipelined kernel takes their segments as work items of its own): their
 *   neighbour lists are summed in segments of 32 CSR entries by separate lane
 *   groups, then combined in segment order (FP32), so a hub of a scale-free
 *   graph does not hold up the step.
 *   kernel_param: staged: row groups per warp (2, 4, 8);
 *                 stream: neighbour rows prefetched per row (4, 8);
 *                 dense: reported MMA width (64, 128, 256);
 *                 scalar: lanes per node row in the sparse product
 */
#define QQA_KERNEL_AUTO 0
#define QQA_KERNEL_DIRECT 1
#define QQA_KERNEL_STAGED 2
#define QQA_KERNEL_STREAM 3
#define QQA_KERNEL_DENSE 4
#define QQA_KERNEL_PIPE 5
#define QQA_KERNEL_SCALAR 6
typedef struct qqa_launch_config {
    int32_t group_lanes;
    int32_t vec_per_lane;
    int32_t block_threads;
    int32_t grid_blocks;
    int32_t use_graphs;
    int32_t kernel;
    int32_t kernel_param;
    int32_t reserved;
} qqa_launch_config;

typedef struct qqa_problem qqa_problem; /* device copy of one graph */
typedef struct qqa_run qqa_run;         /* replica state of one or more instances */

/* ---------------------------------------------------------------- misc */
const char *qqa_last_error(void);
const char *qqa_version(void);
void qqa_default_params(qqa_params *out);
/* Number of kernels this library has launched in this process (graph
 * replays count every kernel node). */
uint64_t qqa_launch_count(void);
/* Number of SMs of the current device, or a negative error code. */
int qqa_device_sm_count(void);

/* ------------------------------------------------------------- problems */
/*
 * Copy a graph to the device (App. D.1: "adjacency matrix A; A_ij = edge weight").
 *   kind     : qqa_kind
 *   n        : nodes (>= 1)
 *   row_ptr  : host int32[n+1], row_ptr[0] = 0, non-decreasing
 *   col      : host int32[row_ptr[n]], each row strictly increasing, no self
 *              loops, and symmetric (j in row i <=> i in row j)
 *   w        : host int32[row_ptr[n]] edge weights (max-cut only, symmetric),
 *              or NULL for unit weights; must be NULL for MIS / max-clique
 * Errors: QQA_EINVAL for any violation above (checked on the host before any
 * copy), QQA_ENOMEM, QQA_ECUDA.
 */
int qqa_create_problem(int32_t kind, int32_t n, const int32_t *row_ptr, const int32_t *col,
                       const int32_t *w, const qqa_allocator *alloc, void *stream, qqa_problem **out);
int qqa_problem_info(const qqa_problem *p, int32_t *kind, int32_t *n, int64_t *nnz);
void qqa_destroy_problem(qqa_problem *p);

/* ----------------------------------------------------------------- runs */
/*
 * Create a run with room for `capacity` (1..65535) instances whose replica counts are at
 * most S_max, all in `precision`. No instance is active yet. The step kernel
 * layout is fixed here from (S_max, precision, cfg); cfg may be NULL.
 * Device memory of the state is allocated per instance by qqa_run_add.
 */
int qqa_run_create_empty(int32_t capacity, int32_t S_max, int32_t precision, const qqa_launch_config *cfg,
                         const qqa_allocator *alloc, void *stream, qqa_run **out);
/*
 * Add one instance: allocate X (two buffers), the FP32 master (BF16 runs),
 * AdamW moments m, v, and evaluation buffers; then draw the initial state
 * p ~ U(0,1] from Philox (seed, node, replica) and zero m, v (step t = 0).
 * The paper does not state the initial state (Sec. 3.2 starts the relaxed
 * variables in [0,1]^N); the uniform draw is this library's reading, and the
 * moments start at zero as AdamW defines them (Sec. 3.4, App. C.3).
 * The problem must outlive the run. Returns the slot index.
 * Errors: QQA_EINVAL (S > S_max, bad params), QQA_EBUSY (no free slot), QQA_ENOMEM.
 */
int qqa_run_add(qqa_run *r, const qqa_problem *prob, const qqa_params *prm, void *stream, int32_t *slot);
/*
 * Restart one slot (slot >= 0) or every active slot (slot = -1) from a fresh
 * initial state drawn with `seed` (the same draw as qqa_run_add) (step t = 0, m = v = 0, history cleared),
 * keeping its allocations. Stream-ordered; the host does not wait for the
 * device (the descriptor table is copied from host memory before it returns).
 */
int qqa_run_reset(qqa_run *r, int32_t slot, uint64_t seed, void *stream);
/* Release one instance's state; its slot becomes free. Stream-ordered. */
int qqa_run_remove(qqa_run *r, int32_t slot, void *stream);
/* create_empty(count, max S) + add() for every problem, in order (slot k = problem k). */
int qqa_run_create(qqa_problem *const *problems, const qqa_params *params, int32_t count,
                   const qqa_launch_config *cfg, const qqa_allocator *alloc, void *stream, qqa_run **out);
void qqa_run_destroy(qqa_run *r);
/* Layout actually used (after auto choices). */
int qqa_run_config(const qqa_run *r, qqa_launch_config *out);
/*
 * Autotuner: time candidate launch shapes of the fused step on a temporary
 * run of these instances and return the fastest in *out (*best_us_per_step
 * receives its time per step, may be NULL). Candidates: kernel (direct,
 * stream with 4 or 8 prefetched neighbours, staged with 2 or 4 row groups per
 * warp) x lanes per row x vectors per lane covering the largest S (at most
 * twice over) x block size. Each candidate runs a 50-step warm-up and then
 * `trial_steps` timed steps (CUDA events on `stream`). The result is cached
 * per (precision, S_max, kinds, count, node and edge totals) for the process.
 * Shapes reduce the per-node replica statistics in different orders, so keep
 * the returned shape for reproducible trajectories. Synchronises.
 */
int qqa_autotune(qqa_problem *const *problems, const qqa_params *params, int32_t count, int32_t trial_steps,
                 const qqa_allocator *alloc, void *stream, qqa_launch_config *out, float *best_us_per_step);

/*
 * Advance every active, unfinished instance by up to `nsteps` annealing steps
 * (one fused kernel launch per step; replayed from a CUDA graph when
 * use_graphs is set). An instance stops at its own `steps`. Asynchronous.
 * One step is the update of Sec. 3.2-3.4: the gradient of the relaxed energy
 * (MIS Eq. 22, max-clique Eq. 24, max-cut Eq. 26 of App. D.1) plus gamma_t
 * times the gradient of the alpha-entropy (Eq. 7, gamma_t linear over the
 * instance's steps, App. C.2) and the communication term (Eq. 10); the AdamW
 * update that replaces the gradient step of Eq. 11 (Sec. 3.4, App. C.3) with
 * the Langevin noise sqrt(2 lr T) xi; and the projection to [0, 1] (Sec. 5
 * "Implementation").
 * Errors: QQA_EINVAL (NULL run, nsteps < 0), QQA_ECUDA.
 */
int qqa_run_steps(qqa_run *r, int32_t nsteps, void *stream);
/*
 * Projection rounding and exact costs of every replica of every active
 * instance (asynchronous); appends each instance's best feasible objective to
 * its history. Results are read with qqa_run_result after qqa_run_sync.
 * The rounding x = [p > 1/2] is the step function the paper applies after
 * annealing (Sec. 5 "Implementation"); the costs are the discrete energies of
 * App. D.1 in integers (independent-set size and edges inside x, cut weight,
 * clique size and missing edges).
 */
int qqa_run_eval(qqa_run *r, void *stream);
/* Wait for the stream, copy the latest evaluation to host mirrors, and check
 * the device status word: QQA_ETIMEOUT if a bounded device wait of the staged,
 * pipelined or tensor-core step ran out (that step left its rows unchanged),
 * else QQA_ENONFINITE if a non-finite value was seen. The status word is not
 * cleared: a run that reported an error keeps reporting it. */
int qqa_run_sync(qqa_run *r, void *stream);
/*
 * Latest evaluation of one slot (after qqa_run_sync). Any pointer may be NULL.
 *   obj, viol : int64[S]   objective (max units) and violation count
 *               (MIS: edges inside x; clique: missing edges inside x; cut: 0)
 *   feasible  : uint8[S]   viol == 0
 *   energy    : double[S]  l(x) = -size + lambda*viol (MIS, clique); -cut (max-cut)
 *   best_s    : feasible replica with the largest objective, ties -> lowest s; -1 if none
 *   best_x    : uint32[ceil(n/32)] bit i%32 of word i/32 = x_i of replica best_s
 *   step      : annealing steps completed when the evaluation ran
 */
int qqa_run_result(const qqa_run *r, int32_t slot, int64_t *obj, int64_t *viol, uint8_t *feasible,
                   double *energy, int32_t *best_s, uint32_t *best_x, int32_t *step);
/*
 * Best feasible objective after each evaluation of a slot (INT64_MIN when no
 * replica was feasible) and the step count it was taken at (the periodic
 * rounding during the anneal, Sec. 5 "Implementation"). `cap` entries at
 * most; *count receives the number available. Reads host mirrors (after sync).
 */
int qqa_run_history(const qqa_run *r, int32_t slot, int32_t cap, int64_t *best_obj, int32_t *at_step,
                    int32_t *count);
/* Steps completed by a slot (host mirror, exact). */
int qqa_run_slot_step(const qqa_run *r, int32_t slot, int32_t *t);

/*
 * Whole anneal of a batch, as the paper runs it (Sec. 3.2-3.4 for the step,
 * Sec. 5 "Implementation" and App. C.2-C.3 for the schedule, the optimizer and
 * the final rounding): create the run, init, K steps with a periodic
 * evaluation every round_every steps, and a final evaluation; then
 * synchronise. The run stays alive for reading results (*out, to be released
 * with qqa_run_destroy; the problems must outlive it).
 * Errors: as qqa_run_create and qqa_run_steps; QQA_ETIMEOUT from the final
 * synchronisation destroys the run. QQA_ENONFINITE still returns the run in
 * *out, so its (clamped) results can be read.
 */
int qqa_anneal(qqa_problem *const *problems, const qqa_params *params, int32_t count,
               const qqa_launch_config *cfg, const qqa_allocator *alloc, void *stream, qqa_run **out);
/*
 * Evaluate (qqa_run_eval + qqa_run_sync) and copy the results of every active
 * slot, concatenated in slot order: obj/viol/feasible/energy have sum(S_k)
 * entries, best_s has one per slot, best_x sum(ceil(n_k/32)) words. All are
 * HOST arrays allocated by the caller; any may be NULL.
 * This is the rounding of Sec. 5 "Implementation" (x = [p > 1/2], taken from
 * the FP32 state or master) with the exact discrete costs of App. D.1; the
 * best replica is the feasible one with the largest objective, ties to the
 * lowest index. Synchronises `stream`.
 * Errors: QQA_EINVAL, QQA_ECUDA, QQA_ETIMEOUT; QQA_ENONFINITE after copying the
 * results.
 */
int qqa_round_eval(qqa_run *r, void *stream, int64_t *obj, int64_t *viol, uint8_t *feasible, double *energy,
                   int32_t *best_s, uint32_t *best_x);

/* --------------------------------------------------------- state / debug */
/*
 * Copy one slot's state to host FP32 arrays [n][S]: X = the state p (the FP32
 * master in BF16 runs), m, v (AdamW moments, widened from BF16 in BF16 runs),
 * and the step count t. Any array pointer may be NULL. Synchronises.
 */
int qqa_run_get_state(qqa_run *r, int32_t slot, void *stream, float *X, float *m, float *v, int32_t *t);
/*
 * Overwrite one slot's state from host FP32 arrays [n][S] (values of X must
 * lie in [0,1], m must be finite and v finite and >= 0; QQA_EINVAL otherwise)
 * and set its step count to t (0 <= t <= steps). BF16 runs
 * keep X as the FP32 master and round it (and m, v) to BF16 storage.
 * Checkpoint/resume: set_state(get_state()) continues bit-identically.
 */
int qqa_run_set_state(qqa_run *r, int32_t slot, void *stream, const float *X, const float *m, const float *v,
                      int32_t t);
/*
 * One step of every active instance that also writes the gradient g of slot
 * `slot` (all terms, before AdamW: Eq. 22/24/26 + gamma_t Eq. 7 + Eq. 10) to
 * host grad[n][S]. Synchronises.
 */
/*
 * Test hook (the paper has no counterpart): overwrite the run's device status
 * word with the given counts of non-finite values and of bounded waits that
 * ran out, so that the reporting of qqa_run_sync can be checked without
 * making a kernel fail. Synchronises.
 */
int qqa_run_debug_set_status(qqa_run *r, uint64_t nonfinite, uint64_t timeouts, void *stream);
int qqa_run_step_debug(qqa_run *r, int32_t slot, void *stream, float *grad);

/* ---------------------------------------------------------- serving */
/*
 * Continuous-batching solve server. Requests (a host CSR graph plus its
 * qqa_params) are queued on submit and admitted in arrival order while the HBM
 * budget and a free slot of the request's replica class allow; a request that
 * does not fit the budget yet is passed over by later ones that do (at most
 * 32 pumps, after which admission waits for it). Each request is charged the
 * device bytes its graph, long-row tables, carved state and tile records take,
 * each allocation rounded up to 512 bytes, and its share of the work lists;
 * each class run is charged slots_per_class x 512 + 8192 bytes of fixed
 * buffers when it is created and keeps them until qqa_server_destroy (class = S
 * rounded up to a power of two, >= 8; one run with a fixed launch shape and
 * its own stream per class). Each qqa_server_pump admits, advances every
 * class by `chunk_steps` annealing steps, or by up to 8 times that for a
 * class with that much less work per step than the largest (the classes
 * overlap on the device;
 * requests of a class share every step launch), evaluates, and retires the
 * requests that reached their own step count, freeing their slot and memory.
 * Requests therefore join and leave batches between chunks. A request's
 * results do not depend on what else is in flight (fixed shape per class).
 * Times are host steady-clock seconds. Not thread-safe: one thread drives a
 * server.
 */
#define QQA_REQ_QUEUED 0
#define QQA_REQ_RUNNING 1
#define QQA_REQ_DONE 2
#define QQA_REQ_FAILED 3
#define QQA_REQ_CANCELLED 4
typedef struct qqa_server qqa_server;
typedef struct qqa_request_info {
    int32_t state;      /* QQA_REQ_* */
    int32_t error;      /* QQA_OK or the code that failed the request (e.g. QQA_ENOMEM) */
    int32_t S, n;
    int32_t best_s;     /* best feasible replica of the final rounding, -1 if none */
    int32_t feasible;   /* feasible replicas in the final rounding */
    int64_t best_obj;   /* its objective (INT64_MIN if none / not done) */
    int64_t bytes;      /* device bytes charged to the budget */
    double t_submit, t_admit, t_done;
    int32_t evaluations;/* periodic roundings recorded (one per chunk) */
    int32_t reserved;
} qqa_request_info;
/* Device bytes of the state, evaluation buffers and graph of a request of n
 * nodes and nnz CSR entries, without the graph-dependent parts (long-row
 * tables and partial sums, history, allocation granules): an estimate for
 * capacity planning; the server charges each request its exact figure. */
int64_t qqa_request_bytes(int32_t n, int64_t nnz, int32_t S, int32_t precision, int32_t weighted);
/* chunk_steps in [1, 50]; cfg fixes the launch shape of every class (NULL = auto); alloc may be NULL. */
int qqa_server_create(int64_t hbm_budget_bytes, int32_t chunk_steps, int32_t slots_per_class, int32_t precision,
                      const qqa_launch_config *cfg, const qqa_allocator *alloc, qqa_server **out);
/* Copy the host graph and params into a new queued request. A request larger
 * than the whole budget is failed at once with QQA_ENOMEM (see poll). */
int qqa_server_submit(qqa_server *s, int32_t kind, int32_t n, const int32_t *row_ptr, const int32_t *col,
                      const int32_t *w, const qqa_params *prm, int64_t *request_id);
/* One iteration: admit, one chunk of steps per class, evaluate, retire. Synchronises. */
int qqa_server_pump(qqa_server *s, int32_t *n_running, int32_t *n_queued, int32_t *n_finished);
/* Drop a queued or running request; its slot and memory are freed. */
int qqa_server_cancel(qqa_server *s, int64_t request_id);
int qqa_server_poll(const qqa_server *s, int64_t request_id, qqa_request_info *info);
/* Final results of a finished request (any pointer may be NULL): obj/viol/
 * feasible/energy [S], best_x [ceil(n/32)], history [evaluations]. */
int qqa_server_result(const qqa_server *s, int64_t request_id, int64_t *obj, int64_t *viol, uint8_t *feasible,
                      double *energy, uint32_t *best_x, int64_t *history);
int qqa_server_stats(const qqa_server *s, int64_t *used_bytes, int32_t *classes);
void qqa_server_destroy(qqa_server *s);

/* ------------------------------------------------------ no allocation */
/*
 * Projection rounding and exact costs (the same results as qqa_round_eval) of
 * a replica state held in caller-owned device memory, using no device
 * allocation at all. The paper has no counterpart: this is for callers that
 * must not allocate device memory when they evaluate - a serving loop that
 * budgets HBM up front and cannot let a request fail on, or stall behind, an
 * allocation, or a framework that owns all device memory itself.
 *   kind, n          : problem kind and node count
 *   nnz              : row_ptr[n]
 *   row_ptr, col, w  : DEVICE CSR arrays as for qqa_create_problem (w NULL =
 *                      unit weights; max-cut only). Not validated on the host;
 *                      the kernels skip out-of-range indices instead of
 *                      reading out of bounds.
 *   S, ld, X         : DEVICE float X[n][ld], replica s of node i at i*ld + s,
 *                      1 <= S <= 1024, S <= ld
 *   lambda           : penalty coefficient of the energy
 *   obj, viol        : DEVICE int64[S]; feasible: DEVICE uint8[S];
 *   energy           : DEVICE double[S]; best_s: DEVICE int32[1]
 *                      (conventions as qqa_run_result)
 *   stream           : cudaStream_t; the call is asynchronous
 * Scratch: a static device array of a little over 4 MiB that every GPU which
 * loads the library holds until exit; n * ceil(S/32) must not exceed 1048576,
 * else QQA_EINVAL. Every call shares that array, so calls whose work overlaps
 * on the GPU race. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and keeps it for that device's CUDA context;
 * a call in a new context (after cudaDeviceReset, say) looks it up again.
 * Make a call that looks the address up before any stream capture begins.
 * Error messages: qqa_noalloc_last_error().
 */
int qqa_round_eval_noalloc(int32_t kind, int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col,
                           const int32_t *w, int32_t S, int64_t ld, const float *X, float lambda, int64_t *obj,
                           int64_t *viol, uint8_t *feasible, double *energy, int32_t *best_s, void *stream);
const char *qqa_noalloc_last_error(void);

/* ------------------------------------------------ categorical colouring */
/*
 * Categorical PQQA for graph colouring with K colours (App. B, App. C.4, and
 * the colouring problem of App. D.1 read as minimising the number of
 * conflicting edges). One instance of n nodes and S replicas; the variables
 * are W[i][k][s] in [0,1] and the relaxation is
 *   sigma_ik = W_ik / sum_k' W_ik'   (Clamp-normalise, App. C.4; 1/K for a zero row).
 * One step, for every node i, colour k and replica s:
 *   g_ik = sum_{j in N(i)} sigma_jk                      relaxed conflicts
 *        + gamma_t (-c_K a K) (K sigma_ik - 1)^(a-1)     categorical alpha-entropy s_K (App. B),
 *                                                        c_K = 1 / ((K-1)((K-1)^(a-1) + 1))
 *        - alpha (sigma_ik - mean_ik) / STD_ik           communication term of Eq. 10 per (i, k)
 *   dR/dW_ik = (g_ik - sum_k' sigma_ik' g_ik') / sum_k' W_ik'
 *   W <- AdamW(W, dR/dW) + sqrt(2 lr T) xi, then clamp to [0, 1]   (as the binary step)
 * with gamma_t on the linear schedule of App. C.2 over prm->steps steps, and
 * xi / the initial W from the binary method's Philox streams with counter row
 * i*K + k. Rounding: x_is = argmax_k sigma_iks (ties to the lowest colour);
 * the cost of a replica is its number of edges {i, j} with x_is = x_js.
 * The state lives in device memory owned by the handle: W, m, v and two
 * buffers of sigma, each n * K * ceil(S/32)*32 floats, the neighbour sums in
 * the same size (graphs of up to 1600 nodes, and dense graphs), and for dense
 * graphs of 112 to 4096 nodes (at least 5% of node pairs are edges) an fp16
 * adjacency of n_pad^2 and two fp16 planes of sigma of n_pad * K * S_pad
 * (n_pad = n rounded up to 128), which the tensor cores use for the
 * neighbour sums. FP32 only.
 */
#define QQA_COLOR_MAX_K 32
typedef struct qqa_color qqa_color;

/*
 * Create an instance and draw the initial W (U(0,1], m = v = 0, t = 0).
 *   n, row_ptr, col : HOST CSR graph, validated as for qqa_create_problem
 *                     (symmetric, sorted rows, no self-loops; unit weights)
 *   K               : colours, 2..QQA_COLOR_MAX_K
 *   prm             : S (1..1024), steps (>= 1), a_ent, lr, weight_decay,
 *                     beta1, beta2, adam_eps, gamma_min, gamma_max,
 *                     alpha_comm, comm_eps, temperature, seed; precision
 *                     must be QQA_FP32; lambda and round_every are unused
 *   stream          : cudaStream_t every later call on the handle uses
 * QQA_EINVAL for bad arguments, QQA_ENOMEM / QQA_ECUDA on device failures.
 */
int qqa_color_create(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t K, const qqa_params *prm,
                     void *stream, qqa_color **out);
void qqa_color_destroy(qqa_color *c);
/* Enqueue up to nsteps steps (fewer when the schedule ends); *done (optional)
 * receives the count. Asynchronous. */
int qqa_color_steps(qqa_color *c, int32_t nsteps, int32_t *done);
/* Wait for the stream; QQA_ENONFINITE if a step produced a non-finite moment,
 * QQA_ETIMEOUT if a bounded device wait of the tensor-core path ran out. */
int qqa_color_sync(qqa_color *c);
/* One step that also writes dR/dW of that step to the HOST array grad[n][K][S]. */
int qqa_color_step_debug(qqa_color *c, float *grad);
/* Test hook (the paper has no counterpart): overwrite the handle's device
 * counters of non-finite moments and of bounded waits that ran out, so that
 * the reporting of qqa_color_sync can be checked. Synchronises. */
int qqa_color_debug_set_status(qqa_color *c, uint64_t nonfinite, uint64_t timeouts);
/* HOST copies [n][K][S] (element ((i*K + k)*S + s)) of W, m, v (any may be
 * NULL) and the step counter. Synchronous. */
int qqa_color_get_state(qqa_color *c, float *W, float *m, float *v, int32_t *t);
/* Replace the state from HOST arrays in the same layout; W must lie in
 * [0, 1], m be finite and v >= 0 (else QQA_EINVAL); 0 <= t <= prm->steps. */
int qqa_color_set_state(qqa_color *c, const float *W, const float *m, const float *v, int32_t t);
/* Round every replica and count its conflicts: conflicts: HOST int64[S];
 * best_s: the replica with the fewest conflicts (ties: lowest s); x_all
 * (optional): HOST uint8[n][S] colours. Synchronous. */
int qqa_color_round(qqa_color *c, int64_t *conflicts, int32_t *best_s, uint8_t *x_all);
/* Shape and step counter of the handle (any pointer may be NULL). */
int qqa_color_info(const qqa_color *c, int32_t *n, int32_t *K, int32_t *S, int32_t *t);

#ifdef __cplusplus
}
#endif

#endif /* QQA_H */
