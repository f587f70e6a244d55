/*
 * flexiwalk.h -- C ABI of a GB300 (sm_103a) engine for the per-step
 * transition sampling of dynamic random walks, after FlexiWalker
 * (Park et al., EuroSys '26, arXiv 2512.00705).
 *
 * The method (paper sections in brackets):
 *   - Every walker at node v with previous node v' draws its next node u
 *     from N(v) with probability w~(v,u) / sum_t w~(v,t), where
 *     w~ = w * h: h is the edge property weight and w the runtime weight
 *     of the walk algorithm  [Sec. 2.1, Eq. (prob)].
 *       node2vec : w = 1/p if u = v', 1 if u in N(v'), 1/q otherwise
 *                  [Eq. (node2vec); the paper writes a, b for p, q]
 *       metapath : w = 1 if label(v,u) = schema[hop mod S], else 0  [Sec. 2.1]
 *       weighted : w = 1  (static walk)  [Sec. 2.1]
 *   - The draw is made by eRJS (rejection against the on-the-fly bound
 *     B = max(w) * h_MAX[v], [Sec. 3.3]) or by eRVS (single-pass reservoir
 *     sampling with exponential keys and jumps, [Sec. 3.2, Alg. 1,
 *     Eq. (jump)]); a first-order cost model picks eRJS iff
 *     r * B < sum-hat, with sum-hat = h_SUM[v] * mean(w)
 *     [Sec. 4.1, Eq. (runtime), Eq. (sum_estimation)].
 *   - An exact inverse-CDF mode (FP32 prefix in neighbour order, one
 *     Philox4x32-10 uniform per hop) reproduces a plain CPU definition bit
 *     for bit; it is the parity mode, not a fast path [Sec. 2.2, ITS].
 *
 * Conventions for every entry point:
 *   - Status codes are returned, never aborts; fw_last_error() gives a
 *     thread-local message for the last failing call of this thread.
 *   - "device" pointers are CUDA device (or managed) memory of the current
 *     device; "host" pointers are ordinary or pinned host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls documented as asynchronous only enqueue work on it.
 *   - Graph data are int32 CSR: offsets[n+1], cols[e] with each row strictly
 *     increasing (sorted, no duplicates), 0 <= cols < n.
 */
#ifndef FLEXIWALK_H
#define FLEXIWALK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FW_OK = 0,
  FW_ERR_ARG = -1,          /* invalid argument                                   */
  FW_ERR_CSR = -2,          /* offsets not monotone / col out of range / row not
                               strictly increasing / weight not finite and > 0    */
  FW_ERR_OOM = -3,          /* device or host allocation failed                   */
  FW_ERR_CUDA = -4,         /* a CUDA runtime call failed                         */
  FW_ERR_TIMEOUT = -5,      /* a bounded wait ran out                             */
  FW_ERR_DEVICE_CHECK = -6, /* a device-side check failed (e.g. start >= n)       */
  FW_ERR_BUSY = -7,         /* resource in use                                    */
  FW_ERR_UNSUPPORTED = -8   /* feature not available for these inputs             */
} fw_status;

typedef enum { FW_ALGO_WEIGHTED = 0, FW_ALGO_NODE2VEC = 1, FW_ALGO_METAPATH = 2 } fw_algo;

typedef enum {
  FW_MODE_AUTO = 0,  /* cost model per walker-step, Eq. (runtime)          */
  FW_MODE_RJS = 1,   /* eRJS only (capped; a capped step finishes by eRVS) */
  FW_MODE_RVS = 2,   /* eRVS only                                           */
  FW_MODE_EXACT = 3  /* exact FP32 inverse CDF (bit-exact parity mode)      */
} fw_mode;

enum { FW_PTR_HOST = 0, FW_PTR_DEVICE = 1 };

enum {
  FW_FLAG_RVS_NOJUMP = 1, /* eRVS with exponential keys only (Alg. 1), no jumps */
  FW_FLAG_COUNTERS = 2,   /* accumulate per-walk counters (slower build path)    */
  FW_FLAG_UNWEIGHTED = 4, /* ignore h: every property weight is 1 (Sec. 5.1)     */
  FW_FLAG_PLAIN_RJS = 8   /* eRJS exactly as Sec. 3.3 (uniform proposal, bound
                             max(w) * h_MAX) even when node2vec's return edge
                             could be proposed separately                        */
};

/* Parameters of one walk job.  Initialise with fw_params_default(). */
typedef struct {
  float p, q;            /* node2vec return / in-out parameters, finite and > 0 */
  uint8_t schema[16];    /* metapath labels; hop j needs schema[j % schema_len]  */
  int32_t schema_len;    /* 1..16 for metapath, ignored otherwise               */
  int32_t mode;          /* fw_mode                                             */
  int32_t flags;         /* FW_FLAG_*                                           */
  float cost_ratio;      /* r = EdgeCost_RJS / EdgeCost_RVS of Eq. (runtime);
                            <= 0 selects the graph's tuned value (default 4)     */
  int32_t rjs_cap;       /* eRJS trials before a step is handed to eRVS;
                            <= 0 selects 64                                      */
  uint32_t walker_base;  /* random-stream id of starts[0]; walker i uses
                            walker_base + i                                      */
} fw_params;

/* Filled in by fw_graph_info(). */
typedef struct {
  int32_t n;
  int64_t e;
  int32_t max_degree;
  int32_t has_weights;
  int32_t has_labels;
  float cost_ratio;          /* current tuned r                                  */
  double preprocess_ms;      /* h_MAX / h_SUM reductions, Sec. 4.2 preprocess()  */
  size_t device_bytes;       /* device memory held by the graph                  */
  int32_t symmetric;         /* 1: every edge (v,u) has a mirror (u,v) with the
                                same weight (found at creation)                   */
} fw_graph_info_t;

/* Per-walk counters (FW_FLAG_COUNTERS).  Byte figures follow the
 * algorithmic byte model: coalesced streams at 4-byte granularity, random
 * single-word gathers at 32-byte sector granularity. */
typedef struct {
  uint64_t hops;           /* walker-steps taken                                 */
  uint64_t rjs_steps;      /* steps finished by eRJS                             */
  uint64_t rvs_steps;      /* steps finished by eRVS (incl. eRJS hand-offs)      */
  uint64_t exact_steps;    /* steps finished by the exact inverse CDF            */
  uint64_t handoffs;       /* eRJS steps that hit the trial cap                  */
  uint64_t rjs_trials;     /* eRJS trials                                        */
  uint64_t rvs_items;      /* neighbours scanned by eRVS                         */
  uint64_t rvs_keys;       /* exponential keys drawn by eRVS (phase 1 + jumps)   */
  uint64_t probes;         /* membership binary-search probes (node2vec)         */
  uint64_t dead_ends;      /* walkers stopped by zero total weight               */
  uint64_t bytes;          /* algorithmic bytes moved                            */
} fw_counters;

typedef struct fw_graph fw_graph;

/* Fill p = q = 1, mode AUTO, cost_ratio = 0 (tuned), rjs_cap = 0 (64),
 * flags 0, walker_base 0, empty schema. */
void fw_params_default(fw_params* params);

/*
 * Build a resident graph: validate the CSR, copy it to the device and run
 * the per-node preprocessing reductions h_MAX[v], h_SUM[v] (Sec. 4.2,
 * preprocess(); "lightweight GPU reduction kernels").
 *   offsets  int32[n+1], cols int32[e]                 (host or device)
 *   weights  float32[e] property weights h, or NULL for h = 1
 *   labels   uint8[e] edge labels, or NULL (metapath then unavailable)
 *   ptr_kind FW_PTR_HOST or FW_PTR_DEVICE for all four arrays
 * The graph copies its inputs; the caller may free them once this call
 * returns.  Synchronous on `stream`.  Errors: FW_ERR_ARG, FW_ERR_CSR,
 * FW_ERR_OOM, FW_ERR_CUDA; *out is NULL on error.
 */
fw_status fw_graph_create(const int32_t* offsets, const int32_t* cols, const float* weights,
                          const uint8_t* labels, int32_t n, int64_t e, int32_t ptr_kind,
                          void* stream, fw_graph** out);

/* Release all device memory of the graph (synchronises the device). */
fw_status fw_graph_destroy(fw_graph* graph);

fw_status fw_graph_info(const fw_graph* graph, fw_graph_info_t* info);

/* Copy the preprocessed h_MAX[n] and h_SUM[n] (float32) into the device
 * buffers given (either may be NULL).  Asynchronous on `stream`. */
fw_status fw_graph_node_stats(const fw_graph* graph, float* hmax, float* hsum, void* stream);

/* Set the graph's cost ratio r of Eq. (runtime) (must be finite, > 0). */
fw_status fw_graph_set_cost_ratio(fw_graph* graph, float ratio);

/*
 * Walk num_walkers walkers for len hops each (Sec. 2.1; one query per
 * walker fetched from a global counter, Sec. 5.3).
 *   starts  device int32[num_walkers], each in [0, n)
 *   out     device int32[num_walkers][len+1], row-major; row i = starts[i]
 *           followed by the len visited nodes, -1 after a dead end
 *   algo    fw_algo;  params as above (NULL = defaults);  seed = Philox key
 * Asynchronous on `stream`.  A start outside [0, n) yields a row of -1 and
 * FW_ERR_DEVICE_CHECK from the next fw_graph_check().  Errors reported
 * directly: FW_ERR_ARG (bad sizes / parameters, metapath without labels),
 * FW_ERR_CUDA.
 */
fw_status fw_walk(const fw_graph* graph, const int32_t* starts, int32_t num_walkers, int32_t len,
                  int32_t algo, const fw_params* params, uint64_t seed, int32_t* out,
                  void* stream);

/*
 * fw_walk with HOST buffers: copies starts (host int32[num_walkers]) to the
 * device, walks, and copies the rows back into out (host
 * int32[num_walkers][len+1]); returns when out is filled.  Pinned host
 * memory gives the fastest copies.  Device staging buffers are owned by the
 * graph and reused across calls (one call at a time per graph: FW_ERR_BUSY
 * otherwise).
 */
fw_status fw_walk_host(fw_graph* graph, const int32_t* starts, int32_t num_walkers, int32_t len,
                       int32_t algo, const fw_params* params, uint64_t seed, int32_t* out,
                       void* stream);

/*
 * Test hook for the sampling kernels: draw ndraws independent next-node
 * samples for the single state (v, v_prev, step) -- v_prev = -1 for no
 * previous node -- with the given mode (AUTO/RJS/RVS/EXACT, through the
 * same device code as fw_walk), and add each pick to counts (device
 * uint64[d(v)], indexed by neighbour position; not cleared here).  Draw i
 * uses random-stream walker id params->walker_base + i.  Dead-end draws are
 * not counted.  Asynchronous on `stream`.
 */
fw_status fw_sample_hist(const fw_graph* graph, int32_t v, int32_t v_prev, int32_t step,
                         int32_t algo, const fw_params* params, uint64_t seed, int64_t ndraws,
                         uint64_t* counts, void* stream);

/*
 * Test hook for the per-step plan (Sec. 3.3 bound, Eq. (sum_estimation),
 * Eq. (runtime)), evaluated by the walk kernel's device code for the
 * `count` states (v[i], has_prev[i]):
 *   bound[i] = B, sum_hat[i] = estimated total weight, mode[i] = 1 (eRJS) or
 *   2 (eRVS).  All arrays device, length count.  Asynchronous.
 */
fw_status fw_step_plan(const fw_graph* graph, const int32_t* v, const int32_t* has_prev,
                       int32_t count, int32_t algo, const fw_params* params, float* bound,
                       float* sum_hat, int32_t* mode, void* stream);

/* Read (synchronising `stream`) or clear the graph's counters. */
fw_status fw_counters_read(const fw_graph* graph, fw_counters* out, void* stream);
fw_status fw_counters_reset(fw_graph* graph, void* stream);

/* Synchronise `stream` and report (then clear) device-side check failures
 * of earlier asynchronous calls on this graph: FW_OK or FW_ERR_DEVICE_CHECK. */
fw_status fw_graph_check(fw_graph* graph, void* stream);

/*
 * fw_walk_host without any device allocation (the paper has no counterpart;
 * this is a deployment convenience).  For callers that cannot allocate
 * device memory when they walk: hosts whose own pool or arena owns the GPU
 * memory, real-time services that forbid allocation after start-up, and
 * plug-ins running under a fixed memory budget.  Same arguments, layout and
 * result as fw_walk_host (host starts / host out, returns when out is
 * filled); the device scratch it needs -- the staged starts, the staged
 * rows and the walk queue counter -- lives in one fixed 16 MiB array inside
 * the library, which every GPU that loads the library holds until exit.
 * Limit: starts (4*num_walkers bytes, rounded up to 256) plus rows
 * (4*num_walkers*(len+1) bytes) must fit in 16 MiB - 256 bytes, else
 * FW_ERR_ARG; larger requests belong to fw_walk_host.  Calls share the
 * array and serialise on a process-wide lock (FW_ERR_BUSY if one is in
 * progress); calls that overlap on the GPU race on it.  The first call on a
 * device looks up the array's device address; make it before any stream
 * capture.  The current device must be the graph's device.
 */
fw_status fw_walk_host_noalloc(const fw_graph* graph, const int32_t* starts, int32_t num_walkers, int32_t len,
                               int32_t algo, const fw_params* params, uint64_t seed, int32_t* out, void* stream);

/* Number of kernel launches this library has issued (process-wide). */
uint64_t fw_launch_count(void);

const char* fw_last_error(void);
const char* fw_status_string(fw_status status);

#ifdef __cplusplus
}
#endif

#endif /* FLEXIWALK_H */
