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
 *       second-order PageRank : see FW_ALGO_PAGERANK2  [Eq. (2ndpr)]
 *   - The draw is made by eRJS (rejection against the on-the-fly bound
 *     B = max(w) * h_MAX[v], [Sec. 3.3]; by default with refined envelopes
 *     that keep the draw exact: three weight classes of h, the return edge
 *     and common neighbours proposed separately, label segments for
 *     metapath -- FW_FLAG_PLAIN_RJS keeps the single uniform proposal) or
 *     by eRVS (single-pass reservoir sampling with exponential keys and
 *     jumps, [Sec. 3.2, Alg. 1, Eq. (jump)]); a first-order cost model
 *     picks eRJS iff r * B < sum-hat, with sum-hat = h_SUM[v] * mean(w)
 *     [Sec. 4.1, Eq. (runtime), Eq. (sum_estimation)].
 *   - An exact inverse-CDF mode (FP32 prefix in neighbour order, one
 *     Philox4x32-10 uniform per hop) reproduces a plain CPU definition bit
 *     for bit; it is the parity mode, not a fast path [Sec. 2.2, ITS].
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the
 *     seed (low word, high word), counter (walker id, hop, stream, draw);
 *     stream 0 is the exact mode's uniform, stream 1 the eRJS trials (draw =
 *     trial; the proposal is Lemire's multiply-shift index of word 0, else
 *     word 1, else none; U from word 2), stream 2 the eRVS keys.  No draw
 *     depends on the launch, so a walk's rows depend only on the graph, the
 *     parameters, the seed and the walker ids.  With a trial budget that no
 *     step reaches, eRJS rows therefore follow from the definition alone.
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

typedef enum {
  FW_ALGO_WEIGHTED = 0,
  FW_ALGO_NODE2VEC = 1,
  FW_ALGO_METAPATH = 2,
  FW_ALGO_PAGERANK2 = 3  /* second-order PageRank, Eq. (2ndpr): with max_d = max(d(v), d(v')),
                            w = ((1-g)/d(v) + g/d(v')) * max_d if u in N(v'), else
                            ((1-g)/d(v)) * max_d (u = v' included); hop 0 first-order */
} fw_algo;

typedef enum {
  FW_MODE_AUTO = 0,  /* cost model per walker-step, Eq. (runtime)          */
  FW_MODE_RJS = 1,   /* eRJS only (capped; a capped step finishes by eRVS) */
  FW_MODE_RVS = 2,   /* eRVS only                                           */
  FW_MODE_EXACT = 3,  /* exact FP32 inverse CDF (bit-exact parity mode)     */
  FW_MODE_RANDOM = 4, /* baseline selection of Sec. 5.4: eRJS or eRVS by a
                         fair coin per walker-step                             */
  FW_MODE_DEGREE = 5  /* baseline selection of Sec. 5.4: eRVS when d(v) < 1000,
                         eRJS otherwise                                        */
} fw_mode;

enum { FW_PTR_HOST = 0, FW_PTR_DEVICE = 1 };

enum {
  FW_FLAG_RVS_NOJUMP = 1, /* eRVS with exponential keys only (Alg. 1), no jumps */
  FW_FLAG_COUNTERS = 2,   /* accumulate per-walk counters (slower build path)    */
  FW_FLAG_UNWEIGHTED = 4, /* ignore h: every property weight is 1 (Sec. 5.1)     */
  FW_FLAG_PLAIN_RJS = 8,  /* eRJS exactly as Sec. 3.3 (uniform proposal, bound
                             max(w) * h_MAX) instead of the refined envelopes:
                             three weight classes (bounds B, B/2, B/4),
                             node2vec's return edge proposed separately, two
                             envelopes for node2vec with q > 1, the common
                             neighbours of second-order PageRank split off       */
  FW_FLAG_PAPER_SUM = 16, /* metapath: plan with the Sec. 4.2 rule (B = h_MAX,
                             sum-hat = h_SUM / 2) even when per-label node
                             statistics exist                                    */
  FW_FLAG_NO_BLOOM = 32,  /* with FW_FLAG_NO_TABLE (or no tables): membership
                             tests search the row without the per-row Bloom
                             pre-check (same answers, same walks)                */
  FW_FLAG_NO_GROUPS = 64, /* metapath: sample over the whole row of v (label
                             test per entry) instead of inside the required
                             label's segment of the label-grouped view           */
  FW_FLAG_NO_TABLE = 128, /* membership tests do not read the row's membership
                             table (an exact hash set of the row's node ids,
                             one 32-byte bucket per test in most cases) but
                             the Bloom filter and a search of the sorted row;
                             same answers, same walks                          */
  FW_FLAG_NO_HUB_SHARE = 256 /* eRVS steps over rows of 32,768 entries or more
                             are scanned in fixed chunks from a phase-1
                             reference; in launches of at most 1/8 of the
                             resident lanes with forced eRVS, idle warps of a
                             block help scan them (CTA-level sharing).  This
                             flag keeps every such step on its own warp: same
                             walks, no sharing                                  */
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
                            <= 0: max(64, ceil(b * m / r)), m the entries
                            that the eRVS hand-off would scan (d(v); in
                            metapath's label-grouped view the required
                            label's entries), r the cost ratio, b the trial
                            budget scale                                      */
  uint32_t walker_base;  /* random-stream id of starts[0]; walker i uses
                            walker_base + i                                      */
  float gamma;           /* second-order PageRank parameter in [0, 1]            */
  /* Launch shape of the samplers (none changes a distribution; 0 selects
   * the graph's tuned value, see fw_autotune method 2): */
  int32_t lane_max_degree; /* eRVS steps over at most this many entries run on
                              the walker's own lane, longer ones on the whole
                              warp; 1..64 (default 8)                          */
  int32_t rjs_batch;       /* eRJS trials a lane runs between two warp ballots
                              for hand-offs; 1..16 (default 2)                 */
  float trial_budget;      /* b of the default rjs_cap, > 0 (default 1)        */
} fw_params;

/* Filled in by fw_graph_info(). */
typedef struct {
  int32_t n;
  int64_t e;
  int32_t max_degree;
  int32_t has_weights;
  int32_t has_labels;
  float cost_ratio;          /* current r of node2vec (= cost_ratios[1])         */
  double preprocess_ms;      /* h_MAX / h_SUM reductions, Sec. 4.2 preprocess()  */
  size_t device_bytes;       /* device memory held by the graph                  */
  int32_t symmetric;         /* 1: every edge (v,u) has a mirror (u,v) with the
                                same weight (found at creation)                   */
  float cost_ratios[4];      /* r per algorithm, indexed by fw_algo             */
  uint64_t fingerprint;      /* hash of sizes and sampled CSR entries (cache key)*/
  float weight_scale;        /* largest per-node scale s_v after
                                fw_graph_quantize_weights, else 0                */
  int32_t lane_max_degrees[4]; /* tuned launch shape per algorithm (fw_params)  */
  int32_t rjs_batches[4];
  float trial_budgets[4];
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

/* Fill p = q = 1, gamma = 0.2, mode AUTO, cost_ratio = 0 (tuned),
 * rjs_cap = 0 (the default trial budget, see fw_params), flags 0,
 * walker_base 0, empty schema. */
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
 * returns.  Besides the CSR it keeps 32-byte edge records (twice with
 * weights and degrees below 2^24: in CSR order and with each row
 * partitioned by weight class),
 * 32-byte node records, per-row Bloom filters, per-row membership tables
 * (an exact hash set of each row's node ids, about 8 bytes per entry; if
 * they do not fit, membership tests search the rows) and, with labels all
 * below 8, per-label node statistics and a label-grouped copy of the rows
 * (36 bytes per entry) for metapath; if that copy does not fit, metapath
 * samples over whole rows.
 * Synchronous on `stream`.  Errors: FW_ERR_ARG, FW_ERR_CSR, FW_ERR_OOM,
 * FW_ERR_CUDA; *out is NULL on error.
 */
fw_status fw_graph_create(const int32_t* offsets, const int32_t* cols, const float* weights,
                          const uint8_t* labels, int32_t n, int64_t e, int32_t ptr_kind,
                          void* stream, fw_graph** out);

/* Release all device memory of the graph (synchronises the device). */
fw_status fw_graph_destroy(fw_graph* graph);

/* Fill *info (host memory) from the graph's host-side state; no device
 * work.  FW_ERR_ARG for a NULL argument. */
fw_status fw_graph_info(const fw_graph* graph, fw_graph_info_t* info);

/* Copy the preprocessed h_MAX[n] and h_SUM[n] (float32) into the device
 * buffers given (either may be NULL).  Asynchronous on `stream`. */
fw_status fw_graph_node_stats(const fw_graph* graph, float* hmax, float* hsum, void* stream);

/* Copy the per-label node statistics into `stats` (device float32
 * [n][8][2]: for node v and label l, the maximum and the sum of h over the
 * edges of v labelled l; h = 1 without weights).  They exist when the graph
 * has labels, all below 8 (FW_ERR_UNSUPPORTED otherwise).  The metapath
 * plan uses them for the required label: B = max, exact sum for Eq.
 * (runtime), and zero sum = dead end.  Asynchronous on `stream`. */
fw_status fw_graph_label_stats(const fw_graph* graph, float* stats, void* stream);

/*
 * Store the property weights as 8-bit codes (a low-precision weight format,
 * named in Sec. 6.2 as an extension of the method): every node v gets the
 * scale of its own row, s_v = h_MAX[v] / 255 (FP32 division), and each
 * weight of the row becomes
 *   code_e = clamp(rint(h_e / s_v), 1, 255)     (round half to even)
 * and from then on the graph samples with the dequantized weights
 *   h'_e = code_e * s_v                          (FP32 product).
 * Codes never round to 0, so every edge keeps a positive weight, and each
 * row's largest weight keeps code 255, so a row's distribution moves by at
 * most one code step of its own maximum per weight however skewed the
 * weights of other rows are.  (Mirrored entries may then differ: h'(u,v)
 * uses s_u.)  The preprocessing (h_MAX, h_SUM, edge records, label
 * statistics) and the fingerprint are recomputed from h'; scans in eRVS and
 * exact mode then read one byte per weight and the row's scale.
 * *scale_out (may be NULL) receives the largest s_v.  A second call is a
 * no-op.  Synchronous on `stream`; no walk may run on the graph meanwhile.
 * Errors: FW_ERR_ARG, FW_ERR_UNSUPPORTED (graph without weights),
 * FW_ERR_OOM / FW_ERR_CUDA (the graph is unchanged when the codes cannot be
 * allocated).
 */
fw_status fw_graph_quantize_weights(fw_graph* graph, float* scale_out, void* stream);

/* Copy the per-node scales s_v of the 8-bit codes into `scales` (device
 * float32[n]).  Asynchronous on `stream`.  FW_ERR_UNSUPPORTED before
 * fw_graph_quantize_weights. */
fw_status fw_graph_weight_scales(const fw_graph* graph, float* scales, void* stream);

/* Set the graph's cost ratio r of Eq. (runtime) for every algorithm (must
 * be finite, > 0). */
fw_status fw_graph_set_cost_ratio(fw_graph* graph, float ratio);

/*
 * Measure and install the cost ratio r = EdgeCost_RJS / EdgeCost_RVS of
 * Eq. (runtime) for `algo` with `params` (Sec. 5.1, profiling kernels).
 *   method 0  the paper's profiling: two light kernels compute transition
 *             weights for 65,536 evenly spaced nodes, eRJS-style (32 random
 *             positions per node, one thread each) and eRVS-style (a
 *             coalesced warp scan of up to 256 neighbours with keys and
 *             jumps); r = ratio of their times per edge
 *   method 1  sweep: time 32-hop sample walks of up to 2^20 walkers that
 *             start at the targets of evenly spaced CSR entries (nodes in
 *             proportion to their degree, as in a mixed walk) for
 *             r in {0.125, 0.25, 0.5, 1, 2, ..., 64}; of the ratios within
 *             3 % of the fastest time, keep the median
 *   method 2  method 1's sweep of r with 64-hop sample walks, then the launch
 *             shape one parameter at a time -- lane_max_degree in
 *             {1, 4, 8, 16, 32, 64}, rjs_batch in {1, 2, 3, 4, 6},
 *             trial_budget in {0.25, 0.5, 1, 2, 4} -- each candidate kept
 *             only if its sample walk (best of three) is at least 2 %
 *             faster than the incumbent, then r swept again under the
 *             chosen shape; installs all four for `algo`
 * cache_path (may be NULL): a text file of earlier results keyed by the
 * graph fingerprint, algo, p, q, gamma, flags, schema and method; a hit
 * skips the measurement, a miss appends the new result.  Synchronous on
 * `stream`.  The ratio and the launch shape only change which sampler runs
 * and how the warp's lanes share the steps, never the distribution.
 */
fw_status fw_autotune(fw_graph* graph, int32_t algo, const fw_params* params, int32_t method,
                      const char* cache_path, float* ratio_out, void* stream);

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
 * fw_walk with an explicit random-stream id per walker: walker i draws from
 * the streams of walker_ids[i] (device uint32[num_walkers]) instead of
 * params->walker_base + i.  A shard of a larger query set (Sec. 5.6 spreads
 * queries over GPUs by a hash of the start node) passes the queries'
 * global indices and gets exactly the rows the whole set would give on one
 * GPU.  Asynchronous; errors as fw_walk.
 */
fw_status fw_walk_ids(const fw_graph* graph, const int32_t* starts, const uint32_t* walker_ids, int32_t num_walkers,
                      int32_t len, int32_t algo, const fw_params* params, uint64_t seed, int32_t* out, void* stream);

/*
 * fw_walk with HOST buffers: copies starts (host int32[num_walkers]) to the
 * device, walks, and copies the rows back into out (host
 * int32[num_walkers][len+1]); returns when out is filled.  Pinned host
 * memory gives the fastest copies.  Device staging buffers are owned by the
 * graph and reused across calls (one call at a time per graph: FW_ERR_BUSY
 * otherwise).  Requests whose rows take 128 MiB or more are walked in up to
 * 16 chunks of consecutive walkers, on `stream` and a second stream owned by
 * the graph, and each chunk's rows are copied out on a third while later
 * chunks still walk; walker i keeps random-stream id walker_base + i, so the
 * rows are those of one fw_walk.  Work already queued on `stream` runs
 * first.
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
 * `count` states (v[i], v_prev[i]) -- v_prev[i] = -1 for no previous node:
 *   bound[i] = B, sum_hat[i] = estimated total weight, mode[i] = 1 (eRJS) or
 *   2 (eRVS).  Metapath uses the Sec. 4.2 rule here (B = h_MAX, sum-hat =
 *   h_SUM/2).  All arrays device, length count.  Asynchronous.
 */
fw_status fw_step_plan(const fw_graph* graph, const int32_t* v, const int32_t* v_prev, int32_t count, int32_t algo,
                       const fw_params* params, float* bound, float* sum_hat, int32_t* mode, void* stream);

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
 * progress); calls that overlap on the GPU race on it.  Every call looks up
 * the array's device address on the current device, so the call stays valid
 * after a cudaDeviceReset (with the graph created again); the first call on a
 * device also loads the module holding the array, so make it before any
 * stream capture.  The current device must be the graph's device.
 */
fw_status fw_walk_host_noalloc(const fw_graph* graph, const int32_t* starts, int32_t num_walkers, int32_t len,
                               int32_t algo, const fw_params* params, uint64_t seed, int32_t* out, void* stream);

/* One job of a batch: the arguments of one fw_walk call. */
typedef struct {
  const int32_t* starts;  /* device int32[num_walkers], each in [0, n)               */
  int32_t num_walkers;
  int32_t len;
  int32_t algo;           /* fw_algo                                                  */
  fw_params params;
  uint64_t seed;
  int32_t* out;           /* device int32[num_walkers][len+1]                        */
} fw_job;

/*
 * Run njobs walk jobs in batches of up to 64: within a batch the walkers of
 * all jobs of one algorithm form one query queue (Sec. 5.3) walked by one
 * persistent launch of the kernel compiled for that algorithm, so jobs of
 * very different sizes and lengths share the GPU instead of running one
 * after another.  The per-algorithm launches of a batch follow each other
 * on `stream` (a batch plan runs them side by side).  Every job's rows are
 * identical to those of fw_walk with the same arguments (draws and sampler
 * choices depend only on the walker's own job).  Asynchronous on `stream`;
 * errors as fw_walk (a bad job is named in the message).
 */
fw_status fw_walk_batch(const fw_graph* graph, const fw_job* jobs, int32_t njobs, void* stream);

/*
 * A batch captured once into a CUDA graph (queue-counter resets and walk
 * launches; the per-algorithm launches of each 64-job chunk are parallel
 * branches of the graph) and replayed by fw_batch_plan_launch on any
 * stream as one graph launch.  The jobs' buffers and parameters are fixed
 * at creation; their contents may change between replays.  The plan owns
 * its queue counters; destroy it after its last replay has finished.
 */
typedef struct fw_batch_plan fw_batch_plan;
fw_status fw_batch_plan_create(const fw_graph* graph, const fw_job* jobs, int32_t njobs,
                               fw_batch_plan** out);
fw_status fw_batch_plan_launch(fw_batch_plan* plan, void* stream);
fw_status fw_batch_plan_destroy(fw_batch_plan* plan);

/*
 * Serving: continuous batching of walk queries against a resident graph.
 * A worker thread admits queued queries in arrival order while a fixed
 * device arena of mem_budget bytes has room for their staged starts and
 * rows (small queries before large ones, see large_query_steps), launches
 * the admitted queries as one batched walk ("wave", up to max_jobs_per_wave
 * queries of one size class) on one of max_waves streams, and retires waves
 * by polling their completion events; queries that arrive while waves run
 * join the next wave, and waves on different streams overlap on the device.
 * Copies whose host and device ranges both continue the previous query's
 * merge into one transfer, so clients that take consecutive queries' output
 * buffers back to back from one pinned pool get few large copies.
 * Results are identical to fw_walk_host with the same arguments, alone or in
 * any mix.  All waits are host-side with caller timeouts; nothing spins on
 * the device.
 */
typedef struct {
  size_t mem_budget;          /* device bytes for staged starts + rows (default 1 GiB;
                                 rounded down to a multiple of 256)                   */
  int32_t max_waves;          /* concurrent waves / streams, 1..64 (default 4)          */
  int32_t max_jobs_per_wave;  /* queries per launch, 1..64 (default 64)                 */
  int64_t large_query_steps;  /* queries with W x L at least this are "large": they get
                                 waves of their own, small queries are admitted first
                                 (a large one after waiting 100 ms goes first), and
                                 large waves leave max(1, max_waves / 8) streams to
                                 small ones; 0: one class, plain arrival order
                                 (default)                                             */
} fw_server_config;

typedef struct {
  uint64_t completed, failed, pending;  /* pending = queued or admitted, not launched   */
  uint64_t waves;                       /* launches so far                              */
  double queries_per_wave;
  double p50_ms, p99_ms, mean_ms, max_ms;  /* submit -> rows in host memory, completed   */
  size_t peak_device_bytes;             /* arena high-water mark                        */
  int32_t peak_inflight_waves;
  uint64_t walker_steps;                /* hops of completed queries (counted on device) */
  double queue_p50_ms, queue_p99_ms;    /* submit -> launch of its wave, completed        */
  double wave_p50_ms, wave_p99_ms;      /* launch of its wave -> rows in host memory      */
  double enqueue_ms_per_wave;           /* worker's host time to enqueue a wave's copies
                                           and launches (mean)                            */
  uint64_t copies;                      /* starts and rows copies issued, after merging   */
} fw_server_stats_t;

typedef struct fw_server fw_server;

void fw_server_config_default(fw_server_config* config);

/* Start a server on `graph` (which must outlive it); allocates the arena. */
fw_status fw_server_create(const fw_graph* graph, const fw_server_config* config, fw_server** out);

/*
 * Queue one query: starts (host int32[num_walkers], checked against [0, n)
 * here) and out (host int32[num_walkers][len+1]) must stay valid until the
 * query is collected; pinned host memory lets copies overlap.  Returns a
 * ticket.  FW_ERR_OOM if the query alone exceeds the memory budget,
 * FW_ERR_ARG for bad arguments, FW_ERR_BUSY while the server shuts down.
 */
fw_status fw_server_submit(fw_server* server, const int32_t* starts, int32_t num_walkers, int32_t len, int32_t algo,
                           const fw_params* params, uint64_t seed, int32_t* out, uint64_t* ticket);

/* Queue `count` queries in one call, each an fw_job whose starts and out
 * are HOST buffers with the meaning of fw_server_submit's (they must stay
 * valid until the query is collected); tickets[i] receives query i's
 * ticket.  All queries are checked first and queued under one lock; on the
 * first invalid one the call stops, returns that query's error (its index
 * in the message) and *submitted (may be NULL) tells how many queries before
 * it were queued. */
fw_status fw_server_submit_many(fw_server* server, const fw_job* queries, int32_t count, uint64_t* tickets,
                                int32_t* submitted);

/* Non-blocking: *done = 1 once out is filled (the ticket is then released
 * and the query's status returned; latency_ms, if not NULL, receives the
 * submit-to-completion time). */
fw_status fw_server_poll(fw_server* server, uint64_t ticket, int32_t* done, double* latency_ms);

/* fw_server_poll for `count` tickets under one lock (host arrays of count
 * entries): done[i] = 1 once query i has finished, its ticket then released,
 * status[i] (may be NULL) its fw_status and latency_ms[i] (may be NULL) its
 * submit-to-completion time.  An unknown ticket gives done[i] = 1 and
 * status[i] = FW_ERR_ARG.  Returns FW_OK unless the arguments are bad. */
fw_status fw_server_poll_many(fw_server* server, const uint64_t* tickets, int32_t count, int32_t* done,
                              double* latency_ms, int32_t* status);

/* Wait up to timeout_s seconds: FW_OK (ticket released), FW_ERR_TIMEOUT
 * (ticket kept; wait again later) or the query's error. */
fw_status fw_server_wait(fw_server* server, uint64_t ticket, double timeout_s, double* latency_ms);

fw_status fw_server_stats(fw_server* server, fw_server_stats_t* out);

/* Stop accepting queries, finish every submitted one, free the server. */
fw_status fw_server_destroy(fw_server* server);

/*
 * Measurement hook for the walk kernel's roofline (no counterpart in the
 * paper, whose kernels it does not change).  eRJS trials, node-record
 * fetches and membership probes are dependent 32-byte gathers at random
 * addresses; on HBM each costs a DRAM access whatever its width, so they
 * are bound by the random accesses per second the memory completes, not by
 * the copy bandwidth.  This call measures that ceiling (5 blocks of 256
 * threads per SM, each thread a chain of 64 dependent gathers whose
 * addresses come from the loaded data; more chains do not raise the rate).
 * table: caller-owned device buffer of table_bytes bytes, a power of two of
 * at least 64 MiB (use one well above the L2 size), 32-byte aligned; it is
 * overwritten.  rate_out: host double, gathers per second (best of three
 * launches after one warm-up, CUDA events on `stream`).  Synchronises
 * `stream`; allocates nothing.  FW_ERR_ARG on a bad size or pointer.
 */
fw_status fw_gather_ceiling(void* table, uint64_t table_bytes, double* rate_out, void* stream);

/* Number of kernel launches this library has issued (process-wide). */
uint64_t fw_launch_count(void);

/* Message of the last failing call of this thread ("" if none); the
 * pointer stays valid until this thread's next call into the library. */
const char* fw_last_error(void);
/* Name of a status code ("FW_OK", "FW_ERR_ARG", ..., "FW_ERR_UNKNOWN" for
 * other values); static storage. */
const char* fw_status_string(fw_status status);

#ifdef __cplusplus
}
#endif

#endif /* FLEXIWALK_H */
