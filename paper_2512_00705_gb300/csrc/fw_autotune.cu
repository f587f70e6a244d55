// fw_autotune.cu -- the cost ratio r = EdgeCost_RJS / EdgeCost_RVS of
// Eq. (runtime), measured on the graph (Sec. 5.1, profiling kernels).
//
// Method 0 follows the paper: two light kernels compute transition weights
// for a fixed sample of nodes and a fixed number of their neighbours, one
// the eRJS way (each thread one trial at a random neighbour position: Philox
// draw, edge-record gather, squeeze / membership test) and one the eRVS way
// (a warp scans the first 256 neighbours of a node as eRVS does: coalesced
// loads, weights, phase-1 keys, jumps, argmax); r is the ratio of their
// times per edge.  The
// kernels run the walk kernel's own device functions, so the ratio reflects
// this GPU's caches and this graph.
// Method 1 (an extension): time short sample walks from degree-biased starts
// for a ladder of r values and keep the fastest.
// Results are cached in a text file keyed by a fingerprint of the graph,
// the algorithm, p, q and the method.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fw_internal.h"

namespace fw {
namespace {

constexpr int kProfileNodes = 65536;  // sampled nodes (evenly spaced ids)
constexpr int kProfileEdges = 32;     // eRJS trials per sampled node
constexpr int kProfileScan = 256;     // neighbours an eRVS scan covers per sampled node (jumps included)

// Sample node i -> its id, a previous node (its first neighbour) and the rows.
__device__ __forceinline__ bool profile_ctx(const DevGraph& g, const Job& J, int32_t i, int32_t stride, StepCtx& c) {
  const int32_t v = i * stride;
  if (v >= g.n) return false;
  const int4 nr = __ldg(g.nrec + 2ll * v);
  if (nr.y == 0) return false;
  c.v = v;
  c.s = nr.x;
  c.d = nr.y;
  c.step = 1;
  c.vp = (J.algo == ALGO_NODE2VEC || J.algo == ALGO_PAGERANK2) ? __ldg(g.col + nr.x) : -1;
  c.w1 = c.w2 = 1.0f;
  if (c.vp >= 0) {
    const int4 pr = __ldg(g.nrec + 2ll * c.vp);
    c.ps = pr.x;
    c.pe = pr.x + pr.y;
    if (J.algo == ALGO_PAGERANK2) pagerank2_weights(J, c.d, pr.y, c.w1, c.w2);
  } else {
    c.ps = c.pe = 0;
  }
  c.wid = (uint32_t)i;
  c.hsc = g.h8 ? __ldg(g.h8scale + v) : 0.0f;
  c.n0 = -1;  // one weight class: the paper's eRJS
  c.n1 = 0;
  return true;
}

__global__ void profile_rjs_kernel(DevGraph g, Job J, int32_t count, int32_t stride, unsigned long long* evals,
                                   unsigned* sink) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t i = (int32_t)(t / kProfileEdges), j = (int32_t)(t % kProfileEdges);
  unsigned found = 0, done = 0;
  if (i < count) {
    StepCtx c;
    if (profile_ctx(g, J, i, stride, c)) {
      const bool second = J.algo == ALGO_NODE2VEC && c.vp >= 0;
      const float hm = J.weighted ? __int_as_float(__ldg(g.nrec + 2ll * c.v).z) : 1.0f;
      const float B = __fmul_rn(second ? J.wmax1 : (J.algo == ALGO_PAGERANK2 && c.vp >= 0 ? c.w1 : 1.0f), hm);
      Accept acc;
      LaneCounters lc;
      found = rjs_trials<false>(g, J, c, B, false, 0.0f, -1, 0.0f, j, 1, acc, lc) ? 1u : 0u;
      done = 1;
    }
  }
  const unsigned nd = __reduce_add_sync(kFull, done), nf = __reduce_add_sync(kFull, found);
  if ((threadIdx.x & 31) == 0 && nd) {
    atomicAdd(evals, (unsigned long long)nd);
    atomicAdd(sink, nf);
  }
}

__global__ void profile_rvs_kernel(DevGraph g, Job J, int32_t count, int32_t stride, unsigned long long* evals,
                                   unsigned* sink) {
  const int lane = threadIdx.x & 31;
  const int32_t i = (int32_t)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (i >= count) return;  // warp-uniform
  StepCtx c;
  if (!profile_ctx(g, J, i, stride, c)) return;  // warp-uniform (same node for the whole warp)
  c.d = min(c.d, kProfileScan);
  LaneCounters lc;
  const int32_t k = rvs_pick<32, false>(g, J, c, lane, true, lc);
  if (lane == 0) {
    atomicAdd(evals, (unsigned long long)c.d);
    atomicAdd(sink, (unsigned)(k + 1));
  }
}

// Sweep starts: the targets of w evenly spaced CSR entries.  A node is then
// picked in proportion to its degree, which is where a walk spends its steps
// once it has mixed (the stationary law of a first-order walk on a symmetric
// graph), so the sample walks weigh hubs as a long walk does.
__global__ void sweep_starts_kernel(const int32_t* __restrict__ col, long long e, int32_t w, int32_t* __restrict__ out) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < w) out[i] = __ldg(col + (long long)((double)i * (double)e / (double)w));
}

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

// A tuned r is stored per graph fingerprint and per everything that changes
// the walk's cost: algorithm, p, q, gamma, the sampler flags and the schema.
struct CacheKey {
  unsigned long long fp;
  int algo;
  float p, q, gamma;
  int flags;
  unsigned schema;  // FNV-1a of the schema entries in use
  int method;
};

// A tuned result: r, and (method 2) the launch shape; 0 = not tuned.
struct Tuned {
  float r = 0.0f;
  int lane_max = 0, rjs_batch = 0;
  float budget = 0.0f;
};

bool cache_lookup(const char* path, const CacheKey& k, Tuned* t) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[320];
  bool hit = false;
  while (std::fgets(line, sizeof(line), f)) {
    unsigned long long fp;
    int algo, method, flags, lane = 0, batch = 0;
    unsigned schema;
    float p, q, gamma, rv, budget = 0.0f;
    const int got = std::sscanf(line, "fp=%llx algo=%d p=%g q=%g gamma=%g flags=%d schema=%x method=%d r=%g "
                                      "lane=%d batch=%d budget=%g",
                                &fp, &algo, &p, &q, &gamma, &flags, &schema, &method, &rv, &lane, &batch, &budget);
    if ((got == 9 || got == 12) && fp == k.fp && algo == k.algo && p == k.p && q == k.q && gamma == k.gamma &&
        flags == k.flags && schema == k.schema && method == k.method && rv > 0.0f &&
        (method != 2 || (got == 12 && lane >= 1 && lane <= 64 && batch >= 1 && batch <= 16 && budget > 0.0f))) {
      t->r = rv;
      t->lane_max = got == 12 ? lane : 0;
      t->rjs_batch = got == 12 ? batch : 0;
      t->budget = got == 12 ? budget : 0.0f;
      hit = true;  // the last matching line wins
    }
  }
  std::fclose(f);
  return hit;
}

void cache_store(const char* path, const CacheKey& k, const Tuned& t) {
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "fp=%016llx algo=%d p=%.9g q=%.9g gamma=%.9g flags=%d schema=%08x method=%d r=%.9g", k.fp, k.algo,
               k.p, k.q, k.gamma, k.flags, k.schema, k.method, t.r);
  if (k.method == 2) std::fprintf(f, " lane=%d batch=%d budget=%.9g", t.lane_max, t.rjs_batch, t.budget);
  std::fprintf(f, "\n");
  std::fclose(f);
}

}  // namespace

// Fingerprint of the resident graph: FNV-1a over the sizes and 4096 evenly
// spaced entries of offsets, cols and weights (gathered by one kernel).
__global__ void fingerprint_gather_kernel(const int32_t* __restrict__ off, const int32_t* __restrict__ col,
                                          const float* __restrict__ h, int32_t n, long long e, int k,
                                          int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const long long io = (long long)n * i / (k - 1);
  out[i] = off[io];
  if (e > 0) {
    const long long ie = (e - 1) * i / (k - 1);
    out[k + i] = col[ie];
    out[2 * k + i] = h ? __float_as_int(h[ie]) : 0;
  } else {
    out[k + i] = out[2 * k + i] = 0;
  }
}

fw_status graph_fingerprint(const fw_graph* g, cudaStream_t st, unsigned long long* out) {
  const int k = 4096;
  int32_t* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int32_t) * 3 * k);
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(fingerprint)");
  std::vector<int32_t> buf(3 * k);
  fingerprint_gather_kernel<<<(k + 255) / 256, 256, 0, st>>>(g->d_off, g->d_col, g->d_h, g->n, g->e, k, d);
  g_launches.fetch_add(1);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf.data(), d, sizeof(int32_t) * 3 * k, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_error(e, "graph fingerprint");
  uint64_t h = 1469598103934665603ull;
  h = fnv1a(h, &g->n, sizeof(g->n));
  h = fnv1a(h, &g->e, sizeof(g->e));
  h = fnv1a(h, buf.data(), sizeof(int32_t) * 3 * k);
  *out = h;
  return FW_OK;
}

static fw_status profile_ratio(fw_graph* g, const Job& J, cudaStream_t st, float* r_out) {
  const int32_t count = g->n < kProfileNodes ? g->n : kProfileNodes;
  if (count == 0) return set_error(FW_ERR_ARG, "empty graph");
  const int32_t stride = g->n / count;
  unsigned long long* d_ev = nullptr;
  cudaError_t e = cudaMalloc(&d_ev, 2 * sizeof(unsigned long long) + 2 * sizeof(unsigned));
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(profiling counters)");
  unsigned* d_sink = reinterpret_cast<unsigned*>(d_ev + 2);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const DevGraph dg = dev_graph(g);
  const long long rjs_threads = (long long)count * kProfileEdges;
  const int rjs_grid = (int)((rjs_threads + 255) / 256);
  const int rvs_grid = (int)(((long long)count * 32 + 255) / 256);
  float best_rjs = 1e30f, best_rvs = 1e30f;
  unsigned long long ev[2] = {0, 0};
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaMemsetAsync(d_ev, 0, 2 * sizeof(unsigned long long) + 2 * sizeof(unsigned), st);
    cudaEventRecord(a, st);
    profile_rjs_kernel<<<rjs_grid, 256, 0, st>>>(dg, J, count, stride, d_ev, d_sink);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    float t0 = 0.0f;
    cudaEventElapsedTime(&t0, a, b);
    cudaEventRecord(a, st);
    profile_rvs_kernel<<<rvs_grid, 256, 0, st>>>(dg, J, count, stride, d_ev + 1, d_sink + 1);
    cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float t1 = 0.0f;
    cudaEventElapsedTime(&t1, a, b);
    g_launches.fetch_add(2);
    if (e == cudaSuccess) e = cudaMemcpy(ev, d_ev, sizeof(ev), cudaMemcpyDeviceToHost);
    if (rep > 0) {  // the first repetition warms caches and loads the module
      best_rjs = std::fmin(best_rjs, t0);
      best_rvs = std::fmin(best_rvs, t1);
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(d_ev);
  if (e != cudaSuccess) return cuda_error(e, "profiling kernels");
  if (ev[0] == 0 || ev[1] == 0) return set_error(FW_ERR_ARG, "no edges to profile");
  const double c_rjs = best_rjs / (double)ev[0], c_rvs = best_rvs / (double)ev[1];
  *r_out = (float)(c_rjs / c_rvs);
  return FW_OK;
}

// Sample walks for the sweeps: up to 2^20 walkers from degree-biased starts.
struct Sample {
  int32_t* starts = nullptr;
  int32_t* out = nullptr;
  int32_t w = 0, len = 0;
  cudaEvent_t a = nullptr, b = nullptr;
  ~Sample() {
    cudaFree(starts);
    cudaFree(out);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

static fw_status make_sample(const fw_graph* g, int32_t len, cudaStream_t st, Sample* sm) {
  sm->w = (int32_t)(g->e < (1ll << 20) ? g->e : (1ll << 20));
  sm->len = len;
  cudaError_t e = cudaMalloc(&sm->starts, sizeof(int32_t) * (size_t)sm->w);
  if (e == cudaSuccess) e = cudaMalloc(&sm->out, sizeof(int32_t) * (size_t)sm->w * (len + 1));
  if (e == cudaSuccess) e = cudaEventCreate(&sm->a);
  if (e == cudaSuccess) e = cudaEventCreate(&sm->b);
  if (e == cudaSuccess) {
    sweep_starts_kernel<<<(sm->w + 255) / 256, 256, 0, st>>>(g->d_col, (long long)g->e, sm->w, sm->starts);
    g_launches.fetch_add(1);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? FW_OK : cuda_error(e, "sweep buffers");
}

// Best of `reps` timings of the sample walk under P.
static fw_status time_sample(const fw_graph* g, int32_t algo, const fw_params& P, Sample& sm, cudaStream_t st,
                             int reps, float* ms_out) {
  float t = 1e30f;
  fw_status s = FW_OK;
  for (int rep = 0; rep < reps && s == FW_OK; ++rep) {
    cudaEventRecord(sm.a, st);
    s = fw_walk(g, sm.starts, sm.w, sm.len, algo, &P, 7, sm.out, st);
    cudaEventRecord(sm.b, st);
    cudaEventSynchronize(sm.b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, sm.a, sm.b);
    t = std::fmin(t, ms);
  }
  *ms_out = t;
  return s;
}

// r over the ladder {1/8, ..., 64} under P's launch shape.  Where the timing
// is flat, sample noise alone would decide; take the median (the ladder is
// geometric: the middle in log r) of the ratios within 3 % of the fastest
// instead, the smaller one of an even count.
static fw_status sweep_r(const fw_graph* g, int32_t algo, fw_params P, Sample& sm, cudaStream_t st, int reps,
                         float* r_out, float* best_ms) {
  const float ladder[] = {0.125f, 0.25f, 0.5f, 1.0f, 2.0f, 4.0f, 8.0f, 16.0f, 32.0f, 64.0f};
  constexpr int kLadder = (int)(sizeof(ladder) / sizeof(ladder[0]));
  float times[kLadder];
  fw_status s = FW_OK;
  for (int li = 0; li < kLadder && s == FW_OK; ++li) {
    P.cost_ratio = ladder[li];
    s = time_sample(g, algo, P, sm, st, reps, &times[li]);
  }
  if (s != FW_OK) return s;
  float best = 1e30f;
  for (int li = 0; li < kLadder; ++li) best = std::fmin(best, times[li]);
  int near[kLadder], count = 0;
  for (int li = 0; li < kLadder; ++li)
    if (times[li] <= 1.03f * best) near[count++] = li;
  *r_out = count == 0 ? 4.0f : ladder[near[(count - 1) / 2]];
  *best_ms = best;
  return FW_OK;
}

static fw_params sweep_params(const fw_params* params) {
  fw_params P;
  if (params) P = *params;
  else fw_params_default(&P);
  P.mode = FW_MODE_AUTO;
  P.flags &= ~FW_FLAG_COUNTERS;
  return P;
}

// Method 1: r from 32-hop sample walks (best of two per candidate).
static fw_status sweep_ratio(fw_graph* g, int32_t algo, const fw_params* params, cudaStream_t st, Tuned* out) {
  if (g->e == 0) {
    out->r = 4.0f;
    return FW_OK;
  }
  Sample sm;
  fw_status s = make_sample(g, 32, st, &sm);
  if (s != FW_OK) return s;
  fw_params P = sweep_params(params);
  P.cost_ratio = 4.0f;
  s = fw_walk(g, sm.starts, sm.w, sm.len, algo, &P, 7, sm.out, st);  // warm-up
  float best = 0.0f;
  if (s == FW_OK) s = sweep_r(g, algo, P, sm, st, 2, &out->r, &best);
  return s;
}

// Method 2: r, then the launch shape one parameter at a time, then r again;
// 64-hop sample walks, best of three per candidate, and a candidate replaces
// the incumbent only when at least 2 % faster, so timing noise between
// near-equal settings does not move the result.
static fw_status sweep_shape(fw_graph* g, int32_t algo, const fw_params* params, cudaStream_t st, Tuned* out) {
  if (g->e == 0) {
    out->r = 4.0f;
    out->lane_max = kLaneMaxDegree;
    out->rjs_batch = kRjsBatchDefault;
    out->budget = 1.0f;
    return FW_OK;
  }
  Sample sm;
  fw_status s = make_sample(g, 64, st, &sm);
  if (s != FW_OK) return s;
  fw_params P = sweep_params(params);
  P.lane_max_degree = kLaneMaxDegree;
  P.rjs_batch = kRjsBatchDefault;
  P.trial_budget = 1.0f;
  P.cost_ratio = 4.0f;
  s = fw_walk(g, sm.starts, sm.w, sm.len, algo, &P, 7, sm.out, st);  // warm-up
  float cur = 0.0f;
  if (s == FW_OK) s = sweep_r(g, algo, P, sm, st, 3, &P.cost_ratio, &cur);
  if (s == FW_OK) s = time_sample(g, algo, P, sm, st, 3, &cur);
  auto try_values = [&](auto member, const auto* values, int nv) {
    for (int i = 0; i < nv && s == FW_OK; ++i) {
      fw_params Q = P;
      Q.*member = values[i];
      if (Q.*member == P.*member) continue;
      float t = 0.0f;
      s = time_sample(g, algo, Q, sm, st, 3, &t);
      if (s == FW_OK && t < 0.98f * cur) {
        P = Q;
        cur = t;
      }
    }
  };
  const int32_t lanes[] = {1, 4, 8, 16, 32, 64};
  const int32_t batches[] = {1, 2, 3, 4, 6};
  const float budgets[] = {0.25f, 0.5f, 1.0f, 2.0f, 4.0f};
  try_values(&fw_params::lane_max_degree, lanes, 6);
  try_values(&fw_params::rjs_batch, batches, 5);
  try_values(&fw_params::trial_budget, budgets, 5);
  float r2 = P.cost_ratio, t2 = 0.0f;
  if (s == FW_OK) s = sweep_r(g, algo, P, sm, st, 3, &r2, &t2);
  if (s == FW_OK && t2 < 0.98f * cur) P.cost_ratio = r2;
  if (s != FW_OK) return s;
  out->r = P.cost_ratio;
  out->lane_max = P.lane_max_degree;
  out->rjs_batch = P.rjs_batch;
  out->budget = P.trial_budget;
  return FW_OK;
}

}  // namespace fw

using namespace fw;

extern "C" fw_status fw_autotune(fw_graph* g, int32_t algo, const fw_params* params, int32_t method,
                                 const char* cache_path, float* ratio_out, void* stream) {
  if (!g) return set_error(FW_ERR_ARG, "graph is NULL");
  if (method < 0 || method > 2)
    return set_error(FW_ERR_ARG, "method must be 0 (profiling kernels), 1 (sweep of r) or 2 (r and launch shape)");
  Job J;
  fw_status s = make_job(g, algo, params, 0x5eedull, &J);
  if (s != FW_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CacheKey key;
  key.algo = algo;
  key.p = params ? params->p : 1.0f;
  key.q = params ? params->q : 1.0f;
  key.gamma = params ? params->gamma : 0.2f;
  key.flags = params ? (params->flags & ~FW_FLAG_COUNTERS) : 0;
  key.schema = 2166136261u;
  for (int i = 0; i < J.schema_len; ++i) key.schema = (key.schema ^ J.schema[i]) * 16777619u;
  key.method = method;
  key.fp = g->fingerprint;
  Tuned t;
  bool cached = cache_path && cache_path[0] && cache_lookup(cache_path, key, &t);
  if (!cached) {
    if (method == 0) s = profile_ratio(g, J, st, &t.r);
    else if (method == 1) s = sweep_ratio(g, algo, params, st, &t);
    else s = sweep_shape(g, algo, params, st, &t);
    if (s != FW_OK) return s;
    if (!(t.r > 0.0f) || !std::isfinite(t.r)) return set_error(FW_ERR_CUDA, "profiling gave no usable ratio");
    if (cache_path && cache_path[0]) cache_store(cache_path, key, t);
  }
  g->ratio_algo[algo] = t.r;
  if (method == 2) {
    g->lane_max_algo[algo] = t.lane_max;
    g->rjs_batch_algo[algo] = t.rjs_batch;
    g->budget_algo[algo] = t.budget;
  }
  if (ratio_out) *ratio_out = t.r;
  return FW_OK;
}
