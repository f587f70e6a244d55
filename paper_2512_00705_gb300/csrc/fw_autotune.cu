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

bool cache_lookup(const char* path, const CacheKey& k, float* r) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[256];
  bool hit = false;
  while (std::fgets(line, sizeof(line), f)) {
    unsigned long long fp;
    int algo, method, flags;
    unsigned schema;
    float p, q, gamma, rv;
    if (std::sscanf(line, "fp=%llx algo=%d p=%g q=%g gamma=%g flags=%d schema=%x method=%d r=%g", &fp, &algo, &p,
                    &q, &gamma, &flags, &schema, &method, &rv) == 9 &&
        fp == k.fp && algo == k.algo && p == k.p && q == k.q && gamma == k.gamma && flags == k.flags &&
        schema == k.schema && method == k.method && rv > 0.0f) {
      *r = rv;
      hit = true;  // the last matching line wins
    }
  }
  std::fclose(f);
  return hit;
}

void cache_store(const char* path, const CacheKey& k, float r) {
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "fp=%016llx algo=%d p=%.9g q=%.9g gamma=%.9g flags=%d schema=%08x method=%d r=%.9g\n", k.fp,
               k.algo, k.p, k.q, k.gamma, k.flags, k.schema, k.method, r);
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

static fw_status sweep_ratio(fw_graph* g, int32_t algo, const fw_params* params, cudaStream_t st, float* r_out) {
  // sample walk per candidate r: up to 2^20 walkers from degree-biased starts, 32 hops
  if (g->e == 0) {
    *r_out = 4.0f;
    return FW_OK;
  }
  const int32_t w = (int32_t)(g->e < (1ll << 20) ? g->e : (1ll << 20));
  const int32_t len = 32;
  int32_t *d_starts = nullptr, *d_out = nullptr;
  cudaError_t e = cudaMalloc(&d_starts, sizeof(int32_t) * (size_t)w);
  if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(int32_t) * (size_t)w * (len + 1));
  if (e == cudaSuccess) {
    sweep_starts_kernel<<<(w + 255) / 256, 256, 0, st>>>(g->d_col, (long long)g->e, w, d_starts);
    g_launches.fetch_add(1);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaFree(d_starts);
    cudaFree(d_out);
    return cuda_error(e, "sweep buffers");
  }
  const float ladder[] = {0.125f, 0.25f, 0.5f, 1.0f, 2.0f, 4.0f, 8.0f, 16.0f, 32.0f, 64.0f};
  fw_params P;
  if (params) P = *params;
  else fw_params_default(&P);
  P.mode = FW_MODE_AUTO;
  P.flags &= ~FW_FLAG_COUNTERS;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  constexpr int kLadder = (int)(sizeof(ladder) / sizeof(ladder[0]));
  float times[kLadder];
  for (int li = 0; li < kLadder; ++li) times[li] = 1e30f;
  fw_status s = FW_OK;
  P.cost_ratio = 4.0f;
  s = fw_walk(g, d_starts, w, len, algo, &P, 7, d_out, st);  // warm-up
  for (int li = 0; li < kLadder && s == FW_OK; ++li) {
    P.cost_ratio = ladder[li];
    float t = 1e30f;
    for (int rep = 0; rep < 2 && s == FW_OK; ++rep) {
      cudaEventRecord(a, st);
      s = fw_walk(g, d_starts, w, len, algo, &P, 7, d_out, st);
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, a, b);
      t = std::fmin(t, ms);
    }
    times[li] = t;
  }
  // Where the timing is flat, sample noise alone would decide; take the
  // median (the ladder is geometric: the middle in log r) of the ratios
  // within 3 % of the fastest instead, the smaller one of an even count.
  float best = 1e30f;
  for (int li = 0; li < kLadder; ++li) best = std::fmin(best, times[li]);
  int near[kLadder], count = 0;
  for (int li = 0; li < kLadder; ++li)
    if (times[li] <= 1.03f * best) near[count++] = li;
  const float best_r = count == 0 ? 4.0f : ladder[near[(count - 1) / 2]];
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(d_starts);
  cudaFree(d_out);
  if (s != FW_OK) return s;
  *r_out = best_r;
  return FW_OK;
}

}  // namespace fw

using namespace fw;

extern "C" fw_status fw_autotune(fw_graph* g, int32_t algo, const fw_params* params, int32_t method,
                                 const char* cache_path, float* ratio_out, void* stream) {
  if (!g) return set_error(FW_ERR_ARG, "graph is NULL");
  if (method != 0 && method != 1) return set_error(FW_ERR_ARG, "method must be 0 (profiling kernels) or 1 (sweep)");
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
  float r = 0.0f;
  bool cached = cache_path && cache_path[0] && cache_lookup(cache_path, key, &r);
  if (!cached) {
    s = method == 0 ? profile_ratio(g, J, st, &r) : sweep_ratio(g, algo, params, st, &r);
    if (s != FW_OK) return s;
    if (!(r > 0.0f) || !std::isfinite(r)) return set_error(FW_ERR_CUDA, "profiling gave no usable ratio");
    if (cache_path && cache_path[0]) cache_store(cache_path, key, r);
  }
  g->ratio_algo[algo] = r;
  if (ratio_out) *ratio_out = r;
  return FW_OK;
}
