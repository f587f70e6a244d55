// fw_api.cu -- the C ABI declared in include/flexiwalk.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fw_internal.h"

namespace fw {

std::atomic<unsigned long long> g_launches{0};

static thread_local std::string t_last_error;

fw_status set_error(fw_status st, const std::string& msg) {
  t_last_error = msg;
  return st;
}

fw_status cuda_error(cudaError_t err, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")";
  return set_error(err == cudaErrorMemoryAllocation ? FW_ERR_OOM : FW_ERR_CUDA, m);
}

DevGraph dev_graph(const fw_graph* g) {
  DevGraph d;
  d.off = g->d_off;
  d.col = g->d_col;
  d.h = g->d_h;
  d.h8 = g->d_h8;
  d.h8scale = g->d_h8scale;
  d.lab = g->d_lab;
  d.hmax = g->d_hmax;
  d.hsum = g->d_hsum;
  d.nrec = g->d_nrec;
  d.erec = g->d_erec;
  d.cerec = g->d_cerec;
  d.lstat = g->d_lstat;
  d.bloom = g->d_bloom;
  d.mtab = g->d_mtab;
  d.lrec = g->d_lrec;
  d.gerec = g->d_gerec;
  d.gh = g->d_gh;
  d.n = g->n;
  d.sym = g->sym;
  return d;
}

static float recip_f32(float p) { return (float)(1.0 / (double)p); }

fw_status make_job(const fw_graph* g, int32_t algo, const fw_params* params, uint64_t seed, Job* job) {
  fw_params P;
  if (params) P = *params;
  else fw_params_default(&P);
  if (algo != ALGO_WEIGHTED && algo != ALGO_NODE2VEC && algo != ALGO_METAPATH && algo != ALGO_PAGERANK2)
    return set_error(FW_ERR_ARG, "unknown algo");
  if (algo == ALGO_PAGERANK2 && !(P.gamma >= 0.0f && P.gamma <= 1.0f))
    return set_error(FW_ERR_ARG, "second-order PageRank needs gamma in [0, 1]");
  if (P.mode < MODE_AUTO || P.mode > MODE_DEGREE) return set_error(FW_ERR_ARG, "unknown mode");
  if (algo == ALGO_NODE2VEC && !(P.p > 0.0f && P.q > 0.0f && std::isfinite(P.p) && std::isfinite(P.q)))
    return set_error(FW_ERR_ARG, "node2vec needs finite p, q > 0");
  if (algo == ALGO_METAPATH) {
    if (!g->d_lab) return set_error(FW_ERR_ARG, "metapath needs edge labels");
    if (P.schema_len < 1 || P.schema_len > 16) return set_error(FW_ERR_ARG, "metapath schema_len must be 1..16");
  }
  if (P.cost_ratio > 0.0f && !std::isfinite(P.cost_ratio)) return set_error(FW_ERR_ARG, "cost_ratio not finite");
  if (P.lane_max_degree < 0 || P.lane_max_degree > 64) return set_error(FW_ERR_ARG, "lane_max_degree must be 0..64");
  if (P.rjs_batch < 0 || P.rjs_batch > 16) return set_error(FW_ERR_ARG, "rjs_batch must be 0..16");
  if (!(P.trial_budget >= 0.0f) || !std::isfinite(P.trial_budget))
    return set_error(FW_ERR_ARG, "trial_budget must be finite and >= 0");
  std::memset(job, 0, sizeof(Job));
  job->algo = algo;
  job->mode = P.mode;
  job->flags = P.flags;
  job->rjs_cap = P.rjs_cap > 0 ? P.rjs_cap : 64;
  job->fixed_cap = P.rjs_cap > 0 ? 1 : 0;
  job->schema_len = algo == ALGO_METAPATH ? P.schema_len : 1;
  std::memcpy(job->schema, P.schema, 16);
  job->weighted = (g->d_h != nullptr && !(P.flags & FW_FLAG_UNWEIGHTED)) ? 1 : 0;
  if (algo == ALGO_NODE2VEC) {
    const float ip = recip_f32(P.p), iq = recip_f32(P.q);
    job->inv_p = ip;
    job->inv_q = iq;
    job->wmax1 = std::fmax(std::fmax(ip, 1.0f), iq);
    job->wmean1 = (float)(((double)ip + 1.0 + (double)iq) / 3.0);
    job->wlo1 = std::fmin(1.0f, iq);
    job->whi1 = std::fmax(1.0f, iq);
    job->need_member = (iq != 1.0f) ? 1 : 0;
    job->second_order = (ip != 1.0f || iq != 1.0f) ? 1 : 0;
    job->split_return = (ip > job->whi1 && !(P.flags & FW_FLAG_PLAIN_RJS)) ? 1 : 0;
    job->split_common = (iq < 1.0f && !(P.flags & FW_FLAG_PLAIN_RJS)) ? 1 : 0;
  } else {
    job->inv_p = job->inv_q = 1.0f;
    job->wmax1 = job->wlo1 = job->whi1 = 1.0f;
    job->wmean1 = algo == ALGO_METAPATH ? 0.5f : 1.0f;
  }
  job->ratio = P.cost_ratio > 0.0f ? P.cost_ratio : g->ratio_algo[algo];
  job->lane_max = P.lane_max_degree > 0 ? P.lane_max_degree : g->lane_max_algo[algo];
  job->rjs_batch = P.rjs_batch > 0 ? P.rjs_batch : g->rjs_batch_algo[algo];
  job->budget = P.trial_budget > 0.0f ? P.trial_budget : g->budget_algo[algo];
  job->key0 = (uint32_t)seed;
  job->key1 = (uint32_t)(seed >> 32);
  job->walker_base = P.walker_base;
  job->pr_g = P.gamma;
  job->pr_1g = 1.0f - P.gamma;
  job->bloom = (g->d_bloom && !(P.flags & FW_FLAG_NO_BLOOM)) ? 1 : 0;
  job->table = (g->d_mtab && !(P.flags & FW_FLAG_NO_TABLE)) ? 1 : 0;
  job->label_stats = (algo == ALGO_METAPATH && g->d_lstat && !(P.flags & FW_FLAG_PAPER_SUM) &&
                      (job->weighted || !g->d_h)) ? 1 : 0;
  job->label_group = (job->label_stats && g->d_lrec && !(P.flags & FW_FLAG_NO_GROUPS)) ? 1 : 0;
  job->classes = (job->weighted && g->d_cerec && !(P.flags & FW_FLAG_PLAIN_RJS)) ? 1 : 0;
  return FW_OK;
}

// The per-graph preprocessing (Sec. 4.2 preprocess()): node records with
// h_MAX / h_SUM and the maximum degree, 32-byte edge records, the weight
// symmetry check and per-label statistics, all from the current weights.
// The label-grouped view of the rows (metapath's fast modes sample inside
// the required label's segment).  Needs the per-label statistics.  If the
// device has no room for it, metapath walks keep the full-row path.
static fw_status build_label_groups(fw_graph* g, cudaStream_t st) {
  const size_t lrec_bytes = 2 * sizeof(int4) * kLabelStats * ((size_t)g->n + 1);
  const size_t gerec_bytes = 2 * sizeof(int4) * (size_t)g->e, gh_bytes = sizeof(float) * (size_t)g->e;
  if (!g->d_lrec) {
    cudaError_t a = cudaMalloc(&g->d_lrec, lrec_bytes);
    if (a == cudaSuccess) a = cudaMalloc(&g->d_gerec, gerec_bytes);
    if (a == cudaSuccess) a = cudaMalloc(&g->d_gh, gh_bytes);
    if (a != cudaSuccess) {
      cudaFree(g->d_lrec);
      cudaFree(g->d_gerec);
      cudaFree(g->d_gh);
      g->d_lrec = nullptr;
      g->d_gerec = nullptr;
      g->d_gh = nullptr;
      cudaGetLastError();  // an allocation failure is not sticky; walks use the full rows
      return FW_OK;
    }
    g->bytes += lrec_bytes + gerec_bytes + gh_bytes;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  cudaError_t le = launch_label_group(g->d_off, g->d_col, g->d_h, g->d_lab, g->d_nrec, g->d_lstat, g->n, g->d_lrec,
                                      g->d_gerec, g->d_gh, g->num_sms, st);
  cudaEventRecord(e1, st);
  cudaError_t se = cudaStreamSynchronize(st);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (le != cudaSuccess) return cuda_error(le, "label-grouped view");
  if (se != cudaSuccess) return cuda_error(se, "sync after label-grouped view");
  g->preprocess_ms += ms;
  return FW_OK;
}

fw_status rebuild_derived(fw_graph* g, cudaStream_t st) {
  const int32_t n = g->n;
  const int64_t e = g->e;
  int* d_maxdeg = reinterpret_cast<int*>(g->d_err) + 8;
  unsigned* d_asym = g->d_err + 12;
  unsigned* d_lbad = g->d_err + 13;
  const bool want_labels = g->d_lab != nullptr && !g->lstat_bad;
  const bool build_bloom = g->d_bloom == nullptr;  // depends on the structure only: built once
  if (build_bloom) {
    cudaError_t ae = cudaMalloc(&g->d_bloom, bloom_bytes(n, e));
    if (ae != cudaSuccess) {
      g->d_bloom = nullptr;
      return cuda_error(ae, "cudaMalloc(row filters)");
    }
    g->bytes += bloom_bytes(n, e);
    // membership tables: without room for them, membership tests search the rows
    ae = cudaMalloc(&g->d_mtab, table_bytes(n, e));
    if (ae != cudaSuccess) {
      g->d_mtab = nullptr;
      cudaGetLastError();  // an allocation failure is not sticky
    } else {
      g->bytes += table_bytes(n, e);
    }
  }
  if (want_labels && !g->d_lstat) {
    cudaError_t ae = cudaMalloc(&g->d_lstat, sizeof(float2) * kLabelStats * ((size_t)n + 1));
    if (ae != cudaSuccess) {
      g->d_lstat = nullptr;
      return cuda_error(ae, "cudaMalloc(label statistics)");
    }
    g->bytes += sizeof(float2) * kLabelStats * ((size_t)n + 1);
  }
  {
    cudaError_t pe = prime_preprocess_kernels();
    if (pe != cudaSuccess) return cuda_error(pe, "load preprocessing kernels");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t le = cudaMemsetAsync(d_maxdeg, 0, sizeof(int), st);
  if (le == cudaSuccess) le = cudaMemsetAsync(d_asym, 0, 2 * sizeof(unsigned), st);
  cudaEventRecord(e0, st);
  if (le == cudaSuccess)
    le = launch_node_stats(g->d_off, g->d_h, n, g->d_hmax, g->d_hsum, g->d_nrec, d_maxdeg, g->num_sms, st);
  if (le == cudaSuccess) le = launch_edge_records(g->d_col, g->d_h, g->d_lab, g->d_nrec, e, g->d_erec, g->num_sms, st);
  if (le == cudaSuccess && g->d_cerec)
    le = launch_class_group(g->d_off, g->d_h, g->d_nrec, g->d_erec, n, g->d_cerec, g->num_sms, st);
  if (le == cudaSuccess) le = launch_symmetry(g->d_off, g->d_col, g->d_h, n, e, d_asym, g->num_sms, st);
  if (le == cudaSuccess && build_bloom)
    le = launch_bloom(g->d_off, g->d_col, n, e, g->d_bloom, g->d_mtab, g->num_sms, st);
  if (le == cudaSuccess && want_labels)
    le = launch_label_stats(g->d_off, g->d_h, g->d_lab, n, g->d_lstat, d_lbad, g->num_sms, st);
  cudaEventRecord(e1, st);
  int maxdeg = 0;
  unsigned flags[2] = {1, 0};
  cudaError_t ce = cudaMemcpyAsync(&maxdeg, d_maxdeg, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(flags, d_asym, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  cudaError_t se = cudaStreamSynchronize(st);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (le != cudaSuccess) return cuda_error(le, "preprocessing kernels");
  if (ce != cudaSuccess) return cuda_error(ce, "read preprocessing results");
  if (se != cudaSuccess) return cuda_error(se, "sync after preprocessing");
  g->max_degree = maxdeg;
  g->sym = flags[0] == 0 ? 1 : 0;
  if (g->d_cerec && maxdeg >= (1 << 24)) {  // edge records carry class counts in 24 bits
    cudaFree(g->d_cerec);
    g->d_cerec = nullptr;
    g->bytes -= 2 * sizeof(int4) * (size_t)e;
  }
  if (want_labels && flags[1] != 0) {  // a label >= kLabelStats: per-label statistics unused
    cudaFree(g->d_lstat);
    g->d_lstat = nullptr;
    g->bytes -= sizeof(float2) * kLabelStats * ((size_t)n + 1);
    g->lstat_bad = true;
  }
  g->preprocess_ms += ms;
  if (g->d_lstat && e > 0) {
    fw_status gs = build_label_groups(g, st);
    if (gs != FW_OK) return gs;
  }
  return FW_OK;
}

static fw_status with_qctr(const fw_graph* g, const Job* jobs, int njobs, long long total, bool count,
                           cudaStream_t st) {
  unsigned long long* q = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&q), sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(queue counter)");
  e = cudaMemsetAsync(q, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = launch_walk(g, jobs, njobs, total, count, q, st);
  cudaError_t e2 = cudaFreeAsync(q, st);
  if (e != cudaSuccess) return cuda_error(e, "walk launch");
  if (e2 != cudaSuccess) return cuda_error(e2, "cudaFreeAsync(queue counter)");
  return FW_OK;
}

}  // namespace fw

using namespace fw;

// ---------------------------------------------------------------------------
extern "C" void fw_params_default(fw_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->p = 1.0f;
  p->q = 1.0f;
  p->gamma = 0.2f;
  p->mode = FW_MODE_AUTO;
}

extern "C" const char* fw_last_error(void) { return t_last_error.c_str(); }

extern "C" const char* fw_status_string(fw_status s) {
  switch (s) {
    case FW_OK: return "FW_OK";
    case FW_ERR_ARG: return "FW_ERR_ARG";
    case FW_ERR_CSR: return "FW_ERR_CSR";
    case FW_ERR_OOM: return "FW_ERR_OOM";
    case FW_ERR_CUDA: return "FW_ERR_CUDA";
    case FW_ERR_TIMEOUT: return "FW_ERR_TIMEOUT";
    case FW_ERR_DEVICE_CHECK: return "FW_ERR_DEVICE_CHECK";
    case FW_ERR_BUSY: return "FW_ERR_BUSY";
    case FW_ERR_UNSUPPORTED: return "FW_ERR_UNSUPPORTED";
  }
  return "FW_ERR_UNKNOWN";
}

extern "C" uint64_t fw_launch_count(void) { return g_launches.load(); }

// Host-side CSR validation (runs before any CUDA call).
static fw_status validate_host_csr(const int32_t* off, const int32_t* col, const float* h, int32_t n, int64_t e) {
  if (off[0] != 0) return set_error(FW_ERR_CSR, "offsets[0] != 0");
  for (int32_t v = 0; v < n; ++v)
    if (off[v + 1] < off[v]) return set_error(FW_ERR_CSR, "offsets not monotone at node " + std::to_string(v));
  if ((int64_t)off[n] != e) return set_error(FW_ERR_CSR, "offsets[n] != e");
  for (int32_t v = 0; v < n; ++v) {
    for (int32_t i = off[v]; i < off[v + 1]; ++i) {
      if (col[i] < 0 || col[i] >= n) return set_error(FW_ERR_CSR, "column out of range in row " + std::to_string(v));
      if (i + 1 < off[v + 1] && col[i + 1] <= col[i])
        return set_error(FW_ERR_CSR, "row " + std::to_string(v) + " not strictly increasing");
    }
  }
  if (h) {
    for (int64_t i = 0; i < e; ++i)
      if (!(h[i] > 0.0f) || !std::isfinite(h[i]))
        return set_error(FW_ERR_CSR, "weight " + std::to_string(i) + " not finite and > 0");
  }
  return FW_OK;
}

static void free_graph(fw_graph* g) {
  if (!g) return;
  cudaFree(g->d_off);
  cudaFree(g->d_col);
  cudaFree(g->d_h);
  cudaFree(g->d_lab);
  cudaFree(g->d_hmax);
  cudaFree(g->d_hsum);
  cudaFree(g->d_nrec);
  cudaFree(g->d_erec);
  cudaFree(g->d_cerec);
  cudaFree(g->d_lstat);
  cudaFree(g->d_h8);
  cudaFree(g->d_h8scale);
  cudaFree(g->d_bloom);
  cudaFree(g->d_mtab);
  cudaFree(g->d_lrec);
  cudaFree(g->d_gerec);
  cudaFree(g->d_gh);
  cudaFree(g->d_err);
  cudaFree(g->d_cnt);
  cudaFree(g->d_stage_starts);
  cudaFree(g->d_stage_out);
  for (cudaStream_t w : g->host_walk)
    if (w) cudaStreamDestroy(w);
  if (g->host_copy) cudaStreamDestroy(g->host_copy);
  for (cudaEvent_t ev : g->host_ev)
    if (ev) cudaEventDestroy(ev);
  delete g;
}

#define FW_TRY(call, what)                                   \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) {                                 \
      fw_status _s = cuda_error(_e, what);                   \
      free_graph(g);                                         \
      return _s;                                             \
    }                                                        \
  } while (0)

extern "C" fw_status fw_graph_create(const int32_t* offsets, const int32_t* cols, const float* weights,
                                     const uint8_t* labels, int32_t n, int64_t e, int32_t ptr_kind, void* stream,
                                     fw_graph** out) {
  if (!out) return set_error(FW_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!offsets || n < 0 || e < 0 || e > 2147483647LL || (e > 0 && !cols))
    return set_error(FW_ERR_ARG, "bad sizes or NULL arrays");
  if (ptr_kind != FW_PTR_HOST && ptr_kind != FW_PTR_DEVICE) return set_error(FW_ERR_ARG, "bad ptr_kind");
  if (ptr_kind == FW_PTR_HOST) {
    fw_status s = validate_host_csr(offsets, cols, weights, n, e);
    if (s != FW_OK) return s;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  fw_graph* g = new (std::nothrow) fw_graph();
  if (!g) return set_error(FW_ERR_OOM, "host allocation");
  g->n = n;
  g->e = e;
  FW_TRY(cudaGetDevice(&g->device), "cudaGetDevice");
  FW_TRY(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device), "cudaDeviceGetAttribute");
  const cudaMemcpyKind kind = ptr_kind == FW_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const size_t eb = (size_t)(e > 0 ? e : 1);
  FW_TRY(cudaMalloc(&g->d_off, sizeof(int32_t) * ((size_t)n + 1)), "cudaMalloc(offsets)");
  FW_TRY(cudaMalloc(&g->d_col, sizeof(int32_t) * eb), "cudaMalloc(cols)");
  if (weights) FW_TRY(cudaMalloc(&g->d_h, sizeof(float) * eb), "cudaMalloc(weights)");
  if (labels) FW_TRY(cudaMalloc(&g->d_lab, eb), "cudaMalloc(labels)");
  FW_TRY(cudaMalloc(&g->d_hmax, sizeof(float) * ((size_t)n + 1)), "cudaMalloc(h_MAX)");
  FW_TRY(cudaMalloc(&g->d_hsum, sizeof(float) * ((size_t)n + 1)), "cudaMalloc(h_SUM)");
  FW_TRY(cudaMalloc(&g->d_nrec, 2 * sizeof(int4) * ((size_t)n + 1)), "cudaMalloc(node records)");
  FW_TRY(cudaMalloc(&g->d_erec, 2 * sizeof(int4) * eb), "cudaMalloc(edge records)");
  if (weights) FW_TRY(cudaMalloc(&g->d_cerec, 2 * sizeof(int4) * eb), "cudaMalloc(class-ordered edge records)");
  FW_TRY(cudaMalloc(&g->d_err, 64), "cudaMalloc(error word)");
  FW_TRY(cudaMalloc(&g->d_cnt, sizeof(DevCounters)), "cudaMalloc(counters)");
  g->bytes = sizeof(int32_t) * ((size_t)n + 1) + eb * (4 + (weights ? 4 : 0) + (labels ? 1 : 0)) +
             2 * sizeof(float) * ((size_t)n + 1) + 2 * sizeof(int4) * ((size_t)n + 1) +
             (weights ? 4 : 2) * sizeof(int4) * eb + 64 + sizeof(DevCounters);
  FW_TRY(cudaMemsetAsync(g->d_err, 0, 64, st), "cudaMemsetAsync");
  FW_TRY(cudaMemsetAsync(g->d_cnt, 0, sizeof(DevCounters), st), "cudaMemsetAsync");
  FW_TRY(cudaMemcpyAsync(g->d_off, offsets, sizeof(int32_t) * ((size_t)n + 1), kind, st), "copy offsets");
  if (e > 0) FW_TRY(cudaMemcpyAsync(g->d_col, cols, sizeof(int32_t) * (size_t)e, kind, st), "copy cols");
  if (weights && e > 0) FW_TRY(cudaMemcpyAsync(g->d_h, weights, sizeof(float) * (size_t)e, kind, st), "copy weights");
  if (labels && e > 0) FW_TRY(cudaMemcpyAsync(g->d_lab, labels, (size_t)e, kind, st), "copy labels");
  if (ptr_kind == FW_PTR_DEVICE) {
    unsigned bits = 0;
    FW_TRY(launch_check_offsets(g->d_off, n, e, g->d_err, g->num_sms, st), "check offsets");
    FW_TRY(cudaMemcpyAsync(&bits, g->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "read check");
    FW_TRY(cudaStreamSynchronize(st), "sync");
    if (bits == 0) {
      FW_TRY(launch_check_rows(g->d_off, g->d_col, g->d_h, n, g->d_err, g->num_sms, st), "check rows");
      FW_TRY(cudaMemcpyAsync(&bits, g->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "read check");
      FW_TRY(cudaStreamSynchronize(st), "sync");
    }
    if (bits != 0) {
      free_graph(g);
      std::string why = (bits & 1u) ? "offsets invalid" : (bits & 2u) ? "column out of range"
                        : (bits & 4u) ? "row not strictly increasing" : "weight not finite and > 0";
      return set_error(FW_ERR_CSR, why);
    }
  }
  {
    fw_status fs = rebuild_derived(g, st);
    if (fs != FW_OK) {
      free_graph(g);
      return fs;
    }
  }
  {
    fw_status fs = graph_fingerprint(g, st, &g->fingerprint);
    if (fs != FW_OK) {
      free_graph(g);
      return fs;
    }
  }
  *out = g;
  return FW_OK;
}

extern "C" fw_status fw_graph_destroy(fw_graph* g) {
  if (!g) return set_error(FW_ERR_ARG, "graph is NULL");
  cudaDeviceSynchronize();
  free_graph(g);
  return FW_OK;
}

extern "C" fw_status fw_graph_info(const fw_graph* g, fw_graph_info_t* info) {
  if (!g || !info) return set_error(FW_ERR_ARG, "NULL argument");
  info->n = g->n;
  info->e = g->e;
  info->max_degree = g->max_degree;
  info->has_weights = g->d_h != nullptr;
  info->has_labels = g->d_lab != nullptr;
  info->cost_ratio = g->ratio_algo[FW_ALGO_NODE2VEC];
  for (int a = 0; a < 4; ++a) info->cost_ratios[a] = g->ratio_algo[a];
  info->fingerprint = g->fingerprint;
  info->preprocess_ms = g->preprocess_ms;
  info->device_bytes = g->bytes;
  info->symmetric = g->sym;
  info->weight_scale = g->d_h8 ? g->hscale : 0.0f;
  for (int a = 0; a < 4; ++a) {
    info->lane_max_degrees[a] = g->lane_max_algo[a];
    info->rjs_batches[a] = g->rjs_batch_algo[a];
    info->trial_budgets[a] = g->budget_algo[a];
  }
  return FW_OK;
}

extern "C" fw_status fw_graph_node_stats(const fw_graph* g, float* hmax, float* hsum, void* stream) {
  if (!g) return set_error(FW_ERR_ARG, "graph is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (hmax && g->n > 0) e = cudaMemcpyAsync(hmax, g->d_hmax, sizeof(float) * g->n, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && hsum && g->n > 0)
    e = cudaMemcpyAsync(hsum, g->d_hsum, sizeof(float) * g->n, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? FW_OK : cuda_error(e, "copy node stats");
}

extern "C" fw_status fw_graph_label_stats(const fw_graph* g, float* stats, void* stream) {
  if (!g || !stats) return set_error(FW_ERR_ARG, "NULL argument");
  if (!g->d_lstat) return set_error(FW_ERR_UNSUPPORTED, "no per-label statistics (no labels, or a label >= 8)");
  cudaError_t e = cudaMemcpyAsync(stats, g->d_lstat, sizeof(float2) * kLabelStats * (size_t)g->n,
                                  cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? FW_OK : cuda_error(e, "copy label statistics");
}

extern "C" fw_status fw_graph_quantize_weights(fw_graph* g, float* scale_out, void* stream) {
  if (!g) return set_error(FW_ERR_ARG, "graph is NULL");
  if (!g->d_h) return set_error(FW_ERR_UNSUPPORTED, "the graph has no weights");
  if (g->d_h8) {
    if (scale_out) *scale_out = g->hscale;
    return FW_OK;  // already quantized
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint8_t* codes = nullptr;
  float* scales = nullptr;
  cudaError_t e = cudaMalloc(&codes, (size_t)(g->e > 0 ? g->e : 1));
  if (e == cudaSuccess) e = cudaMalloc(&scales, sizeof(float) * ((size_t)g->n + 1));
  if (e != cudaSuccess) {
    cudaFree(codes);
    cudaFree(scales);
    return cuda_error(e, "cudaMalloc(weight codes)");
  }
  // the FP32 copy then holds the dequantized weights every derived structure is rebuilt from
  float max_scale = 0.0f;
  e = launch_quantize(g->d_off, g->d_h, g->d_hmax, g->n, codes, scales, &max_scale, g->d_err + 14, g->num_sms, st);
  if (e != cudaSuccess) {
    cudaFree(codes);
    cudaFree(scales);
    return cuda_error(e, "weight quantization");
  }
  g->d_h8 = codes;
  g->d_h8scale = scales;
  g->hscale = max_scale;
  g->bytes += (size_t)g->e + sizeof(float) * (size_t)g->n;
  fw_status s = rebuild_derived(g, st);
  if (s == FW_OK) s = graph_fingerprint(g, st, &g->fingerprint);
  if (s != FW_OK) return s;
  if (scale_out) *scale_out = max_scale;
  return FW_OK;
}

extern "C" fw_status fw_graph_weight_scales(const fw_graph* g, float* scales, void* stream) {
  if (!g || !scales) return set_error(FW_ERR_ARG, "NULL argument");
  if (!g->d_h8scale) return set_error(FW_ERR_UNSUPPORTED, "the graph's weights are not quantized");
  cudaError_t e = cudaMemcpyAsync(scales, g->d_h8scale, sizeof(float) * (size_t)g->n, cudaMemcpyDeviceToDevice,
                                  reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? FW_OK : cuda_error(e, "copy weight scales");
}

extern "C" fw_status fw_graph_set_cost_ratio(fw_graph* g, float ratio) {
  if (!g || !(ratio > 0.0f) || !std::isfinite(ratio)) return set_error(FW_ERR_ARG, "bad ratio");
  for (int a = 0; a < 4; ++a) g->ratio_algo[a] = ratio;
  return FW_OK;
}

extern "C" fw_status fw_walk(const fw_graph* g, const int32_t* starts, int32_t num_walkers, int32_t len, int32_t algo,
                             const fw_params* params, uint64_t seed, int32_t* out, void* stream) {
  if (!g) return set_error(FW_ERR_ARG, "graph is NULL");
  if (num_walkers < 0 || len < 0) return set_error(FW_ERR_ARG, "negative size");
  if (num_walkers > 0 && (!starts || !out)) return set_error(FW_ERR_ARG, "NULL starts/out");
  Job J;
  fw_status s = make_job(g, algo, params, seed, &J);
  if (s != FW_OK) return s;
  if (num_walkers == 0) return FW_OK;
  J.kind = JOB_WALK;
  J.starts = starts;
  J.out = out;
  J.num_walkers = num_walkers;
  J.len = len;
  J.gbase = 0;
  const bool count = params && (params->flags & FW_FLAG_COUNTERS);
  return with_qctr(g, &J, 1, num_walkers, count, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" fw_status fw_walk_ids(const fw_graph* g, const int32_t* starts, const uint32_t* walker_ids,
                                 int32_t num_walkers, int32_t len, int32_t algo, const fw_params* params, uint64_t seed,
                                 int32_t* out, void* stream) {
  if (!g) return set_error(FW_ERR_ARG, "graph is NULL");
  if (num_walkers < 0 || len < 0) return set_error(FW_ERR_ARG, "negative size");
  if (num_walkers > 0 && (!starts || !walker_ids || !out)) return set_error(FW_ERR_ARG, "NULL starts/ids/out");
  Job J;
  fw_status s = make_job(g, algo, params, seed, &J);
  if (s != FW_OK) return s;
  if (num_walkers == 0) return FW_OK;
  J.kind = JOB_WALK;
  J.starts = starts;
  J.wids = walker_ids;
  J.out = out;
  J.num_walkers = num_walkers;
  J.len = len;
  J.gbase = 0;
  const bool count = params && (params->flags & FW_FLAG_COUNTERS);
  return with_qctr(g, &J, 1, num_walkers, count, reinterpret_cast<cudaStream_t>(stream));
}

// Rows of at least this many bytes are walked in chunks so that the copy of
// finished chunks overlaps the walk of later ones.
static constexpr size_t kHostChunkBytes = 64ull << 20;

extern "C" fw_status fw_walk_host(fw_graph* g, const int32_t* starts, int32_t num_walkers, int32_t len, int32_t algo,
                                  const fw_params* params, uint64_t seed, int32_t* out, void* stream) {
  if (!g) return set_error(FW_ERR_ARG, "graph is NULL");
  if (num_walkers < 0 || len < 0) return set_error(FW_ERR_ARG, "negative size");
  if (num_walkers > 0 && (!starts || !out)) return set_error(FW_ERR_ARG, "NULL starts/out");
  Job J;
  fw_status s = make_job(g, algo, params, seed, &J);
  if (s != FW_OK) return s;
  std::unique_lock<std::mutex> lk(g->stage_mu, std::try_to_lock);
  if (!lk.owns_lock()) return set_error(FW_ERR_BUSY, "another fw_walk_host call is using this graph");
  if (num_walkers == 0) return FW_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t row = (size_t)len + 1;
  const size_t nin = (size_t)num_walkers, nout = (size_t)num_walkers * row;
  if (g->stage_starts_cap < nin) {
    cudaFree(g->d_stage_starts);
    g->d_stage_starts = nullptr;
    g->stage_starts_cap = 0;
    cudaError_t e = cudaMalloc(&g->d_stage_starts, nin * sizeof(int32_t));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(staging starts)");
    g->stage_starts_cap = nin;
  }
  if (g->stage_out_cap < nout) {
    cudaFree(g->d_stage_out);
    g->d_stage_out = nullptr;
    g->stage_out_cap = 0;
    cudaError_t e = cudaMalloc(&g->d_stage_out, nout * sizeof(int32_t));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(staging out)");
    g->stage_out_cap = nout;
  }
  if (!g->host_copy) {
    cudaError_t e = cudaSuccess;
    for (cudaStream_t& w : g->host_walk)
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->host_copy, cudaStreamNonBlocking);
    for (int i = 0; i <= kHostChunksMax && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&g->host_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_error(e, "create fw_walk_host streams");
  }
  // Chunk c holds walkers [c*W/K, (c+1)*W/K).  Chunks are walked in turn on
  // `stream` and kHostWalkStreams - 1 more streams, so that a chunk's tail
  // (its last walkers, a few blocks busy for many hops) shares the GPU with
  // the next chunks' bulk, and each chunk's rows are copied out on another
  // stream as soon as its walk ends.  Chunk c's walkers keep their
  // random-stream ids walker_base + index, so the rows equal one fw_walk.
  const size_t bytes_out = nout * sizeof(int32_t);
  const int K = (int)std::min<size_t>((size_t)kHostChunksMax, std::max<size_t>(1, bytes_out / kHostChunkBytes));
  const bool count = params && (params->flags & FW_FLAG_COUNTERS);
  cudaEvent_t* ev = g->host_ev;
  cudaError_t e = cudaMemcpyAsync(g->d_stage_starts, starts, nin * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(ev[kHostChunksMax], st);
  for (cudaStream_t w : g->host_walk)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(w, ev[kHostChunksMax], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(g->host_copy, ev[kHostChunksMax], 0);
  if (e != cudaSuccess) return cuda_error(e, "copy starts");
  s = FW_OK;
  for (int c = 0; c < K && s == FW_OK; ++c) {
    const size_t lo = nin * (size_t)c / (size_t)K, hi = nin * (size_t)(c + 1) / (size_t)K;
    if (hi == lo) continue;
    cudaStream_t ws = (c % kHostWalkStreams) ? g->host_walk[c % kHostWalkStreams - 1] : st;
    Job Jc = J;
    Jc.kind = JOB_WALK;
    Jc.starts = g->d_stage_starts + lo;
    Jc.out = g->d_stage_out + lo * row;
    Jc.num_walkers = (int32_t)(hi - lo);
    Jc.len = len;
    Jc.gbase = 0;
    Jc.walker_base = J.walker_base + (uint32_t)lo;
    s = with_qctr(g, &Jc, 1, (long long)(hi - lo), count, ws);
    if (s != FW_OK) break;
    e = cudaEventRecord(ev[c], ws);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->host_copy, ev[c], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out + lo * row, g->d_stage_out + lo * row, (hi - lo) * row * sizeof(int32_t),
                          cudaMemcpyDeviceToHost, g->host_copy);
    if (e != cudaSuccess) s = cuda_error(e, "copy out");
  }
  // join: `stream` waits for the copies (later work on it sees the rows), then all three drain
  cudaError_t e1 = cudaEventRecord(ev[kHostChunksMax], g->host_copy);
  if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(st, ev[kHostChunksMax], 0);
  cudaError_t e2 = cudaStreamSynchronize(g->host_copy);
  cudaError_t e3 = cudaSuccess;
  for (cudaStream_t w : g->host_walk) {
    const cudaError_t x = cudaStreamSynchronize(w);
    if (e3 == cudaSuccess) e3 = x;
  }
  cudaError_t e4 = cudaStreamSynchronize(st);
  if (s != FW_OK) return s;
  for (cudaError_t x : {e1, e2, e3, e4})
    if (x != cudaSuccess) return cuda_error(x, "sync");
  return FW_OK;
}

extern "C" fw_status fw_sample_hist(const fw_graph* g, int32_t v, int32_t v_prev, int32_t step, int32_t algo,
                                    const fw_params* params, uint64_t seed, int64_t ndraws, uint64_t* counts,
                                    void* stream) {
  if (!g) return set_error(FW_ERR_ARG, "graph is NULL");
  if (v < 0 || v >= g->n || v_prev < -1 || v_prev >= g->n || step < 0 || ndraws < 0 || !counts)
    return set_error(FW_ERR_ARG, "bad state or sizes");
  Job J;
  fw_status s = make_job(g, algo, params, seed, &J);
  if (s != FW_OK) return s;
  J.kind = JOB_HIST;
  J.hist = reinterpret_cast<unsigned long long*>(counts);
  J.hv = v;
  J.hprev = v_prev;
  J.hstep = step;
  const bool count = params && (params->flags & FW_FLAG_COUNTERS);
  const uint32_t base0 = J.walker_base;
  for (int64_t done = 0; done < ndraws;) {
    const int64_t chunk = (ndraws - done) < (1LL << 30) ? (ndraws - done) : (1LL << 30);
    J.walker_base = base0 + (uint32_t)done;
    J.num_walkers = (int32_t)chunk;
    J.len = 1;
    s = with_qctr(g, &J, 1, chunk, count, reinterpret_cast<cudaStream_t>(stream));
    if (s != FW_OK) return s;
    done += chunk;
  }
  return FW_OK;
}

extern "C" fw_status fw_step_plan(const fw_graph* g, const int32_t* v, const int32_t* v_prev, int32_t count,
                                  int32_t algo, const fw_params* params, float* bound, float* sum_hat, int32_t* mode,
                                  void* stream) {
  if (!g || count < 0 || (count > 0 && (!v || !v_prev || !bound || !sum_hat || !mode)))
    return set_error(FW_ERR_ARG, "bad arguments");
  Job J;
  fw_status s = make_job(g, algo, params, 0, &J);
  if (s != FW_OK) return s;
  cudaError_t e = launch_step_plan(g, J, v, v_prev, count, bound, sum_hat, mode, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? FW_OK : cuda_error(e, "step plan kernel");
}

extern "C" fw_status fw_counters_read(const fw_graph* g, fw_counters* out, void* stream) {
  if (!g || !out) return set_error(FW_ERR_ARG, "NULL argument");
  static_assert(sizeof(fw_counters) == sizeof(DevCounters), "counter layout");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(out, g->d_cnt, sizeof(fw_counters), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? FW_OK : cuda_error(e, "read counters");
}

extern "C" fw_status fw_counters_reset(fw_graph* g, void* stream) {
  if (!g) return set_error(FW_ERR_ARG, "graph is NULL");
  cudaError_t e = cudaMemsetAsync(g->d_cnt, 0, sizeof(DevCounters), reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? FW_OK : cuda_error(e, "reset counters");
}

extern "C" fw_status fw_graph_check(fw_graph* g, void* stream) {
  if (!g) return set_error(FW_ERR_ARG, "graph is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned bits = 0;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(&bits, g->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(g->d_err, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_error(e, "check");
  if (bits)
    return set_error(FW_ERR_DEVICE_CHECK, (bits & DEVERR_START) ? "a start node was outside [0, n)"
                                          : (bits & DEVERR_HUB) ? "a shared hub step did not complete in time"
                                                                : "device check failed");
  return FW_OK;
}
