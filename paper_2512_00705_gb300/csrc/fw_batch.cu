// fw_batch.cu -- many walk jobs per launch, and a CUDA-graph plan that
// replays such a batch.
//
// A batch is a table of up to 64 jobs of any sizes, lengths, algorithms and
// parameters (fw_walk_mixed.cu): the jobs of one algorithm form one walker
// queue walked by one persistent launch of the kernel compiled for that
// algorithm, so small jobs do not leave the GPU idle and long jobs do not
// hold a launch of their own.  Each job's rows equal those of a separate
// fw_walk call with the same arguments: every random draw and every sampler
// choice depends only on the walker's own job.
#include <vector>

#include "fw_internal.h"

namespace fw {

static fw_status build_table(const fw_graph* g, const fw_job* jobs, int32_t njobs, std::vector<Job>* tab,
                             long long* total, bool* count) {
  tab->clear();
  *total = 0;
  *count = false;
  for (int32_t i = 0; i < njobs; ++i) {
    const fw_job& in = jobs[i];
    if (in.num_walkers < 0 || in.len < 0) return set_error(FW_ERR_ARG, "job " + std::to_string(i) + ": negative size");
    if (in.num_walkers > 0 && (!in.starts || !in.out))
      return set_error(FW_ERR_ARG, "job " + std::to_string(i) + ": NULL starts/out");
    Job J;
    fw_status s = make_job(g, in.algo, &in.params, in.seed, &J);
    if (s != FW_OK) return set_error(s, "job " + std::to_string(i) + ": " + fw_last_error());
    if (in.num_walkers == 0) continue;
    J.kind = JOB_WALK;
    J.starts = in.starts;
    J.out = in.out;
    J.num_walkers = in.num_walkers;
    J.len = in.len;
    J.gbase = *total;
    *total += in.num_walkers;
    *count = *count || (in.params.flags & FW_FLAG_COUNTERS);
    tab->push_back(J);
  }
  return FW_OK;
}

}  // namespace fw

using namespace fw;

extern "C" fw_status fw_walk_batch(const fw_graph* g, const fw_job* jobs, int32_t njobs, void* stream) {
  if (!g || njobs < 0 || (njobs > 0 && !jobs)) return set_error(FW_ERR_ARG, "bad arguments");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (int32_t first = 0; first < njobs; first += kMaxJobs) {
    const int32_t m = (njobs - first) < kMaxJobs ? (njobs - first) : kMaxJobs;
    std::vector<Job> tab;
    long long total = 0;
    bool count = false;
    fw_status s = build_table(g, jobs + first, m, &tab, &total, &count);
    if (s != FW_OK) return s;
    if (total == 0) continue;
    unsigned long long* q = nullptr;  // one walker queue per algorithm
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&q), sizeof(unsigned long long) * kQueueCounters, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(queue counter)");
    e = cudaMemsetAsync(q, 0, sizeof(unsigned long long) * kQueueCounters, st);
    if (e == cudaSuccess) e = launch_walk(g, tab.data(), (int)tab.size(), total, count, q, st);
    cudaError_t e2 = cudaFreeAsync(q, st);
    if (e != cudaSuccess) return cuda_error(e, "batch launch");
    if (e2 != cudaSuccess) return cuda_error(e2, "cudaFreeAsync(queue counter)");
  }
  return FW_OK;
}

struct fw_batch_plan {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long* qctr = nullptr;  // kQueueCounters queue counters per chunk of 64 jobs
  int kernels = 0;                     // walk kernels per replay
};

static void free_plan(fw_batch_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  cudaFree(p->qctr);
  delete p;
}

extern "C" fw_status fw_batch_plan_create(const fw_graph* g, const fw_job* jobs, int32_t njobs,
                                          fw_batch_plan** out) {
  if (!out) return set_error(FW_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!g || njobs < 0 || (njobs > 0 && !jobs)) return set_error(FW_ERR_ARG, "bad arguments");
  const int32_t chunks = (njobs + kMaxJobs - 1) / kMaxJobs;
  std::vector<std::vector<Job>> tabs(chunks);
  std::vector<long long> totals(chunks);
  std::vector<bool> counts(chunks);
  for (int32_t c = 0; c < chunks; ++c) {
    const int32_t first = c * kMaxJobs;
    const int32_t m = (njobs - first) < kMaxJobs ? (njobs - first) : kMaxJobs;
    bool cnt = false;
    fw_status s = build_table(g, jobs + first, m, &tabs[c], &totals[c], &cnt);
    if (s != FW_OK) return s;
    counts[c] = cnt;
  }
  fw_batch_plan* p = new (std::nothrow) fw_batch_plan();
  if (!p) return set_error(FW_ERR_OOM, "host allocation");
  cudaError_t e = cudaMalloc(&p->qctr, sizeof(unsigned long long) * kQueueCounters * (chunks > 0 ? chunks : 1));
  if (e != cudaSuccess) {
    free_plan(p);
    return cuda_error(e, "cudaMalloc(plan counters)");
  }
  e = prime_walk_occupancy();  // occupancy queries stay outside the capture
  if (e != cudaSuccess) {
    free_plan(p);
    return cuda_error(e, "occupancy query");
  }
  // capture on a private stream (the per-algorithm launches of a chunk fork
  // onto helper streams and join back, so they overlap), then instantiate
  cudaStream_t cap = nullptr, side[kAlgos - 1] = {};
  cudaEvent_t ev[kAlgos] = {};
  e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  for (int i = 0; i < kAlgos - 1 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking);
  for (int i = 0; i < kAlgos && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  const bool capturing = e == cudaSuccess;
  for (int32_t c = 0; c < chunks && e == cudaSuccess; ++c) {
    if (totals[c] == 0) continue;
    unsigned long long* q = p->qctr + (size_t)c * kQueueCounters;
    e = cudaMemsetAsync(q, 0, sizeof(unsigned long long) * kQueueCounters, cap);
    const unsigned long long before = g_launches.load();
    if (e == cudaSuccess) {
      e = tabs[c].size() == 1 ? launch_walk(g, tabs[c].data(), 1, totals[c], counts[c], q, cap)
                              : launch_walk_mixed(g, tabs[c].data(), (int)tabs[c].size(), counts[c], q, cap, side, ev);
    }
    const unsigned long long launched = g_launches.load() - before;
    p->kernels += (int)launched;
    g_launches.fetch_sub(launched);  // counted when the plan is replayed
  }
  if (capturing) {
    cudaError_t e2 = cudaStreamEndCapture(cap, &p->graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  for (cudaStream_t x : side)
    if (x) cudaStreamDestroy(x);
  if (cap) cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    free_plan(p);
    return cuda_error(e, "capture of the batch launch");
  }
  *out = p;
  return FW_OK;
}

extern "C" fw_status fw_batch_plan_launch(fw_batch_plan* p, void* stream) {
  if (!p || !p->exec) return set_error(FW_ERR_ARG, "plan is NULL");
  cudaError_t e = cudaGraphLaunch(p->exec, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "cudaGraphLaunch");
  g_launches.fetch_add((unsigned long long)p->kernels);
  return FW_OK;
}

extern "C" fw_status fw_batch_plan_destroy(fw_batch_plan* p) {
  if (!p) return set_error(FW_ERR_ARG, "plan is NULL");
  cudaDeviceSynchronize();
  free_plan(p);
  return FW_OK;
}
