// fw_walk_mixed.cu -- launches over tables of several jobs.
//
// A table of up to 64 jobs is split by algorithm.  The jobs of one
// algorithm form one walker queue (one concatenated index space) walked by
// one persistent launch of the walk kernel compiled for that algorithm, so
// jobs of very different sizes and lengths still share the GPU.  A single
// kernel that reads the algorithm per job, or that switches between
// algorithm-specialised loops, keeps every algorithm's state live and spills:
// its node2vec steps measured twice as slow as the specialised kernel's.
// The per-algorithm launches run one after another on the caller's stream,
// or side by side on helper streams when the caller provides them (the batch
// plans do, inside their CUDA graph), so that one launch's last walkers share
// the GPU with the next launch's first ones.
#include "fw_internal.h"
#include "fw_walk.cuh"

namespace fw {
namespace {

template <bool COUNT>
cudaError_t launch_group(int a, const fw_graph* g, const Job* jobs, int njobs, long long total,
                         unsigned long long* qctr, cudaStream_t st) {
  switch (a) {
    case ALGO_WEIGHTED: return launch_walk_t<kMaxJobs, COUNT, ALGO_WEIGHTED>(g, jobs, njobs, total, qctr, st);
    case ALGO_NODE2VEC: return launch_walk_t<kMaxJobs, COUNT, ALGO_NODE2VEC>(g, jobs, njobs, total, qctr, st);
    case ALGO_METAPATH: return launch_walk_t<kMaxJobs, COUNT, ALGO_METAPATH>(g, jobs, njobs, total, qctr, st);
    default: return launch_walk_t<kMaxJobs, COUNT, ALGO_PAGERANK2>(g, jobs, njobs, total, qctr, st);
  }
}

template <bool COUNT, bool SHARE = false>
cudaError_t prime_groups(int* b) {
  cudaError_t e = walk_blocks_per_sm<kMaxJobs, COUNT, ALGO_WEIGHTED, SHARE>(b);
  if (e == cudaSuccess) e = walk_blocks_per_sm<kMaxJobs, COUNT, ALGO_NODE2VEC, SHARE>(b);
  if (e == cudaSuccess) e = walk_blocks_per_sm<kMaxJobs, COUNT, ALGO_METAPATH, SHARE>(b);
  if (e == cudaSuccess) e = walk_blocks_per_sm<kMaxJobs, COUNT, ALGO_PAGERANK2, SHARE>(b);
  return e;
}

}  // namespace

cudaError_t prime_walk_mixed_occupancy() {
  int b;
  cudaError_t e = prime_groups<false>(&b);
  if (e == cudaSuccess) e = prime_groups<true>(&b);
  if (e == cudaSuccess) e = prime_groups<false, true>(&b);
  return e;
}

cudaError_t launch_walk_mixed(const fw_graph* g, const Job* jobs, int njobs, bool count, unsigned long long* qctr,
                              cudaStream_t stream, const cudaStream_t* side, cudaEvent_t* ev) {
  if (njobs < 1 || njobs > kMaxJobs) return cudaErrorInvalidValue;
  Job grp[kMaxJobs];
  int present[kAlgos], np = 0;
  long long totals[kAlgos];
  int firsts[kAlgos], counts[kAlgos];
  int m = 0;
  for (int a = 0; a < kAlgos; ++a) {
    firsts[a] = m;
    totals[a] = 0;
    for (int i = 0; i < njobs; ++i) {
      if (jobs[i].algo != a) continue;
      grp[m] = jobs[i];
      grp[m].gbase = totals[a];  // index space of the algorithm's queue
      totals[a] += jobs[i].num_walkers;
      ++m;
    }
    counts[a] = m - firsts[a];
    if (totals[a] > 0) present[np++] = a;
  }
  if (m != njobs) return cudaErrorInvalidValue;  // an algorithm outside 0..kAlgos-1
  const bool fork = side && ev && np > 1;
  cudaError_t e = cudaSuccess;
  if (fork) {  // helper stream i waits for the work queued before the launch on `stream`
    e = cudaEventRecord(ev[0], stream);
    for (int i = 1; i < np && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(side[i - 1], ev[0], 0);
  }
  for (int i = 0; i < np && e == cudaSuccess; ++i) {
    const int a = present[i];
    cudaStream_t st = (fork && i > 0) ? side[i - 1] : stream;
    e = count ? launch_group<true>(a, g, grp + firsts[a], counts[a], totals[a], qctr + a, st)
              : launch_group<false>(a, g, grp + firsts[a], counts[a], totals[a], qctr + a, st);
  }
  if (fork) {  // `stream` waits for the helper streams
    for (int i = 1; i < np && e == cudaSuccess; ++i) {
      e = cudaEventRecord(ev[i], side[i - 1]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev[i], 0);
    }
  }
  return e;
}

}  // namespace fw
