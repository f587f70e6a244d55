// fw_internal.h -- host-side internals shared by the library's translation units.
#pragma once

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "fw_device.cuh"
#include "../../include/flexiwalk.h"

// fw_walk_host splits large requests into at most this many chunks
constexpr int kHostChunksMax = 16;
constexpr int kHostWalkStreams = 4;  // fw_walk_host: chunks in flight (the caller's stream and 3 more)

struct fw_graph {
  int device = 0;
  int num_sms = 0;
  int32_t n = 0;
  int64_t e = 0;
  int32_t max_degree = 0;
  int32_t* d_off = nullptr;
  int32_t* d_col = nullptr;
  float* d_h = nullptr;
  uint8_t* d_lab = nullptr;
  float* d_hmax = nullptr;
  float* d_hsum = nullptr;
  int4* d_nrec = nullptr;
  int4* d_erec = nullptr;
  int4* d_cerec = nullptr;     // edge records, rows partitioned by weight class (weighted graphs)
  float2* d_lstat = nullptr;  // per-label node statistics (nullptr: not available)
  bool lstat_bad = false;     // a label >= kLabelStats occurs
  uint32_t* d_bloom = nullptr; // blocked Bloom filters of the rows (membership pre-check)
  int32_t* d_mtab = nullptr;   // membership tables of the rows (exact; nullptr: not built)
  int4* d_lrec = nullptr;      // label-grouped view for metapath (nullptr: not built)
  int4* d_gerec = nullptr;
  float* d_gh = nullptr;
  uint8_t* d_h8 = nullptr;    // 8-bit weight codes after fw_graph_quantize_weights
  float* d_h8scale = nullptr; // per node: the scale of its row's codes
  float hscale = 0.0f;        // the largest per-node scale (reported by fw_graph_info)
  int32_t sym = 0;
  unsigned* d_err = nullptr;
  fw::DevCounters* d_cnt = nullptr;
  float ratio_algo[4] = {4.0f, 4.0f, 4.0f, 4.0f};  // r of Eq. (runtime) per algorithm (fw_algo order)
  // launch shape per algorithm (fw_params lane_max_degree, rjs_batch, trial_budget), tuned by method 2
  int32_t lane_max_algo[4] = {fw::kLaneMaxDegree, fw::kLaneMaxDegree, fw::kLaneMaxDegree, fw::kLaneMaxDegree};
  int32_t rjs_batch_algo[4] = {fw::kRjsBatchDefault, fw::kRjsBatchDefault, fw::kRjsBatchDefault,
                               fw::kRjsBatchDefault};
  float budget_algo[4] = {1.0f, 1.0f, 1.0f, 1.0f};
  unsigned long long fingerprint = 0;
  double preprocess_ms = 0.0;
  size_t bytes = 0;
  // staging of fw_walk_host
  std::mutex stage_mu;
  int32_t* d_stage_starts = nullptr;
  size_t stage_starts_cap = 0;
  int32_t* d_stage_out = nullptr;
  size_t stage_out_cap = 0;
  // pipelined fw_walk_host: a second walk stream, a copy stream and one event per chunk
  cudaStream_t host_walk[kHostWalkStreams - 1] = {};  // fw_walk_host: walk streams beside the caller's
  cudaStream_t host_copy = nullptr;
  cudaEvent_t host_ev[kHostChunksMax + 1] = {};
};

namespace fw {

extern std::atomic<unsigned long long> g_launches;

fw_status set_error(fw_status st, const std::string& msg);
fw_status cuda_error(cudaError_t err, const char* what);

DevGraph dev_graph(const fw_graph* g);

// Fill a job from the public parameters (validates them).
fw_status graph_fingerprint(const fw_graph* g, cudaStream_t st, unsigned long long* out);

fw_status make_job(const fw_graph* g, int32_t algo, const fw_params* params, uint64_t seed, Job* job);

// Launch the walk over `njobs` jobs (total walkers `total`; njobs <= kMaxJobs).
// `qctr` points to zeroed device counters the launch uses as walker queues:
// one for a single job, kAlgos (one per algorithm) for several.  Several
// jobs give one kernel launch per algorithm present.
cudaError_t launch_walk(const fw_graph* g, const Job* jobs, int njobs, long long total, bool count,
                        unsigned long long* qctr, cudaStream_t stream);
// Several jobs of any algorithms: one launch per algorithm present, on
// `stream` one after another, or (side: kAlgos - 1 helper streams, ev:
// kAlgos events) side by side, joined back into `stream`.  qctr: kAlgos
// zeroed counters.
cudaError_t launch_walk_mixed(const fw_graph* g, const Job* jobs, int njobs, bool count, unsigned long long* qctr,
                              cudaStream_t stream, const cudaStream_t* side = nullptr, cudaEvent_t* ev = nullptr);
constexpr int kQueueCounters = fw::kAlgos;  // counters a multi-job launch needs

// Cache the walk kernels' occupancy (call outside any stream capture).
cudaError_t prime_walk_occupancy();
cudaError_t prime_walk_mixed_occupancy();

cudaError_t launch_node_stats(const int32_t* off, const float* h, int32_t n, float* hmax, float* hsum, int4* nrec,
                              int* maxdeg, int num_sms, cudaStream_t stream);
cudaError_t launch_edge_records(const int32_t* col, const float* h, const uint8_t* lab, const int4* nrec, long long e,
                                int4* erec, int num_sms, cudaStream_t stream);
cudaError_t launch_label_stats(const int32_t* off, const float* h, const uint8_t* lab, int32_t n, float2* out,
                               unsigned* bad, int num_sms, cudaStream_t stream);
cudaError_t launch_class_group(const int32_t* off, const float* h, const int4* nrec, const int4* erec, int32_t n,
                               int4* cerec, int num_sms, cudaStream_t stream);
cudaError_t launch_label_group(const int32_t* off, const int32_t* col, const float* h, const uint8_t* lab,
                               const int4* nrec, const float2* lstat, int32_t n, int4* lrec, int4* gerec, float* gh,
                               int num_sms, cudaStream_t stream);
cudaError_t launch_symmetry(const int32_t* off, const int32_t* col, const float* h, int32_t n, long long e,
                            unsigned* flag, int num_sms, cudaStream_t stream);
cudaError_t launch_quantize(const int32_t* off, float* h, const float* hmax, int32_t n, uint8_t* codes,
                            float* scales, float* max_scale, unsigned* maxbits, int num_sms, cudaStream_t stream);
size_t bloom_bytes(int32_t n, long long e);
size_t table_bytes(int32_t n, long long e);
cudaError_t prime_preprocess_kernels();
cudaError_t launch_bloom(const int32_t* off, const int32_t* col, int32_t n, long long e, uint32_t* bloom,
                         int32_t* mtab, int num_sms, cudaStream_t stream);
fw_status rebuild_derived(fw_graph* g, cudaStream_t stream);
cudaError_t launch_check_offsets(const int32_t* off, int32_t n, int64_t e, unsigned* err, int num_sms,
                                 cudaStream_t stream);
cudaError_t launch_check_rows(const int32_t* off, const int32_t* col, const float* h, int32_t n, unsigned* err,
                              int num_sms, cudaStream_t stream);
cudaError_t launch_step_plan(const fw_graph* g, const Job& job, const int32_t* v, const int32_t* v_prev,
                             int32_t count, float* bound, float* sum_hat, int32_t* mode, cudaStream_t stream);

}  // namespace fw
