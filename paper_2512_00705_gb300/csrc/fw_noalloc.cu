// fw_noalloc.cu -- fw_walk_host_noalloc: the host-buffer walk without any
// device allocation.
//
// Some callers cannot allocate device memory at the time they want a walk:
// hosts that hand every byte of the GPU to their own pool or arena up front
// (a stray cudaMalloc there fails or fragments the pool), real-time or
// embedded services that forbid allocation after start-up, and plug-ins that
// run inside someone else's process under a fixed memory budget.
// fw_walk_host needs device scratch (the staged start array, the staged
// rows, and the walk kernel's queue counter) and allocates it on first use;
// this variant keeps all of that scratch in one file-scope __device__ array
// of fixed size instead, so it makes no allocation call at all.
//
// The array is part of the library's device image: every GPU that loads the
// library holds kNoAllocScratchBytes for it until the process exits.  All
// calls share it and it keeps the previous call's contents; the queue
// counter is cleared at the start of every call.  Calls from this process
// are serialised by a lock (a concurrent call returns FW_ERR_BUSY) and each
// call waits for its own GPU work before returning, so two calls only
// overlap on the GPU if one of them failed after enqueueing work; such
// overlapping calls race on the shared array.
//
// Every call looks up the array's device address on the current device
// (cudaGetSymbolAddress, under the lock), so a device reset and a reloaded
// module leave no stale address behind; the first call on a device also
// loads the module that holds the array, so make it before any stream
// capture.
#include <mutex>

#include "fw_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;   // 16 MiB
constexpr size_t kHeader = 256;                      // queue counter + padding

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device (the symbol's
// host-side name is only a stand-in).
fw_status scratch_address(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return fw::cuda_error(e, "cudaGetSymbolAddress(no-alloc scratch)");
  *out = static_cast<unsigned char*>(p);
  return FW_OK;
}

}  // namespace

extern "C" fw_status fw_walk_host_noalloc(const fw_graph* g, const int32_t* starts, int32_t num_walkers, int32_t len,
                                          int32_t algo, const fw_params* params, uint64_t seed, int32_t* out,
                                          void* stream) {
  using namespace fw;
  if (!g) return set_error(FW_ERR_ARG, "graph is NULL");
  if (num_walkers < 0 || len < 0) return set_error(FW_ERR_ARG, "negative size");
  if (num_walkers > 0 && (!starts || !out)) return set_error(FW_ERR_ARG, "NULL starts/out");
  // staged starts, then staged rows starting on a 256-byte boundary; each
  // term is bounded before it is added, so no product or sum can wrap
  const size_t limit = kNoAllocScratchBytes - kHeader;
  const size_t in_bytes = (size_t)num_walkers * sizeof(int32_t);  // < 2^33
  const size_t rows_off = (in_bytes + 255) & ~(size_t)255;
  const size_t row_bytes = ((size_t)len + 1) * sizeof(int32_t);    // < 2^34
  const bool fits = rows_off <= limit && (num_walkers == 0 || row_bytes <= (limit - rows_off) / (size_t)num_walkers);
  if (!fits)
    return set_error(FW_ERR_ARG, "request of " + std::to_string(num_walkers) + " walkers x " +
                                     std::to_string((long long)len + 1) +
                                     " row entries does not fit the staging array; fw_walk_host_noalloc holds at most " +
                                     std::to_string(limit) + " bytes (use fw_walk_host)");
  const size_t out_bytes = (size_t)num_walkers * row_bytes;
  Job J;
  fw_status s = make_job(g, algo, params, seed, &J);
  if (s != FW_OK) return s;
  std::unique_lock<std::mutex> lk(g_noalloc_mu, std::try_to_lock);
  if (!lk.owns_lock()) return set_error(FW_ERR_BUSY, "another fw_walk_host_noalloc call is in progress");
  if (num_walkers == 0) return FW_OK;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev != g->device) return set_error(FW_ERR_ARG, "the graph lives on another device than the current one");
  unsigned char* base = nullptr;
  s = scratch_address(&base);
  if (s != FW_OK) return s;
  auto* qctr = reinterpret_cast<unsigned long long*>(base);
  auto* d_starts = reinterpret_cast<int32_t*>(base + kHeader);
  auto* d_out = reinterpret_cast<int32_t*>(base + kHeader + rows_off);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  J.kind = JOB_WALK;
  J.starts = d_starts;
  J.out = d_out;
  J.num_walkers = num_walkers;
  J.len = len;
  J.gbase = 0;
  const bool count = params && (params->flags & FW_FLAG_COUNTERS);
  e = cudaMemsetAsync(qctr, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_starts, starts, in_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_walk(g, &J, 1, num_walkers, count, qctr, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, out_bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    fw_status fs = cuda_error(e, "fw_walk_host_noalloc");
    cudaStreamSynchronize(st);  // best effort: let enqueued work finish before the next call
    return fs;
  }
  return FW_OK;
}
