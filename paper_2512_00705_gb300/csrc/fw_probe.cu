// fw_probe.cu -- the random-access ceiling of device memory, for the walk
// kernel's roofline.
//
// Every eRJS trial, node-record fetch and membership probe of a walk is one
// dependent 32-byte gather at an unpredictable address.  On HBM such a
// gather costs a DRAM access whose price does not shrink with the bytes used
// (a 4-byte and a 32-byte gather take the same time, and the DRAM moves 64 to
// 128 bytes for either), so a kernel made of them is bound by the number of
// random accesses the memory system completes per second, well before the
// streaming copy bandwidth.  fw_gather_ceiling measures that number: every
// thread of 5 blocks of 256 per SM runs a chain of dependent 32-byte gathers
// over a caller-supplied table much larger than L2, each address derived
// from the previous load (the rate is the same from 5 to 8 blocks per SM, so
// this is the memory's limit, not the chains' latency; the walk kernel runs
// 4 blocks per SM).
#include "fw_internal.h"

namespace fw {
namespace {

constexpr int kProbeBlock = 256;
constexpr int kProbeBlocksPerSm = 5;  // enough chains to saturate the memory system
constexpr int kProbeChain = 64;       // dependent gathers per thread

__device__ __forceinline__ uint32_t probe_mix(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

__global__ void probe_fill_kernel(int4* __restrict__ t, unsigned long long n16) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n16;
       i += (unsigned long long)gridDim.x * blockDim.x)
    t[i] = make_int4((int)i, (int)((uint32_t)i * 2654435761u), 3, 4);
}

// record index = mix(chain state) & mask, mask + 1 = number of 32-byte records
__global__ void __launch_bounds__(kProbeBlock) probe_gather_kernel(const int4* __restrict__ t, unsigned long long mask,
                                                                   unsigned long long* __restrict__ sink) {
  uint32_t s = probe_mix(blockIdx.x * blockDim.x + threadIdx.x + 12345u);
  int acc = 0;
#pragma unroll 1
  for (int i = 0; i < kProbeChain; ++i) {
    const unsigned long long r =
        ((unsigned long long)probe_mix(s + (uint32_t)i * 0x9E3779B9u) * 0x100000001ull ^ (unsigned long long)i) & mask;
    int4 a, b;
    ld_record(t + 2ull * r, a, b);
    acc += a.x + b.w;
    s = (uint32_t)a.y ^ (uint32_t)acc;
  }
  if (acc == 0x7fffffff) atomicAdd(sink, 1ull);  // keeps the loads alive; practically never taken
}

}  // namespace
}  // namespace fw

using namespace fw;

extern "C" fw_status fw_gather_ceiling(void* table, uint64_t table_bytes, double* rate_out, void* stream) {
  if (!table || !rate_out) return set_error(FW_ERR_ARG, "NULL argument");
  if (table_bytes < (64ull << 20) || (table_bytes & (table_bytes - 1)) != 0)
    return set_error(FW_ERR_ARG, "table_bytes must be a power of two of at least 64 MiB");
  if ((reinterpret_cast<uintptr_t>(table) & 31u) != 0) return set_error(FW_ERR_ARG, "table must be 32-byte aligned");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_error(e, "device query");
  int4* t = static_cast<int4*>(table);
  // the sink word lives in the table's first record: the chains only read it
  unsigned long long* sink = reinterpret_cast<unsigned long long*>(t);
  const unsigned long long mask = table_bytes / 32 - 1;
  const int grid = sms * kProbeBlocksPerSm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.0f;
  if (e == cudaSuccess) {
    probe_fill_kernel<<<sms * 8, 256, 0, st>>>(t, table_bytes / 16);
    g_launches.fetch_add(1);
    e = cudaGetLastError();
  }
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // one warm-up, best of three
    e = cudaEventRecord(e0, st);
    probe_gather_kernel<<<grid, kProbeBlock, 0, st>>>(t, mask, sink);
    g_launches.fetch_add(1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_error(e, "gather ceiling probe");
  *rate_out = (double)grid * kProbeBlock * kProbeChain / (best * 1e-3);
  return FW_OK;
}
