// fw_server.cu -- continuous batching of walk queries against a resident graph.
//
// A worker thread owns the device side.  Queries arrive from any thread
// (fw_server_submit) into a FIFO queue.  The worker
//   1. retires finished waves: polls each in-flight wave's completion event
//      (cudaEventQuery, never a blocking wait), marks its queries done and
//      returns their device memory to the arena;
//   2. admits queries in arrival order within two size classes (small, and
//      large: W x L at least large_query_steps) while the device arena (the
//      memory budget) has room for their staged starts and rows; small
//      queries go first, so a burst of large ones does not hold them up, and a
//      large query that has waited kLargeAging goes first and, while it waits
//      for memory, stops small admissions, so large queries are not starved;
//   3. launches each class's admitted queries as one wave on a free stream
//      (large waves leave an eighth of the streams, at least one, to small
//      ones): upload of
//      the queries' starts, one batched walk (up to 64 queries; one launch
//      per algorithm present, side by side on the wave's helper streams,
//      each algorithm's queries one shared walker queue, so the wave ends
//      with its slowest algorithm rather than after the sum of all), a count
//      of the wave's hops on the device, download of the
//      queries' rows and of the count, an event.  Copies of consecutive
//      queries whose host and device ranges are both contiguous merge.  The CUDA calls run without
//      the server lock, so submitting and polling threads are not held up by
//      them.
// Clients may submit and poll many queries per call (one lock each), which
// keeps a single client thread ahead of tens of thousands of queries/s.
// Copies to or from pageable host memory would block the worker until the
// wave is done (the driver stages them synchronously), so queries whose
// buffers are not page-locked go through a page-locked mirror of the arena
// (allocated on first need): the worker copies their starts into it before
// the upload and their rows out of it after the wave, and every device copy
// stays asynchronous, so waves overlap for any caller.
// Waves on different streams overlap on the device, and queries that arrive
// while waves run join the next wave: continuous batching.  A query's rows
// are identical to those of fw_walk_host with the same arguments, alone or
// in any mix (every draw and sampler choice depends only on its own walkers).
// All waits are on the host and bounded by the caller's timeout.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fw_arena.h"
#include "fw_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { REQ_PENDING = 0, REQ_ADMITTED = 1, REQ_LAUNCHED = 2, REQ_DONE = 3, REQ_FAILED = 4 };

struct Request {
  uint64_t id = 0;
  const int32_t* starts = nullptr;  // host
  int32_t* out = nullptr;           // host
  int32_t num_walkers = 0, len = 0, algo = 0;
  fw_params params;
  uint64_t seed = 0;
  size_t in_bytes = 0, row_bytes = 0;  // staged starts, rows (both multiples of 4)
  size_t starts_off = 0, rows_off = 0;  // their offsets in the arena (and in the mirror)
  bool pinned_in = false, pinned_out = false;  // caller buffers page-locked (copied directly)
  Clock::time_point t_submit, t_launch, t_done;
  int state = REQ_PENDING;
  int cls = 0;  // size class: 0 small, 1 large
  fw_status status = FW_OK;
  std::string error;
};


struct Wave {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaStream_t side[fw::kAlgos - 1] = {};  // the other algorithms' launches run beside the first one's
  cudaEvent_t fork[fw::kAlgos] = {};
  unsigned long long* qctr = nullptr;       // kQueueCounters queue counters, then the hop count (device)
  unsigned long long* hops_host = nullptr;  // the wave's hop count, copied back (pinned host)
  std::vector<Request*> reqs;
  uint64_t copies = 0;  // starts and rows copies the wave enqueued (after merging)
  int cls = 0;          // size class of the wave's queries
  bool busy = false;
};

void destroy_wave(Wave& w) {
  if (w.stream) cudaStreamDestroy(w.stream);
  if (w.done) cudaEventDestroy(w.done);
  for (cudaStream_t& st : w.side)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t& ev : w.fork)
    if (ev) cudaEventDestroy(ev);
}

constexpr int kHopSlot = 8;  // index of the hop count in a wave's 256-byte counter block
// A large query waiting longer than this is admitted before small ones.
constexpr std::chrono::milliseconds kLargeAging{100};

// Hops of a wave: row entries after the start column that hold a node (not
// -1), over the rows of up to kMaxJobs queries; one atomic per warp.
struct HopRows {
  const int32_t* rows[fw::kMaxJobs];
  int32_t walkers[fw::kMaxJobs];
  int32_t width[fw::kMaxJobs];  // len + 1
  int32_t n;
};

__global__ void count_hops_kernel(HopRows t, unsigned long long* __restrict__ hops) {
  unsigned long long local = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int j = 0; j < t.n; ++j) {
    const int32_t w = t.width[j];
    const long long total = (long long)t.walkers[j] * w;
    const int32_t* r = t.rows[j];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride)
      local += (i % w != 0 && __ldg(r + i) >= 0) ? 1ull : 0ull;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(hops, local);
}

}  // namespace

struct fw_server {
  const fw_graph* g = nullptr;
  fw_server_config cfg;
  unsigned char* arena_mem = nullptr;
  unsigned char* mirror = nullptr;  // page-locked mirror of the arena (pageable callers), or nullptr
  bool mirror_failed = false;
  fw::Arena* arena = nullptr;
  std::vector<Wave> waves;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending[2];     // per size class: 0 small, 1 large (W x L >= large_query_steps)
  std::vector<Request*> admitted[2];   // the next wave of each class
  std::unordered_map<uint64_t, Request*> reqs;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  // statistics
  std::vector<double> latencies_ms, queue_ms, wave_ms;  // submit -> done, submit -> launch, launch -> done
  uint64_t completed = 0, failed = 0, waves_launched = 0, queries_in_waves = 0, walker_steps = 0;
  unsigned long long* hops_host = nullptr;  // pinned, one slot per wave
  size_t peak_arena = 0;
  int peak_inflight = 0;
  double enqueue_ms = 0;  // host time spent enqueueing waves
  uint64_t copies = 0;    // starts and rows copies enqueued
  size_t rows_cursor = 0; // end of the last admitted query's rows (next-fit placement)
};

namespace {

void finish(fw_server* s, Request* r, fw_status st, const std::string& err) {
  r->state = st == FW_OK ? REQ_DONE : REQ_FAILED;
  r->status = st;
  r->error = err;
  r->t_done = Clock::now();
  if (st == FW_OK) {
    s->completed++;
    s->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    s->queue_ms.push_back(std::chrono::duration<double, std::milli>(r->t_launch - r->t_submit).count());
    s->wave_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_launch).count());
  } else {
    s->failed++;
  }
}

// Copies of one direction on one stream; a copy whose source and destination
// both continue the pending one extends it (rows of queries admitted one after
// another lie back to back in the arena, and clients often take their output
// buffers back to back from one pool): fewer, larger DMA transfers, which
// reach a higher share of the host link than many small ones.
struct CopyRun {
  cudaMemcpyKind kind;
  cudaStream_t stream;
  unsigned char* dst = nullptr;
  const unsigned char* src = nullptr;
  size_t n = 0;
  uint64_t issued = 0;  // copies enqueued
  CopyRun(cudaMemcpyKind k, cudaStream_t st) : kind(k), stream(st) {}
  cudaError_t add(unsigned char* d, const unsigned char* sp, size_t bytes) {
    if (bytes == 0) return cudaSuccess;
    if (n && d == dst + n && sp == src + n) {
      n += bytes;
      return cudaSuccess;
    }
    const cudaError_t e = flush();
    dst = d;
    src = sp;
    n = bytes;
    return e;
  }
  cudaError_t flush() {
    if (!n) return cudaSuccess;
    const cudaError_t e = cudaMemcpyAsync(dst, src, n, kind, stream);
    n = 0;
    ++issued;
    return e;
  }
};

// Enqueue the GPU work of one wave: stage the starts, walk (one launch per
// algorithm present), copy the rows out, record the wave's event.  Called
// WITHOUT the server lock, so submit / poll are not held up by the CUDA
// calls: it only reads the requests' immutable fields and uses the wave,
// which the worker reserved.  Returns the first failing CUDA call's error.
cudaError_t enqueue_wave(fw_server* s, Wave& w, const std::vector<Request*>& batch) {
  using namespace fw;
  *w.hops_host = 0;
  CopyRun up(cudaMemcpyHostToDevice, w.stream), down(cudaMemcpyDeviceToHost, w.stream);
  std::vector<Job> tab;
  tab.reserve(batch.size());
  long long total = 0;
  cudaError_t e = cudaSuccess;
  for (Request* r : batch) {
    Job J;
    if (make_job(s->g, r->algo, &r->params, r->seed, &J) != FW_OK) return cudaErrorInvalidValue;  // checked at submit
    int32_t* d_starts = reinterpret_cast<int32_t*>(s->arena_mem + r->starts_off);
    int32_t* d_out = reinterpret_cast<int32_t*>(s->arena_mem + r->rows_off);
    J.kind = JOB_WALK;
    J.starts = d_starts;
    J.out = d_out;
    J.num_walkers = r->num_walkers;
    J.len = r->len;
    J.gbase = total;
    total += r->num_walkers;
    tab.push_back(J);
    const unsigned char* src = reinterpret_cast<const unsigned char*>(r->starts);
    if (!r->pinned_in && s->mirror) {  // pageable starts: through the page-locked mirror
      std::memcpy(s->mirror + r->starts_off, r->starts, r->in_bytes);
      src = s->mirror + r->starts_off;
    }
    if (e == cudaSuccess) e = up.add(s->arena_mem + r->starts_off, src, r->in_bytes);
  }
  if (e == cudaSuccess) e = up.flush();
  if (e == cudaSuccess) e = cudaMemsetAsync(w.qctr, 0, sizeof(unsigned long long) * (kHopSlot + 1), w.stream);
  if (e == cudaSuccess && total > 0)
    e = tab.size() == 1 ? launch_walk(s->g, tab.data(), 1, total, false, w.qctr, w.stream)
                        : launch_walk_mixed(s->g, tab.data(), (int)tab.size(), false, w.qctr, w.stream, w.side, w.fork);
  if (e == cudaSuccess && total > 0) {
    HopRows hr;
    hr.n = (int)tab.size();
    long long entries = 0;
    for (int j = 0; j < hr.n; ++j) {
      hr.rows[j] = tab[j].out;
      hr.walkers[j] = tab[j].num_walkers;
      hr.width[j] = tab[j].len + 1;
      entries += (long long)tab[j].num_walkers * (tab[j].len + 1);
    }
    const long long want = (entries + 255) / 256, cap = 4ll * s->g->num_sms;
    count_hops_kernel<<<(int)(want < cap ? want : cap), 256, 0, w.stream>>>(hr, w.qctr + kHopSlot);
    g_launches.fetch_add(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w.hops_host, w.qctr + kHopSlot, sizeof(unsigned long long), cudaMemcpyDeviceToHost, w.stream);
  for (Request* r : batch) {
    if (e != cudaSuccess) break;
    // pageable rows land in the mirror and are copied out when the wave retires
    unsigned char* dst = (!r->pinned_out && s->mirror) ? s->mirror + r->rows_off
                                                        : reinterpret_cast<unsigned char*>(r->out);
    e = down.add(dst, s->arena_mem + r->rows_off, r->row_bytes);
  }
  if (e == cudaSuccess) e = down.flush();
  w.copies = up.issued + down.issued;
  if (e == cudaSuccess) e = cudaEventRecord(w.done, w.stream);
  if (e != cudaSuccess) cudaStreamSynchronize(w.stream);  // let what was enqueued finish before its memory is reused
  return e;
}

// Launch the admitted queries as one wave on the free wave w.  Called and
// returns with the lock held; drops it around the CUDA calls.
void launch_wave(fw_server* s, Wave& w, int cls, std::unique_lock<std::mutex>& lk) {
  std::vector<Request*> batch;
  batch.swap(s->admitted[cls]);
  w.cls = cls;
  const auto now = Clock::now();
  for (Request* r : batch) {
    r->state = REQ_LAUNCHED;
    r->t_launch = now;
  }
  w.busy = true;  // reserved: no other launch takes this wave meanwhile
  bool need_mirror = false;
  for (Request* r : batch) need_mirror = need_mirror || !r->pinned_in || !r->pinned_out;
  lk.unlock();
  if (need_mirror && !s->mirror && !s->mirror_failed) {  // only the worker allocates it
    unsigned char* m = nullptr;
    if (cudaMallocHost(reinterpret_cast<void**>(&m), s->cfg.mem_budget) == cudaSuccess) {
      s->mirror = m;
    } else {
      cudaGetLastError();  // not sticky; pageable queries then copy directly (synchronously)
      s->mirror_failed = true;
    }
  }
  const auto t0 = Clock::now();
  const cudaError_t e = enqueue_wave(s, w, batch);
  const double host_ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  lk.lock();
  s->enqueue_ms += host_ms;
  s->copies += w.copies;
  if (e != cudaSuccess) {
    const std::string msg = std::string("wave launch: ") + cudaGetErrorString(e);
    for (Request* r : batch) {
      s->arena->release(r->rows_off, r->row_bytes);
      s->arena->release(r->starts_off, r->in_bytes);
      finish(s, r, FW_ERR_CUDA, msg);
    }
    w.busy = false;
    s->cv_done.notify_all();
    return;
  }
  w.reqs = std::move(batch);
  s->waves_launched++;
  s->queries_in_waves += w.reqs.size();
}

void worker_main(fw_server* s) {
  cudaSetDevice(s->g->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool progress = false;
    int inflight = 0;
    // 1. retire finished waves
    for (Wave& w : s->waves) {
      if (!w.busy) continue;
      const cudaError_t q = cudaEventQuery(w.done);
      if (q == cudaErrorNotReady) {
        ++inflight;
        continue;
      }
      const fw_status st = q == cudaSuccess ? FW_OK : FW_ERR_CUDA;
      const std::string msg = q == cudaSuccess ? std::string() : std::string("wave: ") + cudaGetErrorString(q);
      if (q == cudaSuccess) {
        s->walker_steps += *w.hops_host;
        if (s->mirror) {  // rows of pageable callers: out of the mirror, without holding the lock
          lk.unlock();
          for (Request* r : w.reqs)
            if (!r->pinned_out)
              std::memcpy(r->out, s->mirror + r->rows_off, r->row_bytes);
          lk.lock();
        }
      }
      for (Request* r : w.reqs) {
        s->arena->release(r->rows_off, r->row_bytes);
        s->arena->release(r->starts_off, r->in_bytes);
        finish(s, r, st, msg);
      }
      w.reqs.clear();
      w.busy = false;
      progress = true;
    }
    if (progress) s->cv_done.notify_all();
    // 2. admit in arrival order within each size class while memory and the
    //    job table allow: small queries first, unless the oldest large query
    //    has waited kLargeAging; then it goes first, and while it waits for
    //    memory no small query is admitted (so large queries are not starved)
    const bool large_first =
        !s->pending[1].empty() && Clock::now() - s->pending[1].front()->t_submit > kLargeAging;
    for (int pass = 0; pass < 2; ++pass) {
      const int c = large_first ? 1 - pass : pass;
      bool blocked = false;
      while (!s->pending[c].empty() && (int)s->admitted[c].size() < s->cfg.max_jobs_per_wave) {
        Request* r = s->pending[c].front();
        size_t roff = s->rows_cursor, soff = 0;
        if (!s->arena->alloc_at(roff, r->row_bytes) && !s->arena->alloc(r->row_bytes, &roff)) {
          blocked = true;  // the head waits for memory
          break;
        }
        if (!s->arena->alloc_top(r->in_bytes, &soff)) {
          s->arena->release(roff, r->row_bytes);
          blocked = true;
          break;
        }
        r->rows_off = roff;
        r->starts_off = soff;
        s->rows_cursor = roff + r->row_bytes;
        r->state = REQ_ADMITTED;
        s->admitted[c].push_back(r);
        s->pending[c].pop_front();
        s->peak_arena = std::max(s->peak_arena, s->arena->used());
        progress = true;
      }
      if (large_first && c == 1 && blocked) break;
    }
    // 3. launch each class's admitted queries on a free stream, small ones
    //    first; large waves leave kSmallSlots of the streams to small ones
    int large_busy = 0;
    for (const Wave& w : s->waves) large_busy += (w.busy && w.cls == 1) ? 1 : 0;
    const int small_slots = s->cfg.max_waves > 1 ? std::max(1, s->cfg.max_waves / 8) : 0;
    for (int c = 0; c < 2; ++c) {
      if (s->admitted[c].empty()) continue;
      if (c == 1 && large_busy >= s->cfg.max_waves - small_slots) continue;
      for (Wave& w : s->waves) {
        if (w.busy) continue;
        launch_wave(s, w, c, lk);
        if (w.busy) ++inflight;
        progress = true;
        break;
      }
    }
    s->peak_inflight = std::max(s->peak_inflight, inflight);
    const bool idle = s->pending[0].empty() && s->pending[1].empty() && s->admitted[0].empty() &&
                      s->admitted[1].empty() && inflight == 0;
    if (s->stop && idle) break;
    if (!progress) {
      if (idle) s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
      else s->cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

}  // namespace

using namespace fw;

extern "C" void fw_server_config_default(fw_server_config* c) {
  if (!c) return;
  c->mem_budget = (size_t)1 << 30;
  c->max_waves = 4;
  c->max_jobs_per_wave = 64;
  c->large_query_steps = 0;
}

extern "C" fw_status fw_server_create(const fw_graph* g, const fw_server_config* cfg, fw_server** out) {
  if (!out) return set_error(FW_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!g) return set_error(FW_ERR_ARG, "graph is NULL");
  fw_server_config c;
  if (cfg) c = *cfg;
  else fw_server_config_default(&c);
  if (c.mem_budget < 4096 || c.max_waves < 1 || c.max_waves > 64 || c.max_jobs_per_wave < 1 ||
      c.max_jobs_per_wave > kMaxJobs || c.large_query_steps < 0)
    return set_error(FW_ERR_ARG, "bad server configuration");
  c.mem_budget &= ~(size_t)255;  // whole 256-byte units: every arena offset stays 4-byte aligned
  cudaError_t e = prime_walk_occupancy();
  if (e != cudaSuccess) return cuda_error(e, "occupancy query");
  fw_server* s = new (std::nothrow) fw_server();
  if (!s) return set_error(FW_ERR_OOM, "host allocation");
  s->g = g;
  s->cfg = c;
  auto fail = [&](cudaError_t err, const char* what) {
    for (Wave& w : s->waves) destroy_wave(w);
    cudaFree(s->arena_mem);
    cudaFreeHost(s->hops_host);
    delete s;
    return cuda_error(err, what);
  };
  e = cudaMalloc(&s->arena_mem, c.mem_budget);
  if (e != cudaSuccess) return fail(e, "cudaMalloc(server arena)");
  e = cudaMallocHost(&s->hops_host, sizeof(unsigned long long) * (size_t)c.max_waves);
  if (e != cudaSuccess) return fail(e, "cudaMallocHost(hop counts)");
  unsigned long long* q = nullptr;
  e = cudaMalloc(&q, 256 * (size_t)c.max_waves);
  if (e != cudaSuccess) return fail(e, "cudaMalloc(wave counters)");
  s->waves.resize(c.max_waves);
  for (int i = 0; i < c.max_waves; ++i) {
    Wave& w = s->waves[i];
    w.qctr = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(q) + 256 * (size_t)i);
    w.hops_host = s->hops_host + i;
    e = cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming);
    for (int k = 0; k < kAlgos - 1 && e == cudaSuccess; ++k)
      e = cudaStreamCreateWithFlags(&w.side[k], cudaStreamNonBlocking);
    for (int k = 0; k < kAlgos && e == cudaSuccess; ++k)
      e = cudaEventCreateWithFlags(&w.fork[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaFree(q);
      return fail(e, "stream / event creation");
    }
  }
  s->arena = new fw::Arena(c.mem_budget);
  s->worker = std::thread(worker_main, s);
  *out = s;
  return FW_OK;
}

// Is p in page-locked (or registered) host memory, so that copies to and
// from it run asynchronously?
static bool host_pinned(const void* p) {
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// A validated request for one query (no lock taken); nullptr and the
// error status on bad arguments.
static Request* new_request(fw_server* s, const int32_t* starts, int32_t num_walkers, int32_t len, int32_t algo,
                            const fw_params* params, uint64_t seed, int32_t* out, fw_status* st) {
  *st = FW_OK;
  if (num_walkers < 0 || len < 0 || (num_walkers > 0 && (!starts || !out))) {
    *st = set_error(FW_ERR_ARG, "bad sizes or NULL buffers");
    return nullptr;
  }
  Job J;
  *st = make_job(s->g, algo, params, seed, &J);  // validate parameters now
  if (*st != FW_OK) return nullptr;
  for (int32_t i = 0; i < num_walkers; ++i)
    if (starts[i] < 0 || starts[i] >= s->g->n) {
      *st = set_error(FW_ERR_ARG, "start " + std::to_string(i) + " outside [0, n)");
      return nullptr;
    }
  // staged starts and rows must fit the budget; each term is bounded before
  // it is added or multiplied, so nothing wraps
  const size_t in_bytes = sizeof(int32_t) * (size_t)num_walkers;  // < 2^34
  const size_t row_bytes = sizeof(int32_t) * ((size_t)len + 1);    // < 2^34
  const size_t budget = s->cfg.mem_budget;
  if (in_bytes > budget || (num_walkers > 0 && row_bytes > (budget - in_bytes) / (size_t)num_walkers)) {
    *st = set_error(FW_ERR_OOM, "query needs more device memory than the server's budget");
    return nullptr;
  }
  Request* r = new (std::nothrow) Request();
  if (!r) {
    *st = set_error(FW_ERR_OOM, "host allocation");
    return nullptr;
  }
  r->starts = starts;
  r->out = out;
  r->num_walkers = num_walkers;
  r->len = len;
  r->algo = algo;
  if (params) r->params = *params;
  else fw_params_default(&r->params);
  r->seed = seed;
  // size class: large queries (W x L >= large_query_steps; 0: none) get waves of their own
  r->cls = (s->cfg.large_query_steps > 0 &&
            (long long)num_walkers * (long long)len >= s->cfg.large_query_steps) ? 1 : 0;
  r->in_bytes = in_bytes;
  r->row_bytes = row_bytes * (size_t)num_walkers;
  r->pinned_in = host_pinned(starts);
  r->pinned_out = host_pinned(out);
  return r;
}

// Queue validated requests under one lock; tickets[i] receives request i's.
static fw_status enqueue(fw_server* s, Request* const* rs, int32_t count, uint64_t* tickets) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      for (int32_t i = 0; i < count; ++i) delete rs[i];
      return set_error(FW_ERR_BUSY, "server is shutting down");
    }
    const auto now = Clock::now();
    for (int32_t i = 0; i < count; ++i) {
      Request* r = rs[i];
      r->t_submit = now;
      r->id = s->next_id++;
      if (r->num_walkers == 0) {
        finish(s, r, FW_OK, "");
      } else {
        s->pending[r->cls].push_back(r);
      }
      s->reqs[r->id] = r;
      tickets[i] = r->id;
    }
  }
  s->cv_work.notify_one();
  return FW_OK;
}

extern "C" fw_status fw_server_submit(fw_server* s, const int32_t* starts, int32_t num_walkers, int32_t len,
                                      int32_t algo, const fw_params* params, uint64_t seed, int32_t* out,
                                      uint64_t* ticket) {
  if (!s || !ticket) return set_error(FW_ERR_ARG, "NULL argument");
  fw_status st;
  Request* r = new_request(s, starts, num_walkers, len, algo, params, seed, out, &st);
  if (!r) return st;
  return enqueue(s, &r, 1, ticket);
}

extern "C" fw_status fw_server_submit_many(fw_server* s, const fw_job* queries, int32_t count, uint64_t* tickets,
                                           int32_t* submitted) {
  if (!s || count < 0 || (count > 0 && (!queries || !tickets))) return set_error(FW_ERR_ARG, "bad arguments");
  if (submitted) *submitted = 0;
  std::vector<Request*> rs;
  rs.reserve((size_t)count);
  fw_status first_error = FW_OK;
  for (int32_t i = 0; i < count; ++i) {
    const fw_job& q = queries[i];
    fw_status st;
    Request* r = new_request(s, q.starts, q.num_walkers, q.len, q.algo, &q.params, q.seed, q.out, &st);
    if (!r) {
      first_error = set_error(st, "query " + std::to_string(i) + ": " + fw_last_error());
      break;
    }
    rs.push_back(r);
  }
  if (!rs.empty()) {
    const fw_status st = enqueue(s, rs.data(), (int32_t)rs.size(), tickets);
    if (st != FW_OK) return st;
    if (submitted) *submitted = (int32_t)rs.size();
  }
  return first_error;
}

static fw_status collect(fw_server* s, std::unordered_map<uint64_t, Request*>::iterator it, double* latency_ms) {
  Request* r = it->second;
  const fw_status st = r->status;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  std::string err = r->error;
  s->reqs.erase(it);
  delete r;
  return st == FW_OK ? FW_OK : set_error(st, err);
}

extern "C" fw_status fw_server_poll(fw_server* s, uint64_t ticket, int32_t* done, double* latency_ms) {
  if (!s || !done) return set_error(FW_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(FW_ERR_ARG, "unknown ticket");
  const int st = it->second->state;
  *done = (st == REQ_DONE || st == REQ_FAILED) ? 1 : 0;
  if (!*done) return FW_OK;
  return collect(s, it, latency_ms);
}

extern "C" fw_status fw_server_poll_many(fw_server* s, const uint64_t* tickets, int32_t count, int32_t* done,
                                         double* latency_ms, int32_t* status) {
  if (!s || count < 0 || (count > 0 && (!tickets || !done))) return set_error(FW_ERR_ARG, "bad arguments");
  std::lock_guard<std::mutex> lk(s->mu);
  for (int32_t i = 0; i < count; ++i) {
    auto it = s->reqs.find(tickets[i]);
    if (it == s->reqs.end()) {
      done[i] = 1;
      if (status) status[i] = FW_ERR_ARG;
      if (latency_ms) latency_ms[i] = 0.0;
      continue;
    }
    Request* r = it->second;
    done[i] = (r->state == REQ_DONE || r->state == REQ_FAILED) ? 1 : 0;
    if (!done[i]) continue;
    if (latency_ms) latency_ms[i] = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    if (status) status[i] = r->status;
    s->reqs.erase(it);
    delete r;
  }
  return FW_OK;
}

extern "C" fw_status fw_server_wait(fw_server* s, uint64_t ticket, double timeout_s, double* latency_ms) {
  if (!s) return set_error(FW_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(FW_ERR_ARG, "unknown ticket");
  Request* r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
  while (r->state != REQ_DONE && r->state != REQ_FAILED) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
        r->state != REQ_DONE && r->state != REQ_FAILED)
      return set_error(FW_ERR_TIMEOUT, "query not finished within the timeout");
  }
  return collect(s, s->reqs.find(ticket), latency_ms);
}

extern "C" fw_status fw_server_stats(fw_server* s, fw_server_stats_t* out) {
  if (!s || !out) return set_error(FW_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->completed = s->completed;
  out->failed = s->failed;
  out->pending = s->pending[0].size() + s->pending[1].size() + s->admitted[0].size() + s->admitted[1].size();
  out->waves = s->waves_launched;
  out->queries_per_wave = s->waves_launched ? (double)s->queries_in_waves / (double)s->waves_launched : 0.0;
  out->peak_device_bytes = s->peak_arena;
  out->peak_inflight_waves = s->peak_inflight;
  out->walker_steps = s->walker_steps;
  out->enqueue_ms_per_wave = s->waves_launched ? s->enqueue_ms / (double)s->waves_launched : 0.0;
  out->copies = s->copies;
  auto pct = [](std::vector<double>& l, double p) {
    return l[std::min(l.size() - 1, (size_t)(p * (double)(l.size() - 1) + 0.5))];
  };
  std::vector<double> l = s->latencies_ms;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    out->p50_ms = pct(l, 0.50);
    out->p99_ms = pct(l, 0.99);
    out->max_ms = l.back();
    double sum = 0;
    for (double x : l) sum += x;
    out->mean_ms = sum / (double)l.size();
    std::vector<double> qw = s->queue_ms, ww = s->wave_ms;
    std::sort(qw.begin(), qw.end());
    std::sort(ww.begin(), ww.end());
    out->queue_p50_ms = pct(qw, 0.50);
    out->queue_p99_ms = pct(qw, 0.99);
    out->wave_p50_ms = pct(ww, 0.50);
    out->wave_p99_ms = pct(ww, 0.99);
  }
  return FW_OK;
}

extern "C" fw_status fw_server_destroy(fw_server* s) {
  if (!s) return set_error(FW_ERR_ARG, "server is NULL");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();  // drains every submitted query
  for (auto& kv : s->reqs) delete kv.second;
  unsigned long long* q = s->waves.empty() ? nullptr : s->waves[0].qctr;
  for (Wave& w : s->waves) {
    destroy_wave(w);
  }
  cudaFree(q);
  cudaFree(s->arena_mem);
  cudaFreeHost(s->hops_host);
  if (s->mirror) cudaFreeHost(s->mirror);
  delete s->arena;
  delete s;
  return FW_OK;
}
