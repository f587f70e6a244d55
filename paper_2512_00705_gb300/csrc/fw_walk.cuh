// fw_walk.cuh -- the walk kernel: its loop, the kernel template and its
// launcher, instantiated for single jobs (fw_kernels.cu) and for tables of
// up to 64 jobs of one algorithm (fw_walk_mixed.cu).
//
// One warp runs the loop over one walker queue [Sec. 5.3]:
//   * query fetch   lanes without a walker take the next global walker
//                   indices with one warp-aggregated atomicAdd on the queue
//                   counter; a table of jobs is one concatenated index space
//                   (job j owns [gbase_j, gbase_j + W_j)).
//   * plan          [Sec. 3.3, Sec. 4.1]: per walker-step the bound B and the
//                   sum estimate give the eRJS / eRVS choice (or a forced mode).
//   * eRJS          [Sec. 3.3, Sec. 5.2]: one walker per lane; a fixed number
//                   of trials per round, then the warp checks by ballot which
//                   lanes need a reservoir step (chosen eRVS, or trial cap hit).
//   * eRVS / exact  [Sec. 3.2, Sec. 5.2]: steps of degree <= a small threshold
//                   run on their own lane; larger ones are handed to the whole
//                   warp one at a time (shuffle of the walker's state), and
//                   the result goes back to the owning lane; hub rows
//                   (d >= kHubMinDeg) are cut into chunks that every warp of
//                   the block scans (CTA-level parallel jumps, see hub steps).
//   * update        [Sec. 4.2, update()]: prev <- cur, cur <- next, row write.
// All loops are bounded (trial cap, degree, walk length, hub wait limit); no
// warp waits on another.
#pragma once

#include "fw_internal.h"

namespace fw {

constexpr int kBlock = 256;
constexpr int kMinBlocks = 4;  // 4 x 256 threads per SM (64 registers; 3, 5 and 6 blocks measured slower)
constexpr int kThreadExactMaxDeg = 16; // exact steps with d <= this run on one lane

// Row writes are staged per lane in shared memory, one aligned group of
// kStageSlots entries at a time, and written out when the group (or the
// row) is complete: scattered 4-byte stores would each cost a DRAM write.
// Slot s of lane t lives at obuf[s * kBlock + t] (no bank conflicts).
constexpr int kStageSlots = 8;  // 32-byte groups
static_assert(kStageSlots % 4 == 0 && (kStageSlots & (kStageSlots - 1)) == 0, "whole int4s, power of two");
struct RowStage {
  int32_t* row;   // current row (nullptr: none)
  int32_t first;  // first valid slot of the staged group
};

__device__ __forceinline__ int32_t stage_slot(const int32_t* a) {
  return (int32_t)((reinterpret_cast<uintptr_t>(a) >> 2) & (uintptr_t)(kStageSlots - 1));
}

// write the staged slots [first, last] of the group holding `a` (a = address of slot `last`)
__device__ __forceinline__ void stage_flush(const int32_t* obuf, int tid, int32_t* a, int32_t first, int32_t last) {
  int32_t* base = a - last;
  if (first == 0 && last == kStageSlots - 1) {
#pragma unroll
    for (int q = 0; q < kStageSlots / 4; ++q)
      reinterpret_cast<int4*>(base)[q] = make_int4(obuf[(4 * q) * kBlock + tid], obuf[(4 * q + 1) * kBlock + tid],
                                                   obuf[(4 * q + 2) * kBlock + tid], obuf[(4 * q + 3) * kBlock + tid]);
  } else {
    for (int32_t k = first; k <= last; ++k) base[k] = obuf[k * kBlock + tid];
  }
}

// stage row[p] = val; `final` marks the last entry the lane will write in this row
__device__ __forceinline__ void stage_put(int32_t* obuf, int tid, RowStage& rs, int32_t p, int32_t val, bool final) {
  int32_t* a = rs.row + p;
  const int32_t slot = stage_slot(a);
  obuf[slot * kBlock + tid] = val;
  if (slot == kStageSlots - 1 || final) {
    stage_flush(obuf, tid, a, rs.first, slot);
    rs.first = 0;
  }
}

// row[from, to) = -1 after a dead end: finish the staged group, then whole groups, then the tail
__device__ __forceinline__ void stage_fill_minus_one(int32_t* obuf, int tid, RowStage& rs, int32_t from, int32_t to) {
  int32_t p = from;
  while (p < to && (p == from || stage_slot(rs.row + p) != 0)) {
    stage_put(obuf, tid, rs, p, -1, p + 1 == to);
    ++p;
  }
  for (; p + kStageSlots <= to; p += kStageSlots) {
    int4* q = reinterpret_cast<int4*>(rs.row + p);
#pragma unroll
    for (int k = 0; k < kStageSlots / 4; ++k) q[k] = make_int4(-1, -1, -1, -1);
  }
  for (; p < to; ++p) rs.row[p] = -1;
}

template <int NJ>
struct JobTableN {
  Job jobs[NJ];
};

// ---------------------------------------------------------------- hub steps
// An eRVS step of degree >= kHubMinDeg is shared by the warps of the block
// (the parallel jump process of Sec. 3.2 at CTA level).  The warp that owns
// the step keys the row's first kHubPhase1 positions (phase 1, the draws of
// the warp scan), and their maximum key K_g becomes the reference from which
// every other position is reached by jumps.  Those positions are cut into
// chunks of kHubChunk; inside a chunk, lane l scans lo + l, lo + l + 32, ...
// and starts with its own jump threshold, drawn from counter (walker, hop,
// 5, lo + l); crossings draw as in the warp scan.  A chunk's keys therefore
// depend on its positions and K_g alone, so the result is the same whether
// the owning warp scans every chunk itself or the block shares them, and
// whatever warp scans which chunk when.
//
// Sharing: the owning warp posts the step to a free slot of the block's task
// table in shared memory (else it scans the chunks alone).  A warp that
// looks (see the walk loop: warps with a waiting lane, and warps whose queue
// ran dry) claims the next chunk of an open task, scans it and enters the
// chunk's best (key, position) by one 64-bit atomicMax on the pair packed in
// key order (equal keys: the larger position, as in warp_argmax), then
// counts the chunk done.  The owning lane takes the result once every chunk
// is done; its warp keeps walking its other lanes and claims chunks itself,
// so no warp waits on another and a task completes even when no other warp
// helps.  Busy warps do not look: with every lane walking, sharing would
// move work between warps without shortening the launch, and the check
// itself costs time on every iteration.
constexpr int32_t kHubMinDeg = 32768;            // eRVS steps of at least this degree are shared
constexpr int32_t kHubPhase1Keys = 32;           // phase-1 keys per lane
constexpr int32_t kHubPhase1 = 32 * kHubPhase1Keys;  // positions keyed in phase 1
constexpr int32_t kHubChunk = 8192;              // positions per chunk (256 per lane)
constexpr int kHubTasks = 4;                     // open hub steps per block
constexpr int32_t kHubMaxChunks = 1 << 19;       // the 20-bit chunk counter never wraps
constexpr uint32_t kHubWaitLimit = 1u << 24;     // loop iterations a lane waits for its step at most
// slot word: state (2 bits) | generation (10 bits) | next unclaimed chunk (20 bits)
constexpr uint32_t kHubFree = 0u, kHubReserved = 1u, kHubOpen = 2u;
constexpr uint32_t kHubGenMask = 0x3ff00000u, kHubNextMask = 0x000fffffu;

struct HubTask {
  uint32_t word;
  int32_t nchunks;
  int32_t done;              // chunks scanned
  int32_t job;
  unsigned long long best;   // packed (ordered key, position) of the best key so far; 0: none
  float ref;                 // K_g: the phase-1 maximum key
  int32_t grp;               // grouped metapath: c.s, c.d are the label segment
  StepCtx c;
};

struct HubBlock {  // shared memory, per block
  HubTask task[kHubTasks];
  int32_t open;    // tasks with chunks left to claim
  int32_t live;    // warps of the block still walking (the others linger to help)
};
constexpr uint32_t kLingerLimit = 1u << 22;  // idle checks of a lingering warp at most

// float key -> unsigned in the same order (no NaN keys arise)
__device__ __forceinline__ uint32_t key_order(float k) {
  const uint32_t u = __float_as_uint(k);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ unsigned long long key_pack(float k, int32_t pos) {
  return (k == -CUDART_INF_F) ? 0ull : (((unsigned long long)key_order(k) << 32) | (uint32_t)pos);
}

__device__ __forceinline__ int32_t hub_chunks(int32_t d) { return (d - kHubPhase1 + kHubChunk - 1) / kHubChunk; }

// Phase 1 of a hub step (the whole warp): keys of positions lane + 32 j,
// j < kHubPhase1Keys, four per Philox block as in rvs_scan.  A chunk lane crosses K_g about ln(1 + n / kHubPhase1)
// times over its n positions, every crossing a divergent key draw, so the
// reference is taken over more positions than a warp scan's phase 1.
// Leaves the lane's best in bestK / best.
template <bool COUNT, int ALG, bool GRP>
__device__ __forceinline__ void hub_phase1(const DevGraph& g, const Job& J, const StepCtx& c, int lane,
                                           LaneCounters& lc, float& bestK, int32_t& best) {
  uint32_t probes = 0;
  bestK = -CUDART_INF_F;
  best = -1;
  int32_t keys = 0;
  uint4 x4 = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll 1
  for (int32_t j = 0; j < kHubPhase1Keys; ++j) {
    const int32_t k = lane + 32 * j;
    const float wt = scan_weight<ALG, GRP>(g, J, c, c.s + k, probes);
    if ((j & 3) == 0) x4 = philox(make_uint4(c.wid, (uint32_t)c.step, 6u, (uint32_t)k), J.key0, J.key1);
    const uint32_t r = (j & 3) == 0 ? x4.x : ((j & 3) == 1 ? x4.y : ((j & 3) == 2 ? x4.z : x4.w));
    if (wt > 0.0f) {
      const float K = logf(u01_open(r)) / wt;
      ++keys;
      if (K >= bestK) {
        bestK = K;
        best = k;
      }
    }
  }
  if (COUNT) rvs_count<ALG, GRP>(J, kHubPhase1Keys, keys, probes, lc);
}

// Chunk [lo, hi) of a hub step (the whole warp): jumps from K_g = ref with
// per-lane thresholds from counter stream 5 (without jumps: every key, as in
// the warp scan).  Leaves the lane's best in bestK / best.
template <bool COUNT, int ALG, bool GRP>
__device__ __forceinline__ void hub_chunk_scan(const DevGraph& g, const Job& J, const StepCtx& c, int32_t lo,
                                               int32_t hi, float ref, bool jump, int lane, LaneCounters& lc,
                                               float& bestK, int32_t& best) {
  uint32_t probes = 0;
  int32_t scanned = 0, keys = 0;
  bestK = -CUDART_INF_F;
  best = -1;
  float r = ref, rem = 0.0f;  // K_g = -inf: the first positive item crosses
  if (jump && r != -CUDART_INF_F) {
    const uint4 x0 = philox(make_uint4(c.wid, (uint32_t)c.step, 5u, (uint32_t)(lo + lane)), J.key0, J.key1);
    rem = (r < 0.0f) ? logf(u01_open(x0.x)) / r : CUDART_INF_F;
  }
  for (int32_t k = lo + lane; k < hi; k += 32) {
    const float wt = scan_weight<ALG, GRP>(g, J, c, c.s + k, probes);
    ++scanned;
    if (!(wt > 0.0f)) continue;
    if (!jump) {
      const uint4 x = philox(make_uint4(c.wid, (uint32_t)c.step, 2u, (uint32_t)k), J.key0, J.key1);
      const float K = logf(u01_open(x.x)) / wt;
      ++keys;
      if (K >= bestK) {
        bestK = K;
        best = k;
      }
    } else {
      rem -= wt;
      if (rem <= 0.0f) {
        const uint4 x = philox(make_uint4(c.wid, (uint32_t)c.step, 2u, (uint32_t)k), J.key0, J.key1);
        // key conditioned on beating r: u' ~ U(exp(r*wt), 1), K = ln(u') / wt
        const float K = log1pf(expm1f(r * wt) * u01_open(x.y)) / wt;
        ++keys;
        bestK = K;
        best = k;
        r = K;
        rem = (r < 0.0f) ? logf(u01_open(x.z)) / r : CUDART_INF_F;
      }
    }
  }
  if (COUNT) rvs_count<ALG, GRP>(J, scanned, keys, probes, lc);
}

// Post a hub step (one lane); -1: every slot taken.
__device__ __forceinline__ int hub_post(HubBlock* hb, const StepCtx& c, int32_t job, bool grp, float ref,
                                        unsigned long long best) {
  for (int i = 0; i < kHubTasks; ++i) {
    HubTask& t = hb->task[i];
    const uint32_t w = *reinterpret_cast<volatile uint32_t*>(&t.word);
    if ((w >> 30) != kHubFree) continue;
    if (atomicCAS(&t.word, w, (kHubReserved << 30) | (w & kHubGenMask)) != w) continue;
    t.c = c;
    t.job = job;
    t.grp = grp ? 1 : 0;
    t.ref = ref;
    t.nchunks = hub_chunks(c.d);
    t.done = 0;
    t.best = best;
    __threadfence_block();  // the fields before the slot opens
    const uint32_t gen = ((w >> 20) + 1u) & 0x3ffu;
    atomicExch(&t.word, (kHubOpen << 30) | (gen << 20));
    atomicAdd(&hb->open, 1);
    return i;
  }
  return -1;
}

// Claim the next unclaimed chunk of the open task in `slot` (one lane);
// false: none left.  The compare-and-swap against the word read fails if
// the slot was claimed, closed or reopened meanwhile, so a successful claim
// also vouches for the chunk count read before it.  Taking a task's last
// chunk closes it for the lingering warps' check.
__device__ __forceinline__ bool hub_claim_slot(HubBlock* hb, int slot, int32_t& chunk) {
  HubTask& t = hb->task[slot];
  uint32_t w = *reinterpret_cast<volatile uint32_t*>(&t.word);
  for (int tries = 0; tries < 64 && (w >> 30) == kHubOpen; ++tries) {
    const int32_t nc = *reinterpret_cast<volatile int32_t*>(&t.nchunks);
    const int32_t nx = (int32_t)(w & kHubNextMask);
    if (nx >= nc) return false;
    const uint32_t old = atomicCAS(&t.word, w, w + 1u);
    if (old == w) {
      if (nx + 1 == nc) atomicSub(&hb->open, 1);
      chunk = nx;
      return true;
    }
    w = old;
  }
  return false;
}

// Scan claimed chunk `chunk` of the task in `slot` (the whole warp,
// converged), enter its best and count it done.
template <bool COUNT, int ALG>
__device__ __forceinline__ void hub_scan_claimed(const DevGraph& g, const Job* sj, HubBlock* hb, int slot,
                                                 int32_t chunk, LaneCounters& lc) {
  const int lane = threadIdx.x & 31;
  HubTask& t = hb->task[slot];  // fixed until this chunk is counted done
  StepCtx hc;
  const volatile int32_t* src = reinterpret_cast<const volatile int32_t*>(&t.c);
  int32_t* dst = reinterpret_cast<int32_t*>(&hc);
#pragma unroll
  for (int q = 0; q < (int)(sizeof(StepCtx) / 4); ++q) dst[q] = src[q];
  const Job& J = sj[*reinterpret_cast<volatile int32_t*>(&t.job)];
  const float ref = *reinterpret_cast<volatile float*>(&t.ref);
  const int32_t lo = kHubPhase1 + chunk * kHubChunk, hi = min(hc.d, lo + kHubChunk);
  const bool jump = !(J.flags & FW_FLAG_RVS_NOJUMP);
  float bk;
  int32_t bi;
  if (ALG == ALGO_METAPATH && *reinterpret_cast<volatile int32_t*>(&t.grp) != 0)
    hub_chunk_scan<COUNT, ALG, true>(g, J, hc, lo, hi, ref, jump, lane, lc, bk, bi);
  else
    hub_chunk_scan<COUNT, ALG, false>(g, J, hc, lo, hi, ref, jump, lane, lc, bk, bi);
  warp_argmax(bk, bi);
  if (lane == 0) {
    if (bk != -CUDART_INF_F) atomicMax(&t.best, key_pack(bk, bi));
    __threadfence_block();  // the result before the chunk counts as done
    atomicAdd(&t.done, 1);
  }
  __syncwarp();
}

// A lingering warp (converged, no walker left): claim and scan one chunk of
// any open task of the block.  Returns whether a chunk was scanned.
template <bool COUNT, int ALG>
__device__ __forceinline__ bool hub_help(const DevGraph& g, const Job* sj, HubBlock* hb, LaneCounters& lc) {
  const int lane = threadIdx.x & 31;
  if (__shfl_sync(kFull, *reinterpret_cast<volatile int32_t*>(&hb->open), 0) <= 0) return false;
  int32_t chunk = 0;
  int slot = -1;
  if (lane == 0) {
    for (int i = 0; i < kHubTasks && slot < 0; ++i)
      if (hub_claim_slot(hb, i, chunk)) slot = i;
  }
  slot = __shfl_sync(kFull, slot, 0);
  if (slot < 0) return false;
  chunk = __shfl_sync(kFull, chunk, 0);
  __syncwarp();
  hub_scan_claimed<COUNT, ALG>(g, sj, hb, slot, chunk, lc);
  return true;
}

// A hub step (the whole warp, converged; cw, JW: the step and its job, jb
// its index, grp: grouped metapath).  Phase 1; then, when a warp of the
// block lingers to help, the step is posted and this warp claims and scans
// chunks alongside the helpers until none is left, waits for the chunks the
// helpers hold (they wait on nothing) and frees the slot; otherwise it scans
// every chunk alone (always, without SHARE).  Returns the position (-1: all
// weights zero, or the join wait ran out, which also sets DEVERR_HUB).
template <bool COUNT, int ALG, bool SHARE>
__device__ __forceinline__ int32_t hub_step(const DevGraph& g, const Job* sj, const Job& JW, const StepCtx& cw,
                                            int32_t jb, bool grp, HubBlock* hb, unsigned* err, LaneCounters& lc) {
  const int lane = threadIdx.x & 31;
  float bk;
  int32_t bi;
  if (ALG == ALGO_METAPATH && grp) hub_phase1<COUNT, ALG, true>(g, JW, cw, lane, lc, bk, bi);
  else hub_phase1<COUNT, ALG, false>(g, JW, cw, lane, lc, bk, bi);
  const float ref = warp_max(bk);
  warp_argmax(bk, bi);
  int slot = -1;
  if (SHARE && lane == 0 && *reinterpret_cast<volatile int32_t*>(&hb->live) < (int32_t)(blockDim.x >> 5))
    slot = hub_post(hb, cw, jb, grp, ref, key_pack(bk, bi));
  if (SHARE) slot = __shfl_sync(kFull, slot, 0);
  if (SHARE && slot >= 0) {
    HubTask& t = hb->task[slot];
    while (true) {
      int32_t chunk = 0;
      bool got = false;
      if (lane == 0) got = hub_claim_slot(hb, slot, chunk);
      if (!__shfl_sync(kFull, (int)got, 0)) break;
      chunk = __shfl_sync(kFull, chunk, 0);
      __syncwarp();
      hub_scan_claimed<COUNT, ALG>(g, sj, hb, slot, chunk, lc);
    }
    // join: the helpers finish the chunks they claimed
    bool ok = false;
    if (lane == 0) {
      const int32_t nc = t.nchunks;
      for (uint32_t it = 0; it < kHubWaitLimit; ++it) {
        if (*reinterpret_cast<volatile int32_t*>(&t.done) >= nc) {
          ok = true;
          break;
        }
        __nanosleep(64);
      }
    }
    ok = __shfl_sync(kFull, (int)ok, 0) != 0;
    if (!ok) {
      if (lane == 0) atomicOr(err, DEVERR_HUB);  // the slot stays taken
      return -1;
    }
    __threadfence_block();
    const unsigned long long r = *reinterpret_cast<volatile unsigned long long*>(&t.best);
    __syncwarp();
    if (lane == 0) {
      const uint32_t wd = *reinterpret_cast<volatile uint32_t*>(&t.word);
      atomicExch(&t.word, wd & kHubGenMask);  // free, keeping the generation
    }
    return r ? (int32_t)(uint32_t)r : -1;
  }
  const bool jump = !(JW.flags & FW_FLAG_RVS_NOJUMP);
  const int32_t nch = hub_chunks(cw.d);
  for (int32_t q = 0; q < nch; ++q) {
    const int32_t lo = kHubPhase1 + q * kHubChunk, hi = min(cw.d, lo + kHubChunk);
    float ck;
    int32_t ci;
    if (ALG == ALGO_METAPATH && grp) hub_chunk_scan<COUNT, ALG, true>(g, JW, cw, lo, hi, ref, jump, lane, lc, ck, ci);
    else hub_chunk_scan<COUNT, ALG, false>(g, JW, cw, lo, hi, ref, jump, lane, lc, ck, ci);
    warp_argmax(ck, ci);
    if (ck > bk || (ck == bk && ci > bi)) {
      bk = ck;
      bi = ci;
    }
  }
  return (bk == -CUDART_INF_F) ? -1 : bi;
}

// The walk loop of one warp over one queue: take walkers, plan, sample and
// write rows until the queue is exhausted and the warp holds no walker.
// `sj` (shared memory) is the queue's job table: its jobs' walkers form the
// index space [0, total), job j owning [sj[j].gbase, sj[j].gbase + W_j).
// ALG fixes the algorithm of every job at compile time; SHARE: hub steps
// may be shared with the block's idle warps (see hub steps).
template <bool COUNT, int ALG, bool SHARE>
__device__ __forceinline__ void walk_loop(const DevGraph& g, const Job* sj, int njobs, long long total,
                                          unsigned long long* __restrict__ qctr, unsigned* __restrict__ err,
                                          int32_t* obuf, HubBlock* hb, LaneCounters& lc) {
  static_assert(ALG >= 0 && ALG < kAlgos, "the walk loop is compiled for one algorithm");
  const int lane = threadIdx.x & 31;
  const int tid = threadIdx.x;
  const unsigned lt_mask = (1u << lane) - 1u;
  RowStage rs;
  rs.row = nullptr;
  rs.first = 0;

  // walker state: c.v current node, c.vp previous node (-1: none), c.step hop,
  // c.s / c.d row of c.v, c.ps / c.pe row of c.vp
  StepCtx c;
  c.v = c.vp = c.s = c.d = c.ps = c.pe = c.step = 0;
  c.wid = 0;
  c.w1 = c.w2 = 1.0f;
  c.n0 = -1;
  c.n1 = 0;
  c.hsc = 0.0f;
  int32_t job = 0, widx = -1;
  int32_t plan = PLAN_NONE, trials = 0, pick = -2, node = -1;
  float B = 0.0f;
  // eRJS with the return edge split off: probability of the return component,
  // position of v' in N(v) (-1: unknown) and h(v, v')
  bool split = false;
  float beta = 0.0f, h_ret = 0.0f;
  // node2vec with 1/q < 1 and d(v') < d(v): two envelopes; beta2 = (E3 + E2) / E
  bool csplit = false;
  float beta2 = 0.0f;
  // metapath in the label-grouped view: c.ps / c.pe then hold the required
  // label's segment of the grouped arrays (metapath has no use for the row of v')
  bool grp = false;
  int32_t pos_ret = -1;
  // from the accepted trial: the next node's record, and h of the edge taken (-1: unknown)
  int4 nxt = make_int4(0, 0, 0, 0);
  int32_t nxt_n0 = 0, nxt_n1 = 0;
  bool nxt_ok = false;
  float h_in = -1.0f;
  bool exhausted = false;  // warp-uniform

  while (true) {
    // ------------------------------------------------------------ fetch
    const bool need = widx < 0;
    const unsigned nm = __ballot_sync(kFull, need);
    if (nm != 0u && !exhausted) {
      const int leader = __ffs(nm) - 1;
      const unsigned cntw = __popc(nm);
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(qctr, (unsigned long long)cntw);
      base = __shfl_sync(kFull, base, leader);
      if (base + cntw >= (unsigned long long)total) exhausted = true;
      if (need) {
        const long long gi = (long long)base + __popc(nm & lt_mask);
        if (gi < total) {
          int j = 0;
          while (j + 1 < njobs && sj[j + 1].gbase <= gi) ++j;
          const Job& J = sj[j];
          job = j;
          widx = (int32_t)(gi - J.gbase);
          if (J.kind == JOB_WALK) {
            const int32_t st = __ldg(J.starts + widx);
            rs.row = J.out + (long long)widx * (J.len + 1);
            rs.first = stage_slot(rs.row);
            if (st < 0 || st >= g.n) {
              atomicOr(err, DEVERR_START);
              stage_fill_minus_one(obuf, tid, rs, 0, J.len + 1);
              widx = -1;
            } else {
              stage_put(obuf, tid, rs, 0, st, J.len == 0);
              c.v = st;
              c.vp = -1;
              c.step = 0;
              if (J.len == 0) widx = -1;
            }
          } else {
            c.v = J.hv;
            c.vp = J.hprev;
            c.step = J.hstep;
            if (c.vp >= 0) {  // during walks the row of v' is carried along; here it is loaded
              const int4 pr = __ldg(g.nrec + 2ll * c.vp);
              c.s = pr.x;
              c.d = pr.y;
            }
          }
          plan = PLAN_NONE;
          pick = -2;
          nxt_ok = false;
          h_in = -1.0f;
        }
      }
    }
    if (!__any_sync(kFull, widx >= 0)) {
      if (exhausted) break;
      continue;
    }

    const Job& J = sj[job];
    // ------------------------------------------------------------ plan
    if (widx >= 0 && plan == PLAN_NONE) {
      c.ps = c.s;  // the row of v' is the previous step's row
      c.pe = c.s + c.d;
      c.wid = J.wids ? __ldg(J.wids + widx) : J.walker_base + (uint32_t)widx;
      // row start, degree, h_MAX, h_SUM and class counts of v: from the accepted trial's edge
      // record, or one load
      int4 nr;
      int32_t n0, n1;
      if (nxt_ok) {
        nr = nxt;
        n0 = nxt_n0;
        n1 = nxt_n1;
      } else {
        int4 nr2;
        ld_record(g.nrec + 2ll * c.v, nr, nr2);
        n0 = nr2.x;
        n1 = nr2.y;
        if (COUNT) lc.bytes += 32;
      }
      nxt_ok = false;
      c.s = nr.x;
      c.d = nr.y;
      if (g.h8) c.hsc = __ldg(g.h8scale + c.v);  // scale of the codes of v's row
      // weight classes in eRJS wherever the bound is a multiple of h_MAX[v]
      const bool cls = J.classes && !(FW_ALGO(J) == ALGO_METAPATH && J.label_stats);
      c.n0 = cls ? n0 : -1;
      c.n1 = n1;
      // eRJS envelope mass in units of the class-0 bound: (4 n0 + 2 n1 + n2) / 4
      const float dsl = cls ? __fmul_rn(0.25f, (float)(c.d + 3 * n0 + n1)) : (float)c.d;
      trials = 0;
      pick = -2;
      split = false;
      csplit = false;
      grp = false;
      beta = 0.0f;
      if (c.d == 0) {
        pick = -1;
        plan = PLAN_RJS;
      } else {
        int32_t m = J.mode;
        if (m == MODE_EXACT) {
          if (FW_ALGO(J) == ALGO_PAGERANK2 && c.vp >= 0) pagerank2_weights(J, c.d, c.pe - c.ps, c.w1, c.w2);
          plan = (c.d <= kThreadExactMaxDeg) ? PLAN_EXACT_T : PLAN_EXACT_W;
        } else {
          float hm, hs, S;
          if (J.weighted) {
            hm = __int_as_float(nr.z);
            hs = __int_as_float(nr.w);
          } else {
            hm = 1.0f;
            hs = (float)c.d;
          }
          int32_t choice;
          if (FW_ALGO(J) == ALGO_METAPATH && J.label_group) {
            // per-label record of v: exact bound and sum over the required label,
            // and where its entries sit in the label-grouped view; none -> dead end
            const uint8_t want = J.schema[c.step % J.schema_len];
            int4 lr = make_int4(0, 0, 0, 0), lr2 = make_int4(0, 0, 0, 0);
            if (want < kLabelStats) {
              ld_record(g.lrec + 2ll * ((long long)c.v * kLabelStats + want), lr, lr2);
              if (COUNT) lc.bytes += 32;
            }
            B = __int_as_float(lr.x);
            S = __int_as_float(lr.y);
            grp = true;
            c.ps = c.s + lr.z;
            c.pe = c.ps + lr.w;
            c.gcls = lr2;
            // expected eRJS trials follow the class envelope: bound B * slots / (16 len)
            const float beff = lr.w > 0 ? __fmul_rn(B, (float)class_slots(lr2, lr.w) / (16.0f * (float)lr.w)) : B;
            choice = (__fmul_rn(J.ratio, beff) < S) ? MODE_RJS : MODE_RVS;
            if (!(S > 0.0f)) pick = -1;
          } else if (FW_ALGO(J) == ALGO_METAPATH && J.label_stats) {
            // metapath with per-label statistics: exact bound and exact sum over
            // the edges whose label the step requires; none -> dead end now
            const uint8_t want = J.schema[c.step % J.schema_len];
            float2 ls = make_float2(0.0f, 0.0f);
            if (want < kLabelStats) {
              ls = __ldg(g.lstat + (long long)c.v * kLabelStats + want);
              if (COUNT) lc.bytes += 8;
            }
            B = ls.x;
            S = ls.y;
            choice = (__fmul_rn(J.ratio, B) < S) ? MODE_RJS : MODE_RVS;
            if (!(S > 0.0f)) pick = -1;
          } else {
            if (FW_ALGO(J) == ALGO_PAGERANK2 && c.vp >= 0) pagerank2_weights(J, c.d, c.pe - c.ps, c.w1, c.w2);
            choice = plan_choice<ALG>(J, hm, hs, c.vp >= 0, c.w1, c.w2, B, S);
            // with weight classes the expected trials scale with the envelope mass dsl * B
            const float frac = dsl / (float)c.d;
            if (cls) choice = (__fmul_rn(J.ratio, __fmul_rn(B, frac)) < S) ? MODE_RJS : MODE_RVS;
            if (FW_ALGO(J) == ALGO_PAGERANK2 && c.vp >= 0 && !(J.flags & FW_FLAG_PLAIN_RJS) &&
                c.pe - c.ps <= kPr2SplitMaxPrev && c.w1 > __fmul_rn(2.0f, c.w2)) {
              // common neighbours split off: eRJS then costs as a first-order walk with bound w2 h_MAX
              split = true;
              B = __fmul_rn(c.w2, hm);
              S = __fmul_rn(c.w2, hs);
              choice = (__fmul_rn(J.ratio, __fmul_rn(B, frac)) < S) ? MODE_RJS : MODE_RVS;
            }
          }
          if (m == MODE_AUTO) {
            m = choice;
          } else if (m == MODE_RANDOM) {  // coin from Philox counter (wid, hop, 4, 0)
            m = (philox(make_uint4(c.wid, (uint32_t)c.step, 4u, 0u), J.key0, J.key1).x >> 31) ? MODE_RJS : MODE_RVS;
          } else if (m == MODE_DEGREE) {
            m = (c.d < kDegreeRuleThreshold) ? MODE_RVS : MODE_RJS;
          }
          plan = (m == MODE_RJS) ? PLAN_RJS : (((grp ? c.pe - c.ps : c.d) <= J.lane_max) ? PLAN_RVS_T : PLAN_RVS_W);
          if (split) {  // second-order PageRank: S_C and the probability of the common-neighbour part
            split = plan == PLAN_RJS;
            if (split) {
              uint32_t pb = 0;
              h_ret = common_h_sum(g, J, c, pb);
              if (COUNT) {
                lc.probes += pb;
                lc.bytes += 32ull * pb + 4ull * (uint32_t)(c.pe - c.ps);
              }
              const float wc = __fmul_rn(__fsub_rn(c.w1, c.w2), h_ret);
              beta = wc / (wc + dsl * B);
            }
          } else if (FW_ALGO(J) == ALGO_NODE2VEC && plan == PLAN_RJS && c.vp >= 0 &&
                     (J.split_return || (J.split_common && (float)(c.pe - c.ps) < dsl))) {
            // the return edge alone sets max(w) = 1/p: propose it separately and
            // bound the other neighbours by max(1, 1/q) * h_MAX[v]; with 1/q < 1 and
            // a row of v' shorter than the envelope of N(v), two envelopes (see rjs_trials)
            split = true;
            csplit = J.split_common && (float)(c.pe - c.ps) < dsl;
            B = csplit ? hm : __fmul_rn(J.whi1, hm);
            pos_ret = -1;
            bool have = false;
            if (g.sym && h_in >= 0.0f && J.kind == JOB_WALK) {
              h_ret = h_in;  // symmetric weights: h(v, v') = h(v', v), the edge just taken
              have = true;
            } else {
              uint32_t pb = 0;
              pos_ret = row_find(g.col, c.s, c.s + c.d, c.vp, g.n, pb);
              if (COUNT) {
                lc.probes += pb;
                lc.bytes += 32ull * pb;
              }
              if (pos_ret >= 0) {
                h_ret = load_h(g, J, pos_ret, c.hsc);
                pos_ret -= c.s;
                have = true;
              }
            }
            if (csplit) {
              const float e3 = have ? __fmul_rn(J.inv_p, h_ret) : 0.0f;
              const float e2 = __fmul_rn(__fmul_rn(__fsub_rn(1.0f, J.inv_q), (float)(c.pe - c.ps)), hm);
              const float e1 = __fmul_rn(__fmul_rn(J.inv_q, dsl), hm);
              const float tot = __fadd_rn(__fadd_rn(e3, e2), e1);
              beta = e3 / tot;
              beta2 = __fadd_rn(e3, e2) / tot;
            } else if (have) {
              const float wret = __fmul_rn(J.inv_p, h_ret);
              beta = wret / (wret + dsl * B);
            }
          }
        }
      }
    }
    // ------------------------------------------------------------ eRJS trials
    if (widx >= 0 && plan == PLAN_RJS && pick == -2) {
      Accept acc;
      if (rjs_trials<COUNT, ALG>(g, J, c, B, split, beta, pos_ret, h_ret, trials, J.rjs_batch, acc, lc, csplit, beta2,
                                 grp)) {
        pick = acc.k;
        node = acc.node;
        h_in = acc.h;
        nxt = acc.rec;
        nxt_n0 = acc.rec_n0;
        nxt_n1 = acc.rec_n1;
        nxt_ok = acc.rec_ok;
        if (COUNT) lc.rjs_steps++;
      } else {
        trials += J.rjs_batch;
        // trial budget: the cap, or (default) as many trials as the eRVS scan
        // they stand in for would cost under the cost model, d / r, times the
        // budget scale
        const int32_t dd = grp ? c.pe - c.ps : c.d;  // entries the eRVS hand-off would scan
        const int32_t cap =
            J.fixed_cap ? J.rjs_cap : max(J.rjs_cap, (int32_t)fminf(ceilf(J.budget * (float)dd / J.ratio), 1.0e9f));
        if (trials >= cap) {
          plan = (dd <= J.lane_max) ? PLAN_RVS_T : PLAN_RVS_W;
          if (COUNT) lc.handoffs++;
        }
      }
    }
    // ------------------------------------------------------------ single-lane eRVS / exact
    if (widx >= 0 && pick == -2 && plan == PLAN_RVS_T) {
      if ((FW_ALGO(J) == ALGO_METAPATH) && grp) {
        StepCtx cg = c;
        cg.s = c.ps;
        cg.d = c.pe - c.ps;
        const int32_t j = rvs_pick<1, COUNT, ALG, true>(g, J, cg, 0, !(J.flags & FW_FLAG_RVS_NOJUMP), lc);
        pick = -1;
        if (j >= 0) {  // the grouped record gives the node, its position in the row and its node record
          int4 a, b;
          ld_record(g.gerec + 2ll * (cg.s + j), a, b);
          if (COUNT) lc.bytes += 32;
          pick = b.z;
          node = a.x;
          nxt = make_int4(a.z, a.w, b.x, b.y);
          nxt_n0 = nxt_n1 = 0;  // metapath plans without weight classes
          nxt_ok = true;
        }
      } else {
        pick = rvs_pick<1, COUNT, ALG>(g, J, c, 0, !(J.flags & FW_FLAG_RVS_NOJUMP), lc);
        if (pick >= 0) node = __ldg(g.col + c.s + pick);
      }
      h_in = -1.0f;
      if (COUNT) lc.rvs_steps++;
    }
    if (widx >= 0 && pick == -2 && plan == PLAN_EXACT_T) {
      const float u = u01(philox(make_uint4(c.wid, (uint32_t)c.step, 0u, 0u), J.key0, J.key1).x);
      pick = exact_pick<1, COUNT, ALG>(g, J, c, 0, u, lc);
      if (pick >= 0) node = __ldg(g.col + c.s + pick);
      h_in = -1.0f;
      if (COUNT) lc.exact_steps++;
    }
    // ------------------------------------------------------------ warp hand-off
    unsigned wm = __ballot_sync(kFull, widx >= 0 && pick == -2 && (plan == PLAN_RVS_W || plan == PLAN_EXACT_W));
    while (wm != 0u) {
      const int src = __ffs(wm) - 1;
      wm &= wm - 1u;
      StepCtx w;
      w.v = __shfl_sync(kFull, c.v, src);
      w.vp = __shfl_sync(kFull, c.vp, src);
      w.s = __shfl_sync(kFull, c.s, src);
      w.d = __shfl_sync(kFull, c.d, src);
      w.ps = __shfl_sync(kFull, c.ps, src);
      w.pe = __shfl_sync(kFull, c.pe, src);
      w.step = __shfl_sync(kFull, c.step, src);
      w.wid = __shfl_sync(kFull, c.wid, src);
      if (ALG == ALGO_PAGERANK2) {
        w.w1 = __shfl_sync(kFull, c.w1, src);
        w.w2 = __shfl_sync(kFull, c.w2, src);
      }
      w.hsc = g.h8 ? __shfl_sync(kFull, c.hsc, src) : 0.0f;
      const int jb = __shfl_sync(kFull, job, src);
      const int pl = __shfl_sync(kFull, plan, src);
      bool wg = false;
      if (ALG == ALGO_METAPATH) wg = __shfl_sync(kFull, (int)grp, src) != 0;
      const Job& JW = sj[jb];
      int32_t k;
      const int32_t hd = (ALG == ALGO_METAPATH && wg) ? w.pe - w.ps : w.d;
      if (pl == PLAN_EXACT_W) {
        const float u = u01(philox(make_uint4(w.wid, (uint32_t)w.step, 0u, 0u), JW.key0, JW.key1).x);
        k = exact_pick<32, COUNT, ALG>(g, JW, w, lane, u, lc);
      } else if (hd >= kHubMinDeg && hub_chunks(hd) <= kHubMaxChunks) {
        StepCtx cw = w;
        if (ALG == ALGO_METAPATH && wg) {
          cw.s = w.ps;
          cw.d = hd;
        }
        k = hub_step<COUNT, ALG, SHARE>(g, sj, JW, cw, jb, wg, hb, err, lc);
      } else if (ALG == ALGO_METAPATH && wg) {
        StepCtx cg = w;
        cg.s = w.ps;
        cg.d = w.pe - w.ps;
        k = rvs_pick<32, COUNT, ALG, true>(g, JW, cg, lane, !(JW.flags & FW_FLAG_RVS_NOJUMP), lc);
      } else {
        k = rvs_pick<32, COUNT, ALG>(g, JW, w, lane, !(JW.flags & FW_FLAG_RVS_NOJUMP), lc);
      }
      if (lane == src && ALG == ALGO_METAPATH && wg) {
        pick = -1;
        if (k >= 0) {  // grouped position -> node, position in the row, node record
          int4 a, b;
          ld_record(g.gerec + 2ll * (w.ps + k), a, b);
          if (COUNT) lc.bytes += 32;
          pick = b.z;
          node = a.x;
          nxt = make_int4(a.z, a.w, b.x, b.y);
          nxt_n0 = nxt_n1 = 0;  // metapath plans without weight classes
          nxt_ok = true;
        }
        h_in = -1.0f;
        if (COUNT) lc.rvs_steps++;
      } else if (lane == src) {
        pick = k;
        if (k >= 0) node = __ldg(g.col + w.s + k);
        h_in = -1.0f;
        if (COUNT) {
          if (pl == PLAN_EXACT_W) lc.exact_steps++;
          else lc.rvs_steps++;
        }
      }
    }
    // ------------------------------------------------------------ commit
    if (widx >= 0 && pick != -2) {
      const int32_t end = (J.kind == JOB_WALK) ? J.len : J.hstep + 1;
      if (J.kind == JOB_WALK) {
        if (pick >= 0) {
          stage_put(obuf, tid, rs, c.step + 1, node, c.step + 1 == end);
        } else {
          stage_fill_minus_one(obuf, tid, rs, c.step + 1, J.len + 1);
        }
      } else if (pick >= 0) {
        atomicAdd(J.hist + pick, 1ull);
      }
      if (pick >= 0) {
        c.vp = c.v;
        c.v = node;
        ++c.step;
        if (COUNT) {
          lc.hops++;
          lc.bytes += 4;
        }
        if (c.step >= end) widx = -1;
      } else {
        if (COUNT) lc.dead_ends++;
        widx = -1;
      }
      plan = PLAN_NONE;
      pick = -2;
    }
  }
}

// A warp with no walker left stops counting among the block's walking warps
// and, while any still walk, scans chunks of their hub steps (sleeping
// between checks).  Lingering is optional help: nothing waits for it, and the
// bound only caps how long a warp stays.
template <bool COUNT, int ALG>
__device__ __forceinline__ void hub_linger(const DevGraph& g, const Job* sj, HubBlock* hb, LaneCounters& lc) {
  if ((threadIdx.x & 31) == 0) atomicSub(&hb->live, 1);
  for (uint32_t it = 0; it < kLingerLimit; ++it) {
    if (hub_help<COUNT, ALG>(g, sj, hb, lc)) continue;
    if (__shfl_sync(kFull, *reinterpret_cast<volatile int32_t*>(&hb->live), 0) <= 0) break;
    __nanosleep(256);
  }
}

// Per-warp sums of the lane counters, added once to the device counters.
__device__ __forceinline__ void flush_counters(const LaneCounters& lc, DevCounters* cnt) {
  const int lane = threadIdx.x & 31;
  const unsigned long long v[11] = {lc.hops,     lc.rjs_steps, lc.rvs_steps, lc.exact_steps,
                                    lc.handoffs, lc.rjs_trials, lc.rvs_items, lc.rvs_keys,
                                    lc.probes,   lc.dead_ends, lc.bytes};
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(cnt);
#pragma unroll
  for (int f = 0; f < 11; ++f) {
    unsigned long long x = v[f];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if (lane == 0 && x) atomicAdd(dst + f, x);
  }
}

// Copy a job table into shared memory (all threads of the block).
__device__ __forceinline__ void load_jobs(const Job* src_jobs, int njobs, Job* sj) {
  const int words = njobs * (int)(sizeof(Job) / 4);
  const int* src = reinterpret_cast<const int*>(src_jobs);
  int* dst = reinterpret_cast<int*>(sj);
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

// Single-job (or one-algorithm) launch: the job table in shared memory, one
// walk loop per warp over the launch's queue.  SHARE: idle warps linger to
// help the block's hub steps.
template <int NJ, bool COUNT, int ALG, bool SHARE = false>
__global__ void __launch_bounds__(kBlock, kMinBlocks) walk_kernel(DevGraph g, JobTableN<NJ> tab, int njobs, long long total,
                                                      unsigned long long* __restrict__ qctr,
                                                      unsigned* __restrict__ err, DevCounters* __restrict__ cnt) {
  __shared__ Job sj[NJ];
  __shared__ int32_t obuf[kStageSlots * kBlock];
  __shared__ HubBlock hb;
  load_jobs(tab.jobs, njobs, sj);
  if (SHARE && threadIdx.x < kHubTasks) hb.task[threadIdx.x].word = 0u;
  if (SHARE && threadIdx.x == 0) {
    hb.open = 0;
    hb.live = (int32_t)(blockDim.x >> 5);
  }
  __syncthreads();
  LaneCounters lc;
  lc.zero();
  walk_loop<COUNT, ALG, SHARE>(g, sj, njobs, total, qctr, err, obuf, &hb, lc);
  if (SHARE) hub_linger<COUNT, ALG>(g, sj, &hb, lc);
  if (COUNT) flush_counters(lc, cnt);
}

template <int NJ, bool COUNT, int ALG, bool SHARE = false>
inline cudaError_t walk_blocks_per_sm(int* out) {
  static std::atomic<int> cached{0};
  int b = cached.load();
  if (b == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, walk_kernel<NJ, COUNT, ALG, SHARE>, kBlock, 0);
    if (e != cudaSuccess) return e;
    b = b > 0 ? b : 1;
    cached.store(b);
  }
  *out = b;
  return cudaSuccess;
}

// Hub sharing pays where warps would idle: launches that fill at most 1/8
// of the resident lanes, with eRVS forced (in the cost model's choice hub
// rows go to eRJS almost always) on a graph with hub rows.  The lingering
// code costs the loop about 13 % per step (measured on R-MAT s22), so big
// launches and the cost model's walks use the kernel without it; the rows
// are the same either way.
inline bool hub_share_pays(const fw_graph* g, const Job* jobs, int njobs, long long total, long long lanes) {
  if (g->max_degree < kHubMinDeg || total * 8 > lanes) return false;
  bool rvs = false;
  for (int i = 0; i < njobs; ++i) {
    if (jobs[i].flags & FW_FLAG_NO_HUB_SHARE) return false;
    rvs = rvs || jobs[i].mode == MODE_RVS;
  }
  return rvs;
}

template <int NJ, bool COUNT, int ALG>
inline cudaError_t launch_walk_t(const fw_graph* g, const Job* jobs, int njobs, long long total,
                                 unsigned long long* qctr, cudaStream_t stream) {
  int blocks_per_sm = 1;
  cudaError_t oe = walk_blocks_per_sm<NJ, COUNT, ALG>(&blocks_per_sm);
  if (oe != cudaSuccess) return oe;
  JobTableN<NJ> tab;
  for (int i = 0; i < njobs; ++i) tab.jobs[i] = jobs[i];
  const long long cap = (long long)g->num_sms * blocks_per_sm;
  if (!COUNT && hub_share_pays(g, jobs, njobs, total, cap * kBlock)) {
    int bs = 1;
    oe = walk_blocks_per_sm<NJ, false, ALG, true>(&bs);
    if (oe != cudaSuccess) return oe;
    // one warp's worth of walkers per block: the other warps of each block are free to help
    const long long want = (total + 31) / 32, cs = (long long)g->num_sms * bs;
    const int grid = (int)(want < cs ? (want > 0 ? want : 1) : cs);
    walk_kernel<NJ, false, ALG, true><<<grid, kBlock, 0, stream>>>(dev_graph(g), tab, njobs, total, qctr, g->d_err,
                                                                   g->d_cnt);
  } else {
    const long long want = (total + kBlock - 1) / kBlock;
    const int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    walk_kernel<NJ, COUNT, ALG><<<grid, kBlock, 0, stream>>>(dev_graph(g), tab, njobs, total, qctr, g->d_err,
                                                             g->d_cnt);
  }
  g_launches.fetch_add(1);
  return cudaGetLastError();
}

}  // namespace fw
