// fw_device.cuh -- device building blocks of the dynamic-random-walk engine.
//
// Every sampler here draws the next node of one walker-step from
//   p(u) = w~(v,u) / sum_t w~(v,t),  w~ = w * h          [Sec. 2.1, Eq. (prob)]
// with w from Eq. (node2vec), the MetaPath label rule, or w = 1 (weighted).
//   * eRJS   [Sec. 3.3]: propose X uniform over N(v), accept iff U*B < w~(X),
//            B = max(w) * h_MAX[v] >= max w~ (the proof in Sec. 3.3 shows the
//            accepted value follows p for any such bound).  Refined envelopes
//            keep that argument: X proposed in proportion to a per-entry
//            bound (weight classes of h), or from a mixture of components
//            each proposed and accepted against its own bound (return edge,
//            common neighbours, label segments); see rjs_trials.
//   * eRVS   [Sec. 3.2, Alg. 1, Eq. (jump)]: exponential keys
//            K_i = ln(u_i) / w~_i (the log of u_i^(1/w~_i)), argmax wins;
//            with jumps, a lane skips items until its cumulative weight passes
//            ln(r) / K_ref and draws the crossing item's key conditioned on
//            beating K_ref (A-ExpJ of Efraimidis & Spirakis, IPL 2006).
//   * exact  [Sec. 2.2, ITS]: FP32 prefix in neighbour order, t = u * W_{d-1},
//            first k with t < W_k (fallback: last k with w~_k > 0).
// Random numbers come from Philox4x32-10 (Salmon et al., SC'11) keyed by the
// walk seed with counter (walker id, hop, stream, draw); stream 0 is the exact
// mode, 1 eRJS (draw = trial), 2 eRVS crossings (draw = neighbour position),
// 5-7 eRVS jump thresholds and phase-1 keys (see rvs_scan and the hub
// steps).  No draw depends on the lane, block or co-running walkers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

namespace fw {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxJobs = 64;
constexpr int kLaneMaxDegree = 8;    // default: eRVS steps with d <= this run on one lane
constexpr int kRjsBatchDefault = 2;  // default: eRJS trials per round before the warp ballot
constexpr int kLabelStats = 8;       // per-label node statistics for labels 0..7
constexpr int kWClasses = 5;         // weight classes inside a metapath label segment

enum : int32_t { ALGO_WEIGHTED = 0, ALGO_NODE2VEC = 1, ALGO_METAPATH = 2, ALGO_PAGERANK2 = 3 };
constexpr int kAlgos = 4;  // a multi-job launch keeps one walker queue per algorithm
enum : int32_t { MODE_AUTO = 0, MODE_RJS = 1, MODE_RVS = 2, MODE_EXACT = 3, MODE_RANDOM = 4, MODE_DEGREE = 5 };
constexpr int32_t kDegreeRuleThreshold = 1000;  // Sec. 5.4 degree-based selection
enum : int32_t { JOB_WALK = 0, JOB_HIST = 1 };
enum : int32_t { PLAN_NONE = 0, PLAN_RJS = 1, PLAN_RVS_T = 2, PLAN_RVS_W = 3, PLAN_EXACT_T = 4, PLAN_EXACT_W = 5 };
enum : uint32_t { DEVERR_START = 1u, DEVERR_HUB = 2u };

struct DevGraph {
  const int32_t* __restrict__ off;
  const int32_t* __restrict__ col;
  const float* __restrict__ h;     // nullptr: h = 1
  const uint8_t* __restrict__ h8;  // 8-bit weight codes (nullptr: FP32 weights); h(v,u) = code * h8scale[v]
  const float* __restrict__ h8scale; // per node: the scale of the codes of its row
  const uint8_t* __restrict__ lab; // nullptr: no labels
  const float* __restrict__ hmax;
  const float* __restrict__ hsum;
  const int4* __restrict__ nrec;   // per node 32 bytes: {row start, degree, h_MAX bits, h_SUM bits},
                                   // {n0, n1, 0, 0}: entries of weight class 0 (h > h_MAX / 2) and
                                   // class 1 (h_MAX / 4 < h <= h_MAX / 2); one sector per plan
  const int4* __restrict__ erec;   // per edge 32 bytes: {col, h bits, target row start, target degree},
                                   // {target h_MAX bits, target h_SUM bits, label | target n0 << 8,
                                   // target n1}: one sector per eRJS trial
  const int4* __restrict__ cerec;  // the edge records with every row partitioned stably into weight
                                   // classes 0, 1, 2 (class 2: h <= h_MAX / 4); nullptr: no classes
  const float2* __restrict__ lstat; // per node and label l < kLabelStats: {max h, sum h} over the
                                   // edges with that label (nullptr: labels absent or >= kLabelStats)
  const uint32_t* __restrict__ bloom; // blocked Bloom filters of the rows (nullptr: none)
  const int32_t* __restrict__ mtab;   // per-row membership tables of the node ids (nullptr: none)
  // label-grouped view of the rows (metapath; nullptr: not built): each row
  // reordered stably by (label, weight class).  lrec per node and label
  // l < kLabelStats, 32 bytes: {max h bits, sum h bits, segment start
  // relative to the row start, segment length}, {entries of classes
  // 0 .. kWClasses-2}; class c holds h in (max / 2^(c+1), max / 2^c], the
  // last class the rest.  gerec: edge records in grouped order with the
  // entry's original position in the row in place of the label; gh: h in
  // grouped order.
  const int4* __restrict__ lrec;
  const int4* __restrict__ gerec;
  const float* __restrict__ gh;
  int32_t n;
  int32_t sym;                     // 1: h(v,u) = h(u,v) for every edge (checked at creation)
};

// One walk job (a batch is a table of these).  Walkers of all jobs form one
// global index space: job j owns [gbase, gbase + num_walkers).
struct Job {
  const int32_t* starts;
  const uint32_t* wids;    // random-stream id per walker (nullptr: walker_base + index)
  int32_t* out;
  unsigned long long* hist;
  long long gbase;
  int32_t num_walkers, len;
  int32_t kind, algo, mode, flags;
  int32_t rjs_cap, schema_len;
  int32_t weighted;        // 1: use h, 0: h = 1
  int32_t second_order;    // node2vec with (1/p, 1/q) != (1, 1): w depends on v'
  int32_t need_member;     // node2vec with 1/q != 1: membership test needed
  int32_t fixed_cap;       // 1: rjs_cap is a fixed trial cap; 0: cap = max(rjs_cap, ceil(budget * d / ratio))
  int32_t lane_max;        // eRVS steps over at most this many entries run on the walker's lane
  int32_t rjs_batch;       // eRJS trials per round before the warp's hand-off ballot
  float budget;            // trial budget scale of the default cap
  int32_t split_return;    // node2vec with 1/p > max(1, 1/q): eRJS proposes the return edge separately
  int32_t split_common;    // node2vec with 1/q < 1: eRJS may use the two-envelope proposal (d(v') < d(v))
  int32_t label_stats;     // metapath: plan with the per-label h_MAX / h_SUM of the required label
  int32_t label_group;     // metapath: fast modes sample inside the required label's segment
  int32_t classes;         // eRJS proposes from three weight classes (bounds B, B / 2, B / 4)
  int32_t bloom;           // 1: membership tests in N(v') consult the row's Bloom filter first
  int32_t table;           // 1: membership tests read the row's membership table instead of searching
  float inv_p, inv_q;      // FP32 1/p, 1/q
  float wmax1, wmean1;     // max / mean of w when a previous node exists
  float wlo1, whi1;        // min / max of {1, 1/q}: squeeze bounds of a non-return neighbour
  float ratio;             // r of Eq. (runtime)
  float pr_g, pr_1g;       // second-order PageRank: gamma and 1 - gamma (FP32)
  uint32_t key0, key1, walker_base;
  int32_t hv, hprev, hstep;  // JOB_HIST: the fixed state
  uint8_t schema[16];
};

struct JobTable {
  Job jobs[kMaxJobs];
};

// Counters kept by the counting build of the kernel (FW_FLAG_COUNTERS).
struct DevCounters {
  unsigned long long hops, rjs_steps, rvs_steps, exact_steps, handoffs, rjs_trials, rvs_items, rvs_keys,
      probes, dead_ends, bytes;
};

struct LaneCounters {
  uint32_t hops, rjs_steps, rvs_steps, exact_steps, handoffs, rjs_trials, rvs_items, rvs_keys, probes,
      dead_ends;
  unsigned long long bytes;
  __device__ void zero() {
    hops = rjs_steps = rvs_steps = exact_steps = handoffs = rjs_trials = rvs_items = rvs_keys = probes = dead_ends = 0;
    bytes = 0;
  }
};

// Algorithm of job J.  The walk kernels pass it as the template argument
// ALG >= 0, so the other algorithms' code folds away; ALG = -1 reads it
// from the job (the autotuner's profiling kernels).
#define FW_ALGO(J) ((ALG) >= 0 ? (ALG) : (J).algo)

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with the published multipliers; high halves are XORed
// with the other counter words and the round key; the key advances by the
// published Weyl increments between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// [0,1) on a 2^-24 grid
__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * 0x1.0p-24f; }
// (0,1): odd multiples of 2^-24, never 0 or 1 (safe for log)
__device__ __forceinline__ float u01_open(uint32_t x) { return (float)(((x >> 9) << 1) | 1u) * 0x1.0p-24f; }

// ---------------------------------------------------------------- gathers
// One 32-byte edge record in a single 256-bit read-only load that does not
// allocate in L1: records are gathered at random, so L1 lines would only
// evict the rows that membership searches and scans reuse.  (Measured on
// R-MAT s22 node2vec: 2-3 % faster than an allocating load, and ld.global.cg
// 5-14 % slower; DRAM bytes per hop are the same for all three, about four
// sectors per record.)
__device__ __forceinline__ void ld_record(const int4* p, int4& a, int4& b) {
  asm volatile("ld.global.nc.L1::no_allocate.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
               : "l"(p));
}

// ---------------------------------------------------------------- per-step context
struct StepCtx {
  int32_t v, vp;    // current and previous node (vp < 0: none)
  int32_t s, d;     // row start and degree of v
  int32_t ps, pe;   // row range of vp (node2vec membership)
  int32_t step;     // hop index
  uint32_t wid;     // random-stream walker id
  float w1, w2;     // second-order PageRank weights of this step: u in N(v') / otherwise
  int32_t n0, n1;   // eRJS weight classes: entries of v in classes 0 and 1 (n0 < 0: one class)
  int4 gcls;        // grouped metapath: entries of weight classes 0..3 in the label segment [ps, pe)
  float hsc;        // 8-bit weight codes: the scale of v's row (unused with FP32 weights)
};

// Slots of a label segment's weight-class envelope: class c < kWClasses
// gives each of its entries 2^(kWClasses-1-c) slots (its bound is max / 2^c).
__device__ __forceinline__ uint32_t class_slots(const int4& n, int32_t len) {
  const uint32_t n4 = (uint32_t)(len - n.x - n.y - n.z - n.w);
  return 16u * (uint32_t)n.x + 8u * (uint32_t)n.y + 4u * (uint32_t)n.z + 2u * (uint32_t)n.w + n4;
}

// Eq. (2ndpr) weights for degrees dv = d(v), dp = d(v'):
// t1 = (1-g)/dv, t2 = g/dp, m = max(dv, dp), w1 = (t1 + t2) * m, w2 = t1 * m.
__device__ __forceinline__ void pagerank2_weights(const Job& J, int32_t dv, int32_t dp, float& w1, float& w2) {
  const float fv = (float)dv, fp = (float)dp;
  const float t1 = __fdiv_rn(J.pr_1g, fv);
  const float t2 = __fdiv_rn(J.pr_g, fp);
  const float m = fmaxf(fv, fp);
  w1 = __fmul_rn(__fadd_rn(t1, t2), m);
  w2 = __fmul_rn(t1, m);
}

// Position of u in the sorted row col[lo, hi) (all ids in [0, n)), or -1.
// A few interpolation probes first -- the guess puts u at its place between
// the bracketing values; a row of a graph with randomly permuted ids is close
// to a uniform sample of [0, n), so it lands within a few entries -- then
// bisection of the remaining window of at most 8 entries (one or two
// sectors, already in L1).  Exits early on a hit.  At most
// kInterpProbes + ceil(log2(d + 1)) probes.  (Probes that read a whole
// 32-byte sector, and searching the shorter of N(u) and N(v') on symmetric
// graphs, were measured slower: each probe costs more and lands in colder
// rows.)
constexpr int kInterpProbes = 4;
__device__ __forceinline__ int32_t row_find(const int32_t* __restrict__ col, int32_t lo, int32_t hi, int32_t u,
                                            int32_t n, uint32_t& probes) {
  float va = -1.0f, vb = (float)n;  // every id in [lo, hi) lies strictly between va and vb
#pragma unroll 1
  for (int it = 0; it < kInterpProbes && hi - lo > 8; ++it) {
    const float f = ((float)u - va) / (vb - va);
    int32_t g = lo + (int32_t)(f * (float)(hi - lo));
    g = min(max(g, lo), hi - 1);
    const int32_t c = __ldg(col + g);
    ++probes;
    if (c == u) return g;
    if (c < u) {
      lo = g + 1;
      va = (float)c;
    } else {
      hi = g;
      vb = (float)c;
    }
  }
  int32_t len = hi - lo;
  while (len > 0) {
    const int32_t half = len >> 1;
    const int32_t c = __ldg(col + lo + half);
    ++probes;
    if (c == u) return lo + half;
    if (c < u) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return -1;
}

// ---------------------------------------------------------------- membership
// Blocked Bloom filters over the rows: a pre-check in front of row_find that
// never changes an answer, it only skips searches whose answer is "absent"
// (most node2vec candidates with q > 1 lie at distance 2 from v').  Node x
// owns the 256-bit blocks [bb(x), bb(x+1)) with bb(x) = floor(off[x]/32) + x,
// one block per 32 row entries plus one; entry u of the row sets kBloomBits
// bits of one of them, so a filter holds at least 8 bits per entry (false
// positive rate about 3 %).  Block and bits come from a 64-bit mix of u (the
// 64-bit finalizer of MurmurHash3, A. Appleby).  Rows shorter than
// kBloomMinDeg span one or two sectors and are searched directly.
constexpr int32_t kBloomMinDeg = 16;
constexpr int kBloomBits = 4;
constexpr int32_t kPr2SplitMaxPrev = 64;  // second-order PageRank: longest N(v') enumerated for the split

__device__ __forceinline__ unsigned long long bloom_mix(uint32_t u) {
  unsigned long long k = (unsigned long long)u + 0x9E3779B97F4A7C15ull;
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// First word of the block of row x = [rs, re) that entry hash hk maps to.
__device__ __forceinline__ long long bloom_word(int32_t x, int32_t rs, int32_t re, unsigned long long hk) {
  const long long b0 = (long long)(rs >> 5) + x;
  const uint32_t nb = (uint32_t)((re >> 5) - (rs >> 5) + 1);
  return 8ll * (b0 + (long long)__umulhi((uint32_t)(hk >> 32), nb));
}

// Membership tables: an exact set of each row's node ids for rows of at least
// kBloomMinDeg entries.  Node x owns the 32-byte buckets [tb(x), tb(x+1)),
// tb(x) = floor(off[x]/4) + x -- more than d/4 buckets of 8 slots, so at most
// half the slots hold an id and the rest are -1.  Id u lives in the first
// free slot at or after its home bucket umulhi(hash(u), buckets) (linear
// probing by bucket, wrapping within the row; hash = the high word of the
// Bloom mix).  Slots fill in order and are never cleared, so every bucket
// from u's home to the one holding u is full: a lookup reads one bucket,
// answers "present" on a match and "absent" on a free slot, and moves on
// only from a full bucket without u (about 5 % of lookups at load 1/2).
__device__ __forceinline__ long long table_bucket0(int32_t x, int32_t rs) { return (long long)(rs >> 2) + x; }
__device__ __forceinline__ uint32_t table_buckets(int32_t rs, int32_t re) {
  return (uint32_t)((re >> 2) - (rs >> 2) + 1);
}

// One 32-byte bucket in a single load that does not allocate in L1 (as
// ld_record; a bucket read as two 16-byte loads costs two random accesses).
// Written as four 64-bit words: the eight-word form of ld_record in this
// function crashes the assembler of CUDA 13.0.
__device__ __forceinline__ void ld_bucket(const int32_t* p, int4& a, int4& c) {
  unsigned long long q0, q1, q2, q3;
  asm volatile("ld.global.nc.L1::no_allocate.v4.b64 {%0, %1, %2, %3}, [%4];"
               : "=l"(q0), "=l"(q1), "=l"(q2), "=l"(q3)
               : "l"(p));
  a = make_int4((int)q0, (int)(q0 >> 32), (int)q1, (int)(q1 >> 32));
  c = make_int4((int)q2, (int)(q2 >> 32), (int)q3, (int)(q3 >> 32));
}

// Buckets after a full home bucket (rare): one 32-byte load each.
static __device__ __noinline__ bool table_contains_more(const int32_t* __restrict__ tab, long long b0, uint32_t nb,
                                                        uint32_t b, int32_t u, uint32_t& probes) {
  for (uint32_t k = 1; k < nb; ++k) {
    b = (b + 1 == nb) ? 0u : b + 1;
    int4 a, c;
    ld_bucket(tab + 8ll * (b0 + b), a, c);
    ++probes;
    if (a.x == u || a.y == u || a.z == u || a.w == u || c.x == u || c.y == u || c.z == u || c.w == u) return true;
    if (c.w == -1) return false;
  }
  return false;
}

__device__ __forceinline__ bool table_contains(const int32_t* __restrict__ tab, int32_t x, int32_t rs, int32_t re,
                                               uint32_t hhi, int32_t u, uint32_t& probes) {
  const long long b0 = table_bucket0(x, rs);
  const uint32_t nb = table_buckets(rs, re);
  const uint32_t b = __umulhi(hhi, nb);
  int4 a, c;  // the home bucket
  ld_bucket(tab + 8ll * (b0 + b), a, c);
  ++probes;
  if (a.x == u || a.y == u || a.z == u || a.w == u || c.x == u || c.y == u || c.z == u || c.w == u) return true;
  if (c.w == -1) return false;  // slots fill in order: a free last slot means u is not in the row
  return table_contains_more(tab, b0, nb, b, u, probes);
}

// Bloom test of u against row x (one probe): false means u is certainly
// not in the row.
__device__ __forceinline__ bool bloom_maybe(const DevGraph& g, int32_t x, int32_t rs, int32_t re,
                                            unsigned long long hk, uint32_t& probes) {
  const uint32_t* blk = g.bloom + bloom_word(x, rs, re, hk);
  ++probes;
  uint32_t hit = 1u;
#pragma unroll
  for (int j = 0; j < kBloomBits; ++j) {
    const uint32_t bit = (uint32_t)(hk >> (8 * j)) & 255u;
    hit &= __ldg(blk + (bit >> 5)) >> (bit & 31u);
  }
  return (hit & 1u) != 0u;
}

// Is u in the row [rs, re) of node x?  Rows of at least kBloomMinDeg
// entries: the membership table (one probe per bucket read), or without it
// the Bloom filter (one probe) and a search of the row where the filter
// passes; shorter rows: the search.  Exact.
__device__ __forceinline__ bool row_member(const DevGraph& g, const Job& J, int32_t x, int32_t rs, int32_t re,
                                           int32_t u, uint32_t& probes) {
  if (re - rs >= kBloomMinDeg) {
    if (J.table) return table_contains(g.mtab, x, rs, re, (uint32_t)(bloom_mix((uint32_t)u) >> 32), u, probes);
    if (J.bloom && !bloom_maybe(g, x, rs, re, bloom_mix((uint32_t)u), probes)) return false;
  }
  return row_find(g.col, rs, re, u, g.n, probes) >= 0;
}

// Membership for the scans of eRVS and exact mode, which test every
// neighbour of v against the same row of v': the Bloom filter first (its
// 32-byte blocks, 8 bits per entry, stay cached through the scan), then the
// table where the filter passes (or, without tables, the search).  Exact.
__device__ __forceinline__ bool row_member_scan(const DevGraph& g, const Job& J, int32_t x, int32_t rs, int32_t re,
                                                int32_t u, uint32_t& probes) {
  if (re - rs >= kBloomMinDeg) {
    const unsigned long long hk = bloom_mix((uint32_t)u);
    if (J.bloom && !bloom_maybe(g, x, rs, re, hk, probes)) return false;
    if (J.table) return table_contains(g.mtab, x, rs, re, (uint32_t)(hk >> 32), u, probes);
  }
  return row_find(g.col, rs, re, u, g.n, probes) >= 0;
}

// Position of u in the row [rs, re) of node x, or -1: the table or the
// filter answers "absent" without a search; otherwise the search gives the
// position.  Exact.
__device__ __forceinline__ int32_t row_lookup(const DevGraph& g, const Job& J, int32_t x, int32_t rs, int32_t re,
                                              int32_t u, uint32_t& probes) {
  if (re - rs >= kBloomMinDeg) {
    if (J.table) {
      if (!table_contains(g.mtab, x, rs, re, (uint32_t)(bloom_mix((uint32_t)u) >> 32), u, probes)) return -1;
    } else if (J.bloom && !bloom_maybe(g, x, rs, re, bloom_mix((uint32_t)u), probes)) {
      return -1;
    }
  }
  return row_find(g.col, rs, re, u, g.n, probes);
}

// Is u in N(v') (the row [c.ps, c.pe) of c.vp)?  SCAN: the test of a scan
// over N(v) (eRVS, exact mode) rather than of one eRJS trial.
template <bool SCAN = false>
__device__ __forceinline__ bool prev_contains(const DevGraph& g, const Job& J, const StepCtx& c, int32_t u,
                                              uint32_t& probes) {
  return SCAN ? row_member_scan(g, J, c.vp, c.ps, c.pe, u, probes) : row_member(g, J, c.vp, c.ps, c.pe, u, probes);
}


// Property weight of CSR entry i of the row whose code scale is sc: FP32, or
// an 8-bit code times sc.
__device__ __forceinline__ float load_h(const DevGraph& g, const Job& J, int32_t i, float sc) {
  if (!J.weighted) return 1.0f;
  return g.h8 ? __fmul_rn((float)__ldg(g.h8 + i), sc) : __ldg(g.h + i);
}

// Second-order PageRank with a short row of v' (Eq. 2ndpr): the common
// neighbours C = N(v) and N(v') carry w1 > w2, all others w2.  Enumerating
// N(v') finds C and S_C = sum of h(v, x) over x in C (FP32, in N(v') order).
// With t in [0, S_C), common_pick returns the x in C where that running sum
// first exceeds t (the last one if rounding leaves none), its position in
// N(v) relative to the row start, and h(v, x).
static __device__ __noinline__ float common_h_sum(const DevGraph& g, const Job& J, const StepCtx& c, uint32_t& probes) {
  float sc = 0.0f;
  for (int32_t j = c.ps; j < c.pe; ++j) {
    const int32_t pos = row_lookup(g, J, c.v, c.s, c.s + c.d, __ldg(g.col + j), probes);
    if (pos >= 0) sc = __fadd_rn(sc, load_h(g, J, pos, c.hsc));
  }
  return sc;
}

static __device__ __noinline__ int32_t common_pick(const DevGraph& g, const Job& J, const StepCtx& c, float t,
                                               int32_t& k, float& hx, uint32_t& probes) {
  float run = 0.0f;
  int32_t node = -1;
  for (int32_t j = c.ps; j < c.pe; ++j) {
    const int32_t x = __ldg(g.col + j);
    const int32_t pos = row_lookup(g, J, c.v, c.s, c.s + c.d, x, probes);
    if (pos < 0) continue;
    const float h = load_h(g, J, pos, c.hsc);
    run = __fadd_rn(run, h);
    node = x;
    k = pos - c.s;
    hx = h;
    if (t < run) break;
  }
  return node;
}

// Transition weight of the neighbour at CSR index i (= s + k) of step c.
// Transition weight w~ = w * hk of neighbour u (label lb) of step c.
template <int ALG = -1>
__device__ __forceinline__ float weight_of(const DevGraph& g, const Job& J, const StepCtx& c, float hk, int32_t u,
                                           uint8_t lb, uint32_t& probes) {
  if (FW_ALGO(J) == ALGO_NODE2VEC) {
    if (c.vp < 0 || !J.second_order) return hk;
    float w;
    if (u == c.vp) w = J.inv_p;                       // dist(v',u) = 0
    else if (!J.need_member) w = 1.0f;                // 1/q == 1: distances 1 and 2 weigh the same
    else w = prev_contains<true>(g, J, c, u, probes) ? 1.0f : J.inv_q;
    return __fmul_rn(w, hk);
  }
  if (FW_ALGO(J) == ALGO_METAPATH) return (lb == J.schema[c.step % J.schema_len]) ? hk : 0.0f;  // w in {0, 1}
  if (FW_ALGO(J) == ALGO_PAGERANK2 && c.vp >= 0)
    return __fmul_rn(prev_contains<true>(g, J, c, u, probes) ? c.w1 : c.w2, hk);
  return hk;
}

// Does step c's weight read the neighbour's id / its label?
template <int ALG = -1>
__device__ __forceinline__ bool weight_needs_col(const Job& J, const StepCtx& c) {
  return (FW_ALGO(J) == ALGO_NODE2VEC && c.vp >= 0 && J.second_order) || (FW_ALGO(J) == ALGO_PAGERANK2 && c.vp >= 0);
}

template <int ALG = -1>
__device__ __forceinline__ float item_weight(const DevGraph& g, const Job& J, const StepCtx& c, int32_t i,
                                             uint32_t& probes) {
  const float hk = load_h(g, J, i, c.hsc);
  const int32_t u = weight_needs_col<ALG>(J, c) ? __ldg(g.col + i) : -1;
  const uint8_t lb = (FW_ALGO(J) == ALGO_METAPATH) ? __ldg(g.lab + i) : (uint8_t)0;
  return weight_of<ALG>(g, J, c, hk, u, lb, probes);
}

// ---------------------------------------------------------------- plan
// Bound (Sec. 3.3), sum estimate (Eq. sum_estimation) and choice (Eq. runtime).
template <int ALG = -1>
__device__ __forceinline__ int32_t plan_choice(const Job& J, float hm, float hs, bool has_prev, float w1, float w2,
                                               float& B, float& S) {
  const bool second = (FW_ALGO(J) == ALGO_NODE2VEC) && has_prev;
  const bool pr2 = (FW_ALGO(J) == ALGO_PAGERANK2) && has_prev;
  const float wmax = second ? J.wmax1 : (pr2 ? w1 : 1.0f);
  const float wmean = second ? J.wmean1 : (pr2 ? __fmul_rn(__fadd_rn(w1, w2), 0.5f)
                                               : ((FW_ALGO(J) == ALGO_METAPATH) ? 0.5f : 1.0f));
  B = __fmul_rn(wmax, hm);
  S = __fmul_rn(hs, wmean);
  return (__fmul_rn(J.ratio, B) < S) ? MODE_RJS : MODE_RVS;
}

// ---------------------------------------------------------------- eRJS
// Exactly uniform index in [0, d) by Lemire's multiply-shift with rejection
// (ACM TOMACS 2019): x0 proposes, x1 is the one retry; false when both fall
// in the rejection zone (the trial then proposes nothing).
__device__ __forceinline__ bool lemire_index(uint32_t x0, uint32_t x1, uint32_t d, uint32_t& k) {
  unsigned long long m = (unsigned long long)x0 * d;
  uint32_t l = (uint32_t)m;
  if (l < d) {
    const uint32_t thr = (0u - d) % d;
    if (l < thr) {
      m = (unsigned long long)x1 * d;
      l = (uint32_t)m;
      if (l < thr) return false;
    }
  }
  k = (uint32_t)(m >> 32);
  return true;
}

// One eRJS acceptance: the neighbour position, the node, its effective
// property weight, and the target's node record (rec_ok = 0: unknown).
struct Accept {
  int32_t k, node;
  float h;
  int4 rec;        // target's {row start, degree, h_MAX bits, h_SUM bits}
  int32_t rec_n0, rec_n1;  // target's weight-class counts
  bool rec_ok;
};

// Run trials [t0, t0+nt) of one walker-step; returns true on acceptance.
// Trial t uses Philox counter (wid, hop, 1, t): x.x (x.y on Lemire's rare
// retry) proposes X uniformly in [0,d) by Lemire's multiply-shift with
// rejection (ACM TOMACS 2019); x.z gives U in [0,1); x.w picks the return
// component when the return edge is split off (beta > 0).
//
// Plain eRJS (Sec. 3.3): accept X iff U*B < w~(X).
// Split return edge (node2vec when 1/p dominates the bound): with
// probability beta = w~_ret / (w~_ret + d*B) the trial proposes v' and
// accepts it; otherwise X is uniform over N(v), X = v' proposes nothing, and
// X != v' is accepted iff U*B < w~(X) with B = max(1, 1/q) * h_MAX[v].
// Accepted v' has probability beta and accepted x has (1-beta) w~(x)/(d B):
// both proportional to w~, so the accepted draw follows Eq. (prob).
// Split common neighbours (second-order PageRank, short N(v'), w1 > 2 w2):
// w~(x) = w2 h(x) + (w1 - w2) h(x) [x in C].  With probability
// beta = (w1-w2) S_C / ((w1-w2) S_C + d*B), B = w2 * h_MAX[v], the trial
// picks x in C with probability h(x) / S_C (h_ret holds S_C) and accepts it;
// otherwise X is uniform over N(v) and accepted iff U*B < w2 h(X).  The two
// parts are proportional to the two terms of w~, so again the accepted
// draw follows Eq. (prob).
// Two envelopes (node2vec with 1/q < 1 and d(v') < d(v)): write
// w~(x) = (1/q) h(x) + (1 - 1/q) h(x) [x in N(v')] for x != v'.  The first
// term is covered by (1/q) h_MAX[v] on N(v), the second by
// (1 - 1/q) h_MAX[v] on N(v'); with the return edge as a third component,
// a trial picks a component in proportion to its envelope mass
// (E3 = w~_ret, E2 = (1 - 1/q) d(v') h_MAX, E1 = (1/q) d(v) h_MAX; `beta`
// and `beta2` are E3 / E and (E3 + E2) / E) and accepts with probability
// target / envelope: component 1 proposes X uniform over N(v) (X = v'
// proposes nothing) and accepts iff U h_MAX < h(X), with no membership test;
// component 2 proposes X uniform over N(v') and accepts iff X is in N(v) and
// U h_MAX < h(v, X).  The accepted x carries (1/q) h(x) from the first and
// (1 - 1/q) h(x) [x in N(v')] from the second: w~(x) in total.  The envelope
// mass is (1/q) d + (1 - 1/q) d' < d, so fewer trials than the one-envelope
// bound max(1, 1/q) h_MAX = h_MAX (B = h_MAX is passed in this case).
template <bool COUNT, int ALG = -1>
__device__ __forceinline__ bool rjs_trials(const DevGraph& g, const Job& J, const StepCtx& c, float B, bool split,
                                           float beta, int32_t pos_ret, float h_ret, int32_t t0, int32_t nt,
                                           Accept& acc, LaneCounters& lc, bool csplit = false, float beta2 = 0.0f,
                                           bool grp = false) {
  const uint32_t d = (uint32_t)c.d;
  const uint8_t want = (FW_ALGO(J) == ALGO_METAPATH) ? J.schema[c.step % J.schema_len] : 0;
  const bool second = (FW_ALGO(J) == ALGO_NODE2VEC) && c.vp >= 0 && J.second_order;
  uint32_t probes = 0;
  bool found = false;
  for (int32_t t = t0; t < t0 + nt; ++t) {
    const uint4 x = philox(make_uint4(c.wid, (uint32_t)c.step, 1u, (uint32_t)t), J.key0, J.key1);
    if (COUNT) lc.rjs_trials++;
    const float ucomp = u01(x.w);
    if (beta > 0.0f && ucomp < beta) {
      if (FW_ALGO(J) == ALGO_PAGERANK2) {
        uint32_t pb = 0;
        acc.node = common_pick(g, J, c, __fmul_rn(u01(x.z), h_ret), acc.k, acc.h, pb);
        probes += pb;
      } else {
        acc.k = pos_ret >= 0 ? pos_ret : 0;
        acc.node = c.vp;
        acc.h = h_ret;
      }
      acc.rec_ok = false;
      found = true;
      break;
    }
    int4 a, b;  // {col, h, target row start, target degree}, {target h_MAX, target h_SUM, label, 0}
    if ((FW_ALGO(J) == ALGO_METAPATH) && grp) {
      // metapath inside the required label's segment [c.ps, c.pe) of the grouped
      // arrays, every entry of w = 1, ordered by weight class: slot t of the
      // class envelope (class_slots) proposes an entry of class c in proportion
      // to its bound B / 2^c, B = max h over the segment; accept iff U * bound < h
      static_assert(kWClasses == 5, "slot walk below is written for five classes");
      uint32_t t;
      if (!lemire_index(x.x, x.y, class_slots(c.gcls, c.pe - c.ps), t)) continue;
      uint32_t base = 0, kg;
      float Bg = B;
      const uint32_t n0 = (uint32_t)c.gcls.x, n1 = (uint32_t)c.gcls.y, n2 = (uint32_t)c.gcls.z,
                     n3 = (uint32_t)c.gcls.w;
      if (t < 16u * n0) {
        kg = t >> 4;
      } else {
        t -= 16u * n0;
        base = n0;
        Bg = __fmul_rn(0.5f, B);
        if (t < 8u * n1) {
          kg = base + (t >> 3);
        } else {
          t -= 8u * n1;
          base += n1;
          Bg = __fmul_rn(0.25f, B);
          if (t < 4u * n2) {
            kg = base + (t >> 2);
          } else {
            t -= 4u * n2;
            base += n2;
            Bg = __fmul_rn(0.125f, B);
            if (t < 2u * n3) {
              kg = base + (t >> 1);
            } else {
              kg = base + n3 + (t - 2u * n3);
              Bg = __fmul_rn(0.0625f, B);
            }
          }
        }
      }
      ld_record(g.gerec + 2ll * (c.ps + (int32_t)kg), a, b);  // b.z: position in the row
      if (COUNT) lc.bytes += 32;
      const float hg = J.weighted ? __int_as_float(a.y) : 1.0f;
      if (__fmul_rn(u01(x.z), Bg) < hg) {
        acc.k = b.z;
        acc.node = a.x;
        acc.h = hg;
        acc.rec = make_int4(a.z, a.w, b.x, b.y);
        acc.rec_n0 = acc.rec_n1 = 0;  // the label-grouped path plans without weight classes
        acc.rec_ok = true;
        found = true;
        break;
      }
      continue;
    }
    if ((FW_ALGO(J) == ALGO_NODE2VEC) && csplit && ucomp < beta2) {
      // component 2: X uniform over N(v'), accepted iff X in N(v) and U h_MAX < h(v, X)
      uint32_t k2;
      if (!lemire_index(x.x, x.y, (uint32_t)(c.pe - c.ps), k2)) continue;
      const int32_t X = __ldg(g.col + c.ps + (int32_t)k2);
      uint32_t pb = 0;
      const int32_t pos = row_lookup(g, J, c.v, c.s, c.s + c.d, X, pb);  // X = v is never in N(v)
      probes += pb;
      if (COUNT) lc.bytes += 32;
      if (pos < 0) continue;
      ld_record(g.erec + 2ll * pos, a, b);
      if (COUNT) lc.bytes += 32;
      const float hx = J.weighted ? __int_as_float(a.y) : 1.0f;
      if (__fmul_rn(u01(x.z), B) < hx) {
        acc.k = pos - c.s;
        acc.node = X;
        acc.h = hx;
        acc.rec = make_int4(a.z, a.w, b.x, b.y);
        acc.rec_n0 = (int32_t)((uint32_t)b.z >> 8);
        acc.rec_n1 = b.w;
        acc.rec_ok = true;
        found = true;
        break;
      }
      continue;
    }
    uint32_t ku;
    float Bc = B;  // bound of the proposed entry's class
    const int4* er;
    if (c.n0 >= 0) {
      // three weight classes of bounds B, B / 2, B / 4 (h <= h_MAX / 2^c in class c): slot t of
      // 4 n0 + 2 n1 + n2 proposes an entry of class c in proportion to its bound
      const uint32_t n0 = (uint32_t)c.n0, n1 = (uint32_t)c.n1;
      uint32_t t;
      if (!lemire_index(x.x, x.y, 4u * n0 + 2u * n1 + (d - n0 - n1), t)) continue;
      if (t < 4u * n0) {
        ku = t >> 2;
      } else if (t - 4u * n0 < 2u * n1) {
        ku = n0 + ((t - 4u * n0) >> 1);
        Bc = __fmul_rn(0.5f, B);
      } else {
        ku = n0 + n1 + (t - 4u * n0 - 2u * n1);
        Bc = __fmul_rn(0.25f, B);
      }
      er = g.cerec + 2ll * (c.s + (int32_t)ku);
    } else {
      if (!lemire_index(x.x, x.y, d, ku)) continue;  // this trial proposes nothing; trials stay i.i.d.
      er = g.erec + 2ll * (c.s + (int32_t)ku);
    }
    const int32_t k = (int32_t)ku;
    ld_record(er, a, b);
    if (COUNT) lc.bytes += 32;
    const int32_t u = a.x;
    const float hk = J.weighted ? __int_as_float(a.y) : 1.0f;
    const float UB = __fmul_rn(u01(x.z), Bc);
    bool accept;
    if (second) {
      if (u == c.vp) {
        if (split) continue;                    // the return component owns v'
        accept = UB < __fmul_rn(J.inv_p, hk);
      } else if (csplit) {
        accept = UB < hk;                       // component 1: (1/q) h against (1/q) h_MAX
      } else if (UB >= __fmul_rn(J.whi1, hk)) {
        accept = false;                         // squeeze: above the largest possible weight
      } else if (UB < __fmul_rn(J.wlo1, hk)) {
        accept = true;                          // squeeze: below the smallest possible weight
      } else {
        uint32_t pb = 0;
        const bool adj = prev_contains(g, J, c, u, pb);
        probes += pb;
        accept = UB < __fmul_rn(adj ? 1.0f : J.inv_q, hk);
      }
    } else if (FW_ALGO(J) == ALGO_METAPATH) {
      accept = ((uint8_t)b.z == want) && (UB < hk);
    } else if (FW_ALGO(J) == ALGO_PAGERANK2 && c.vp >= 0 && split) {
      accept = UB < __fmul_rn(c.w2, hk);        // the w2 part; C is proposed by the split
    } else if (FW_ALGO(J) == ALGO_PAGERANK2 && c.vp >= 0) {
      if (UB >= __fmul_rn(c.w1, hk)) {
        accept = false;                         // squeeze: above the larger weight
      } else if (UB < __fmul_rn(c.w2, hk)) {
        accept = true;                          // squeeze: below the smaller weight
      } else {
        uint32_t pb = 0;
        const bool adj = prev_contains(g, J, c, u, pb);
        probes += pb;
        accept = UB < __fmul_rn(adj ? c.w1 : c.w2, hk);
      }
    } else {
      accept = UB < hk;
    }
    if (accept) {
      acc.k = k;
      if (c.n0 >= 0 && J.kind == JOB_HIST) {  // class order: the histogram wants the position in the row
        uint32_t pq = 0;
        acc.k = row_find(g.col, c.s, c.s + c.d, u, g.n, pq) - c.s;
      }
      acc.node = u;
      acc.h = hk;
      acc.rec = make_int4(a.z, a.w, b.x, b.y);
      acc.rec_n0 = (int32_t)((uint32_t)b.z >> 8);
      acc.rec_n1 = b.w;
      acc.rec_ok = true;
      found = true;
      break;
    }
  }
  if (COUNT) {
    lc.probes += probes;
    lc.bytes += 32ull * probes;
  }
  return found;
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ float warp_max(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(kFull, x, o));
  return x;
}

// argmax of (key, index); equal keys -> larger index (Alg. 1 uses >=)
__device__ __forceinline__ void warp_argmax(float& key, int32_t& idx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ok = __shfl_xor_sync(kFull, key, o);
    const int32_t oi = __shfl_xor_sync(kFull, idx, o);
    if (ok > key || (ok == key && oi > idx)) {
      key = ok;
      idx = oi;
    }
  }
}

// ---------------------------------------------------------------- eRVS
// T lanes cooperate on one walker-step (T = 1: a single lane; T = 32: the
// warp, all lanes converged with identical arguments).  Lane `lane` scans
// positions lane, lane+T, ...  Phase 1 keys the first T*m positions (m per
// lane, see phase1_items); their maximum is the reference K_ref from which
// every lane jumps over the rest of its own subsequence; the final argmax
// over lanes picks the neighbour.  Counter
// draws: phase 1 keys the lane's positions k, k+T, k+2T, k+3T from one block
// (wid, hop, 6, k) (x.x .. x.w; a Philox block costs more than the key it
// feeds, so one per four keys); the lane's first jump threshold is the
// block's unused x.w when phase 1 ends inside a block, else x.x of
// (wid, hop, 7, first position of the lane); a crossing at k draws
// (wid, hop, 2, k): x.y = its key, x.z = the lane's next threshold.  Returns position k or -1 (all
// weights zero: dead end).
// GRP: scan the label-grouped h (c.s, c.d are a segment of the grouped
// arrays, every entry of weight h); the result is a grouped position.
template <int ALG, bool GRP>
__device__ __forceinline__ float scan_weight(const DevGraph& g, const Job& J, const StepCtx& c, int32_t i,
                                             uint32_t& probes) {
  if (GRP) return J.weighted ? __ldg(g.gh + i) : 1.0f;
  return item_weight<ALG>(g, J, c, i, probes);
}

// Phase 1 keys each lane's first m positions, m growing with the entries per
// lane (1 .. kPhase1Max): the keys of phase 1 are drawn by all lanes at once,
// while each jump crossing afterwards runs in the one lane that crosses and
// stalls the rest of the warp; a larger phase 1 raises the reference K_g and
// leaves fewer crossings (about ln(1 + n/(T m)) per lane for n entries per
// lane), so a long row costs fewer divergent crossing blocks.
constexpr int32_t kPhase1Max = 8;
__device__ __forceinline__ int32_t phase1_items(int32_t d, int T) {
  const int32_t per = (d + T - 1) / T;
  return T == 1 ? 1 : min(kPhase1Max, max(1, per / 8));
}

// Counting build: a lane's share of an eRVS scan (summed over the lanes
// they give the step's totals).
template <int ALG, bool GRP>
__device__ __forceinline__ void rvs_count(const Job& J, int32_t scanned, int32_t keys, uint32_t probes,
                                          LaneCounters& lc) {
  lc.rvs_items += scanned;
  lc.rvs_keys += keys;
  lc.probes += probes;
  const int per = GRP ? (J.weighted ? 4 : 0)
                      : ((FW_ALGO(J) == ALGO_NODE2VEC) ? (J.weighted ? 8 : 4)
                                                       : (FW_ALGO(J) == ALGO_METAPATH ? (J.weighted ? 5 : 1)
                                                                                      : (J.weighted ? 4 : 0)));
  lc.bytes += (unsigned long long)scanned * per + 32ull * probes;
}

// The scan of positions [lo, hi) of the row: lane `lane` of T takes
// lo + lane, lo + lane + T, ...; phase 1 and the jumps as described above,
// with the reference taken over these T lanes.  Leaves the lane's best key
// and position in bestK / best (before any argmax over lanes).  Draws are
// keyed by the absolute position, so a range's result does not depend on
// which lanes or warps scan the other ranges.
template <int T, bool COUNT, int ALG = -1, bool GRP = false>
__device__ __forceinline__ void rvs_scan(const DevGraph& g, const Job& J, const StepCtx& c, int32_t lo, int32_t hi,
                                         int lane, bool jump, LaneCounters& lc, float& bestK, int32_t& best) {
  uint32_t probes = 0;
  bestK = -CUDART_INF_F;
  best = -1;
  uint32_t xz = 0;
  int32_t scanned = 0, keys = 0;
  const int32_t n = hi - lo;
  const int32_t m = phase1_items(n, T);
  uint4 x4 = make_uint4(0u, 0u, 0u, 0u);
  for (int32_t j = 0; j < m; ++j) {
    const int32_t k = lo + lane + T * j;
    if (k >= hi) break;
    const float wt = scan_weight<ALG, GRP>(g, J, c, c.s + k, probes);
    if ((j & 3) == 0) x4 = philox(make_uint4(c.wid, (uint32_t)c.step, 6u, (uint32_t)k), J.key0, J.key1);
    const uint32_t r = (j & 3) == 0 ? x4.x : ((j & 3) == 1 ? x4.y : ((j & 3) == 2 ? x4.z : x4.w));
    ++scanned;
    if (wt > 0.0f) {
      const float K = logf(u01_open(r)) / wt;
      ++keys;
      if (K >= bestK) {
        bestK = K;
        best = k;
      }
    }
  }
  if (n > T * m) {
    // the lane's first jump threshold: x.w of its last phase-1 block when that block fed fewer than four keys
    if (jump)
      xz = (m & 3) ? x4.w : philox(make_uint4(c.wid, (uint32_t)c.step, 7u, (uint32_t)(lo + lane)), J.key0, J.key1).x;
    float ref = bestK;
    if (T > 1) ref = warp_max(bestK);
    // remaining weight before the next crossing; K_ref = -inf: first positive item crosses
    float rem = (ref == -CUDART_INF_F) ? 0.0f : ((ref < 0.0f) ? logf(u01_open(xz)) / ref : CUDART_INF_F);
    for (int32_t k = lo + lane + T * m; k < hi; k += T) {
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
          // key conditioned on beating ref: u' ~ U(exp(ref*wt), 1), K = ln(u') / wt
          const float a = ref * wt;
          const float K = log1pf(expm1f(a) * u01_open(x.y)) / wt;
          ++keys;
          bestK = K;
          best = k;
          ref = K;
          rem = (ref < 0.0f) ? logf(u01_open(x.z)) / ref : CUDART_INF_F;
        }
      }
    }
  }
  if (COUNT) rvs_count<ALG, GRP>(J, scanned, keys, probes, lc);
}

template <int T, bool COUNT, int ALG = -1, bool GRP = false>
__device__ __forceinline__ int32_t rvs_pick(const DevGraph& g, const Job& J, const StepCtx& c, int lane, bool jump,
                                            LaneCounters& lc) {
  float bestK;
  int32_t best;
  rvs_scan<T, COUNT, ALG, GRP>(g, J, c, 0, c.d, lane, jump, lc, bestK, best);
  if (T > 1) warp_argmax(bestK, best);
  return (bestK == -CUDART_INF_F) ? -1 : best;
}

// ---------------------------------------------------------------- exact
// Exact inverse CDF with one uniform u: W_k accumulated with FP32 adds in
// neighbour order (T = 32: the warp loads 32 weights at a time and replays
// the additions in order through shuffles, so the sum is the serial one).
template <int T, bool COUNT, int ALG = -1>
__device__ __forceinline__ int32_t exact_pick(const DevGraph& g, const Job& J, const StepCtx& c, int lane, float u,
                                              LaneCounters& lc) {
  uint32_t probes = 0;
  float total = 0.0f;
  for (int32_t base = 0; base < c.d; base += T) {
    const int32_t k = base + lane;
    const float wt = (k < c.d) ? item_weight<ALG>(g, J, c, c.s + k, probes) : 0.0f;
    const int32_t cnt = min(T, c.d - base);
    if (T == 1) {
      total = __fadd_rn(total, wt);
    } else {
      for (int32_t j = 0; j < cnt; ++j) total = __fadd_rn(total, __shfl_sync(kFull, wt, j));
    }
  }
  int32_t pick = -1;
  if (total > 0.0f) {
    const float t = __fmul_rn(u, total);
    float run = 0.0f;
    for (int32_t base = 0; base < c.d && pick < 0; base += T) {
      const int32_t k = base + lane;
      const float wt = (k < c.d) ? item_weight<ALG>(g, J, c, c.s + k, probes) : 0.0f;
      const int32_t cnt = min(T, c.d - base);
      if (T == 1) {
        run = __fadd_rn(run, wt);
        if (t < run) pick = k;
      } else {
        float mine = 0.0f;
        for (int32_t j = 0; j < cnt; ++j) {
          run = __fadd_rn(run, __shfl_sync(kFull, wt, j));
          if (j == lane) mine = run;
        }
        const unsigned hit = __ballot_sync(kFull, lane < cnt && t < mine);
        if (hit) pick = base + __ffs(hit) - 1;
      }
    }
    if (pick < 0) {  // rounding left t >= W_{d-1}: last positive weight
      for (int32_t base = ((c.d - 1) / T) * T; base >= 0 && pick < 0; base -= T) {
        const int32_t k = base + lane;
        const float wt = (k < c.d) ? item_weight<ALG>(g, J, c, c.s + k, probes) : 0.0f;
        if (T == 1) {
          if (wt > 0.0f) pick = k;
        } else {
          const unsigned hit = __ballot_sync(kFull, wt > 0.0f);
          if (hit) pick = base + 31 - __clz(hit);
        }
      }
    }
  }
  if (COUNT) {
    lc.probes += probes;
    const int per = (FW_ALGO(J) == ALGO_NODE2VEC) ? (J.weighted ? 8 : 4) : (FW_ALGO(J) == ALGO_METAPATH ? (J.weighted ? 5 : 1) : (J.weighted ? 4 : 0));
    const int32_t mine = (lane < c.d) ? (c.d - lane + T - 1) / T : 0;
    lc.bytes += 2ull * mine * per + 32ull * probes;
  }
  return pick;
}

}  // namespace fw
