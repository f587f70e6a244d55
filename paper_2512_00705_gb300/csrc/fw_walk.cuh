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
//                   the result goes back to the owning lane.
//   * update        [Sec. 4.2, update()]: prev <- cur, cur <- next, row write.
// All loops are bounded (trial cap, degree, walk length); there are no waits.
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

// The walk loop of one warp over one queue: take walkers, plan, sample and
// write rows until the queue is exhausted and the warp holds no walker.
// `sj` (shared memory) is the queue's job table: its jobs' walkers form the
// index space [0, total), job j owning [sj[j].gbase, sj[j].gbase + W_j).
// ALG fixes the algorithm of every job at compile time.
template <bool COUNT, int ALG>
__device__ __forceinline__ void walk_loop(const DevGraph& g, const Job* sj, int njobs, long long total,
                                          unsigned long long* __restrict__ qctr, unsigned* __restrict__ err,
                                          int32_t* obuf, LaneCounters& lc) {
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
      if (pl == PLAN_EXACT_W) {
        const float u = u01(philox(make_uint4(w.wid, (uint32_t)w.step, 0u, 0u), JW.key0, JW.key1).x);
        k = exact_pick<32, COUNT, ALG>(g, JW, w, lane, u, lc);
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
// walk loop per warp over the launch's queue.
template <int NJ, bool COUNT, int ALG>
__global__ void __launch_bounds__(kBlock, kMinBlocks) walk_kernel(DevGraph g, JobTableN<NJ> tab, int njobs, long long total,
                                                      unsigned long long* __restrict__ qctr,
                                                      unsigned* __restrict__ err, DevCounters* __restrict__ cnt) {
  __shared__ Job sj[NJ];
  __shared__ int32_t obuf[kStageSlots * kBlock];
  load_jobs(tab.jobs, njobs, sj);
  __syncthreads();
  LaneCounters lc;
  lc.zero();
  walk_loop<COUNT, ALG>(g, sj, njobs, total, qctr, err, obuf, lc);
  if (COUNT) flush_counters(lc, cnt);
}

template <int NJ, bool COUNT, int ALG>
inline cudaError_t walk_blocks_per_sm(int* out) {
  static std::atomic<int> cached{0};
  int b = cached.load();
  if (b == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, walk_kernel<NJ, COUNT, ALG>, kBlock, 0);
    if (e != cudaSuccess) return e;
    b = b > 0 ? b : 1;
    cached.store(b);
  }
  *out = b;
  return cudaSuccess;
}

template <int NJ, bool COUNT, int ALG>
inline cudaError_t launch_walk_t(const fw_graph* g, const Job* jobs, int njobs, long long total,
                                 unsigned long long* qctr, cudaStream_t stream) {
  int blocks_per_sm = 1;
  cudaError_t oe = walk_blocks_per_sm<NJ, COUNT, ALG>(&blocks_per_sm);
  if (oe != cudaSuccess) return oe;
  JobTableN<NJ> tab;
  for (int i = 0; i < njobs; ++i) tab.jobs[i] = jobs[i];
  const long long want = (total + kBlock - 1) / kBlock;
  const long long cap = (long long)g->num_sms * blocks_per_sm;
  const int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
  walk_kernel<NJ, COUNT, ALG><<<grid, kBlock, 0, stream>>>(dev_graph(g), tab, njobs, total, qctr, g->d_err, g->d_cnt);
  g_launches.fetch_add(1);
  return cudaGetLastError();
}

}  // namespace fw
