/*
 * fw_oracle.c -- plain CPU oracle for the per-step transition sampling of
 * dynamic random walks (FlexiWalker, arXiv 2512.00705).
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg are the only users.  The GPU library neither
 * links nor calls this file, and the two share no code, header, table or
 * constant: the only common ground is the seeded input generator that feeds
 * both.  Nothing here is tuned for speed; every function follows a
 * definition from the paper, cited at the function.
 *
 * Compile with -ffp-contract=off: every FP32 product and sum below is one
 * IEEE-754 single-precision operation, rounded to nearest, in source order.
 *
 * Definitions followed:
 *   Eq. (prob), Sec. 2.1      w~(v,u) = w(v,u) * h(v,u);  p(u) = w~(v,u) / sum_t w~(v,t)
 *   Eq. (node2vec), Sec. 2.1  w = 1/a if dist(v',u)=0, 1 if dist(v',u)=1, 1/b if dist(v',u)=2
 *                             (the paper's a, b are node2vec's p, q)
 *   MetaPath, Sec. 2.1        w in {0,1}: 1 iff the edge label equals the schema entry of the step
 *   Eq. (2ndpr), Sec. 2.1     second-order PageRank: with max_d = max(d(v), d(v')),
 *                             w = ((1-g)/d(v) + g/d(v')) * max_d if dist(v',u) = 1,
 *                             else ((1-g)/d(v)) * max_d
 *   ITS, Sec. 2.2             one uniform, cumulative weights, first index whose cumulative
 *                             weight exceeds the scaled uniform
 *   RJS, Sec. 2.2 / 3.3       propose a neighbour uniformly, accept it iff U * B < w~, with the
 *                             bound B = max(w) * h_MAX[v]; repeat until a proposal is accepted
 *   Lemire, "Fast random integer generation in an interval", ACM TOMACS 29(1), 2019:
 *                             index floor(x * d / 2^32) of a 32-bit word x, rejected when the
 *                             low 32 bits of x * d fall below 2^32 mod d
 *   Sec. 3.3 (bound), Sec. 4.1 Eq. (runtime), Eq. (sum_estimation), Sec. 4.2 (sum helper):
 *                             B = max(w) * h_MAX[v]; sum-hat = h_SUM[v] * mean of the
 *                             distinct return values of w; eRJS iff r * B < sum-hat
 *   Philox4x32-10             Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 *                             as 1, 2, 3", SC'11.
 *   8-bit weights, Sec. 6.2   (an extension the paper names, not specified by it) symmetric
 *                             linear quantization with one scale per graph:
 *                             s = max h / 255, code = clamp(rint(h / s), 1, 255), h' = code * s
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - Hop 0 of node2vec has no previous node (vprev < 0): w = 1 for every
 *     neighbour.
 *   - dist(v',u) = 1 means u is in the out-adjacency of v' (graphs are symmetrised).
 *   - A walk of length L makes L hops; its row holds L+1 entries starting with
 *     the start node.  A walker whose current node has zero total transition
 *     weight (no neighbours, or no neighbour with a matching label) stops and
 *     the rest of its row is -1.
 *   - The metapath label required at hop j is schema[j mod S].
 *   - Second-order PageRank: u = v' (distance 0) takes the "otherwise" weight;
 *     hop 0 (no v') is a first-order step (w = 1).  FP32 recipe:
 *     t1 = (1 - g) / d(v), t2 = g / d(v'), m = max(d(v), d(v')),
 *     w = (t1 + t2) * m or t1 * m, each operation rounded once.
 *   - Exact-mode uniform: Philox4x32-10 with key = (seed low 32, seed high 32)
 *     and counter = (walker id, hop index, 0, 0); u = (x0 >> 8) * 2^-24.
 *   - Exact-mode pick: W_k = W_{k-1} + w~_k in FP32 in neighbour order,
 *     t = u * W_{d-1} in FP32, pick the smallest k with t < W_k; if rounding
 *     leaves none, pick the last k with w~_k > 0.
 *   - RJS random numbers: trial t of hop j of walker i draws
 *     x = Philox4x32-10(counter (i, j, 1, t), the exact-mode key); the proposal
 *     is Lemire's index of x0, or of x1 when x0 is rejected, and the trial
 *     proposes nothing when both are; U = (x2 >> 8) * 2^-24.  Trials run
 *     t = 0, 1, 2, ... and the first accepted proposal is the hop.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_WEIGHTED = 0, OR_NODE2VEC = 1, OR_METAPATH = 2, OR_PAGERANK2 = 3 };
enum { OR_MODE_RJS = 1, OR_MODE_RVS = 2 };

int or_step_plan(float hmax, float hsum, int32_t has_prev, int32_t dv, int32_t dprev, int32_t algo, float p,
                 float q, float gamma, float r, float *bound, float *sum_hat);

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon et al., SC'11): a 10-round Feistel-like bijection on
 * a 128-bit counter under a 64-bit key.  Round: two 32x32->64 multiplies by
 * the published constants, the high halves are XORed with the other two
 * counter words and the key; the key is bumped by the published Weyl
 * constants between rounds.
 * ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Exact-mode uniform for (seed, walker, hop): u in [0,1) on a 2^-24 grid. */
float or_exact_uniform(uint64_t seed, uint32_t walker, uint32_t hop) {
  uint32_t ctr[4] = {walker, hop, 0u, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  or_philox4x32_10(ctr, key, x);
  return (float)(x[0] >> 8) * 0x1.0p-24f;
}

/* The FP32 node2vec constants 1/p and 1/q: the reciprocal is taken in double
 * from the FP32 parameter and rounded once to FP32. */
float or_recip(float p) { return (float)(1.0 / (double)p); }

/* Is u an out-neighbour of x?  Rows are sorted ascending (checked by the
 * caller's input validation); bsearch is the C library's binary search. */
static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}
static int is_neighbour(const int32_t *offsets, const int32_t *cols, int32_t x, int32_t u) {
  int64_t s = offsets[x], e = offsets[x + 1];
  if (e <= s) return 0;
  return bsearch(&u, cols + s, (size_t)(e - s), sizeof(int32_t), cmp_i32) != NULL;
}

/*
 * Transition weights w~_k (FP32) of the d neighbours of v at hop `step`,
 * Eq. (prob) with w from Eq. (node2vec) or the MetaPath rule (Sec. 2.1).
 * h == NULL means h = 1 (the unweighted variants of Sec. 5.1).
 * vprev < 0 means there is no previous node (hop 0).
 * Returns d, or -1 on bad arguments.  wt may be NULL (degree query).
 */
int64_t or_transition_weights(const int32_t *offsets, const int32_t *cols, const float *h,
                              const uint8_t *labels, int32_t n, int32_t v, int32_t vprev,
                              int32_t step, int32_t algo, float p, float q, float gamma,
                              const uint8_t *schema, int32_t schema_len, float *wt) {
  if (!offsets || !cols || v < 0 || v >= n || vprev >= n || step < 0) return -1;
  if (algo == OR_NODE2VEC && !(p > 0 && q > 0 && isfinite(p) && isfinite(q))) return -1;
  if (algo == OR_METAPATH && (!labels || !schema || schema_len < 1)) return -1;
  if (algo == OR_PAGERANK2 && !(gamma >= 0.0f && gamma <= 1.0f)) return -1;
  if (algo != OR_WEIGHTED && algo != OR_NODE2VEC && algo != OR_METAPATH && algo != OR_PAGERANK2) return -1;
  const int64_t s = offsets[v], d = (int64_t)offsets[v + 1] - s;
  if (!wt) return d;
  const float inv_p = or_recip(p), inv_q = or_recip(q);
  float pr_w1 = 1.0f, pr_w2 = 1.0f; /* second-order PageRank weights of this step */
  if (algo == OR_PAGERANK2 && vprev >= 0) {
    const float dv = (float)d, dp = (float)(offsets[vprev + 1] - offsets[vprev]);
    const float t1 = (1.0f - gamma) / dv;
    const float t2 = gamma / dp;
    const float m = dv > dp ? dv : dp;
    pr_w1 = (t1 + t2) * m;
    pr_w2 = t1 * m;
  }
  for (int64_t k = 0; k < d; ++k) {
    const int32_t u = cols[s + k];
    const float hk = h ? h[s + k] : 1.0f;
    float w;
    if (algo == OR_WEIGHTED) {
      w = 1.0f;
    } else if (algo == OR_NODE2VEC) {
      if (vprev < 0) w = 1.0f;                                       /* reading: no v'     */
      else if (u == vprev) w = inv_p;                                /* dist(v',u) = 0     */
      else if (is_neighbour(offsets, cols, vprev, u)) w = 1.0f;      /* dist(v',u) = 1     */
      else w = inv_q;                                                /* dist(v',u) = 2     */
    } else if (algo == OR_PAGERANK2) {
      if (vprev < 0) w = 1.0f;                                       /* reading: no v'     */
      else w = is_neighbour(offsets, cols, vprev, u) ? pr_w1 : pr_w2; /* dist 1 / otherwise */
    } else {
      w = (labels[s + k] == schema[step % schema_len]) ? 1.0f : 0.0f;
    }
    wt[k] = w * hk; /* one FP32 multiply */
  }
  return d;
}

/* Exact transition probabilities (fp64), Eq. (prob).  All zero when the total
 * weight is zero (a dead end).  Returns d or -1. */
int64_t or_transition_probs(const int32_t *offsets, const int32_t *cols, const float *h,
                            const uint8_t *labels, int32_t n, int32_t v, int32_t vprev,
                            int32_t step, int32_t algo, float p, float q, float gamma,
                            const uint8_t *schema, int32_t schema_len, double *probs) {
  int64_t d = or_transition_weights(offsets, cols, h, labels, n, v, vprev, step, algo, p, q, gamma,
                                    schema, schema_len, NULL);
  if (d < 0 || !probs) return d;
  float *wt = (float *)malloc((size_t)(d > 0 ? d : 1) * sizeof(float));
  if (!wt) return -1;
  or_transition_weights(offsets, cols, h, labels, n, v, vprev, step, algo, p, q, gamma, schema,
                        schema_len, wt);
  double total = 0.0;
  for (int64_t k = 0; k < d; ++k) total += (double)wt[k];
  for (int64_t k = 0; k < d; ++k) probs[k] = total > 0.0 ? (double)wt[k] / total : 0.0;
  free(wt);
  return d;
}

/* Inverse-transform pick (Sec. 2.2, ITS) over FP32 weights with one uniform
 * u in [0,1).  Returns the chosen index, or -1 when the total is zero. */
int64_t or_icdf_pick(const float *wt, int64_t d, float u) {
  float total = 0.0f;
  for (int64_t k = 0; k < d; ++k) total = total + wt[k];
  if (!(total > 0.0f)) return -1;
  const float t = u * total;
  float run = 0.0f;
  for (int64_t k = 0; k < d; ++k) {
    run = run + wt[k];
    if (t < run) return k;
  }
  for (int64_t k = d - 1; k >= 0; --k)
    if (wt[k] > 0.0f) return k;
  return -1;
}

/*
 * Full walks in exact mode.  out is row-major [W][L+1]; row i starts with
 * starts[i].  The walker id used by the random stream is walker_base + i.
 * Returns the number of hops taken (entries other than the start and -1),
 * or -1 on bad arguments.
 */
static int64_t walk_impl(const int32_t *offsets, const int32_t *cols, const float *h,
                         const uint8_t *labels, int32_t n, const int32_t *starts, int32_t num_walkers,
                         int32_t len, int32_t algo, float p, float q, float gamma, const uint8_t *schema,
                         int32_t schema_len, uint64_t seed, uint32_t walker_base, const uint32_t *ids,
                         int32_t sampler, int32_t *out, int32_t nthreads, int64_t *trials_out);

int64_t or_walk(const int32_t *offsets, const int32_t *cols, const float *h,
                const uint8_t *labels, int32_t n, const int32_t *starts, int32_t num_walkers,
                int32_t len, int32_t algo, float p, float q, float gamma, const uint8_t *schema,
                int32_t schema_len, uint64_t seed, uint32_t walker_base, int32_t *out,
                int32_t nthreads) {
  return walk_impl(offsets, cols, h, labels, n, starts, num_walkers, len, algo, p, q, gamma, schema, schema_len,
                   seed, walker_base, NULL, 0, out, nthreads, NULL);
}

/* Same walks with an explicit random-stream id per walker (ids[i] instead
 * of walker_base + i); ids are inputs, no arithmetic changes. */
int64_t or_walk_ids(const int32_t *offsets, const int32_t *cols, const float *h,
                    const uint8_t *labels, int32_t n, const int32_t *starts, const uint32_t *ids,
                    int32_t num_walkers, int32_t len, int32_t algo, float p, float q, float gamma,
                    const uint8_t *schema, int32_t schema_len, uint64_t seed, int32_t *out,
                    int32_t nthreads) {
  if (!ids && num_walkers > 0) return -1;
  return walk_impl(offsets, cols, h, labels, n, starts, num_walkers, len, algo, p, q, gamma, schema, schema_len,
                   seed, 0, ids, 0, out, nthreads, NULL);
}

/* The same walks with every hop drawn by rejection sampling (RJS, Sec. 3.3)
 * against the bound B = max(w) * h_MAX[v] of or_step_plan, with the random
 * numbers of the RJS reading in the header.  Rows follow the same
 * distribution as or_walk's; they are not the same rows.
 *
 * envelope 0: the paper's proposal, one of the d neighbours uniformly, each
 * bounded by B.  envelope 1 for metapath (a data layout, not in the paper):
 * only the entries whose label the hop requires are proposed, M being their
 * largest h; class c < 4 holds h in (M/2^(c+1), M/2^c], class 4 the rest; the
 * entries are read in class order (row order inside a class), a trial draws
 * one of 16 n0 + 8 n1 + 4 n2 + 2 n3 + n4 slots (slot t naming entry t/16 of
 * class 0, and so on) and accepts iff U * M/2^c < h; no such entry: a dead
 * end.  envelope 1 otherwise (weighted graphs; a refinement of the Sec. 3.3
 * bound, not in the paper): the neighbours fall into weight classes,
 * class 0 with h > h_MAX/2, class 1 with h_MAX/4 < h <= h_MAX/2, class 2 the
 * rest, of n0, n1, n2 entries, bounded by B, B/2 and B/4; the row is read in
 * class order (class 0 entries in row order, then class 1, then class 2) and
 * a trial draws one of 4 n0 + 2 n1 + n2 slots, slot t naming entry t/4 of
 * class 0, then (t - 4 n0)/2 of class 1, then t - 4 n0 - 2 n1 of class 2;
 * it is accepted iff U * (bound of its class) < w~.  Each entry is proposed
 * in proportion to its class bound, which is at least its w~, so accepted
 * draws follow Eq. (prob) as with the single bound.  trials_out (may be
 * NULL) receives the number of trials of all hops, void ones included. */
int64_t or_walk_rjs(const int32_t *offsets, const int32_t *cols, const float *h, const uint8_t *labels, int32_t n,
                    const int32_t *starts, int32_t num_walkers, int32_t len, int32_t algo, float p, float q,
                    float gamma, const uint8_t *schema, int32_t schema_len, uint64_t seed, uint32_t walker_base,
                    int32_t envelope, int32_t *out, int32_t nthreads, int64_t *trials_out) {
  if (envelope != 0 && envelope != 1) return -1;
  if (envelope == 1 && algo != OR_METAPATH && !h) return -1;
  return walk_impl(offsets, cols, h, labels, n, starts, num_walkers, len, algo, p, q, gamma, schema, schema_len,
                   seed, walker_base, NULL, 1 + envelope, out, nthreads, trials_out);
}

/* Lemire's map of a 32-bit word onto [0, d), d >= 1: *k = floor(x * d / 2^32)
 * unless the low word of x * d is below 2^32 mod d (then 0 is returned and
 * the word is not used); the accepted words give every index equally often. */
static int lemire_index(uint32_t x, uint32_t d, uint32_t *k) {
  const uint64_t m = (uint64_t)x * (uint64_t)d;
  const uint32_t low = (uint32_t)m;
  const uint32_t thr = (uint32_t)((UINT64_C(0x100000000) - d) % d); /* 2^32 mod d */
  if (low < thr) return 0;
  *k = (uint32_t)(m >> 32);
  return 1;
}

/* One RJS hop at v with FP32 weights wt[0..d) and bound B (Sec. 3.3): trials
 * t = 0, 1, ... until U * bound < wt[k] for the proposed k.  With hrow (the
 * row's h, envelope 1 of or_walk_rjs) the proposal follows the weight-class
 * slots, ord[] receiving the class order.  Returns k, or -1 when no
 * neighbour has weight (the proposal would never be accepted). */
static int64_t rjs_pick(const float *wt, int64_t d, float B, const float *hrow, float hmax, int32_t *ord,
                        uint64_t seed, uint32_t wid, uint32_t hop, int64_t *trials) {
  int any = 0;
  for (int64_t k = 0; k < d; ++k) any |= wt[k] > 0.0f;
  if (!any) return -1;
  uint32_t n0 = 0, n1 = 0, slots = (uint32_t)d;
  if (hrow) {
    const float half = 0.5f * hmax, quarter = 0.25f * hmax;
    uint32_t m = 0;
    for (int c = 0; c < 3; ++c) {
      for (int64_t k = 0; k < d; ++k) {
        const int ck = hrow[k] > half ? 0 : (hrow[k] > quarter ? 1 : 2);
        if (ck == c) ord[m++] = (int32_t)k;
      }
      if (c == 0) n0 = m;
      if (c == 1) n1 = m - n0;
    }
    slots = 4u * n0 + 2u * n1 + ((uint32_t)d - n0 - n1);
  }
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t t = 0;; ++t) {
    const uint32_t ctr[4] = {wid, hop, 1u, t};
    uint32_t x[4], sl;
    or_philox4x32_10(ctr, key, x);
    ++*trials;
    if (!lemire_index(x[0], slots, &sl) && !lemire_index(x[1], slots, &sl)) continue;
    int64_t k = sl;
    float bound = B;
    if (hrow) {
      if (sl < 4u * n0) {
        k = ord[sl / 4u];
      } else if (sl - 4u * n0 < 2u * n1) {
        k = ord[n0 + (sl - 4u * n0) / 2u];
        bound = 0.5f * B;
      } else {
        k = ord[n0 + n1 + (sl - 4u * n0 - 2u * n1)];
        bound = 0.25f * B;
      }
    }
    const float U = (float)(x[2] >> 8) * 0x1.0p-24f;
    if (U * bound < wt[k]) return k;
  }
}

/* One RJS hop of a metapath walk under the label-segment envelope of
 * or_walk_rjs (envelope 1): entries of label `want` among the d of the row
 * (labrow, hrow; hrow NULL: h = 1).  Returns the row position, or -1 when
 * no entry has the label. */
static int64_t rjs_pick_label(const float *hrow, const uint8_t *labrow, uint8_t want, int64_t d, int32_t *ord,
                              uint64_t seed, uint32_t wid, uint32_t hop, int64_t *trials) {
  float M = 0.0f;
  for (int64_t k = 0; k < d; ++k) {
    const float x = hrow ? hrow[k] : 1.0f;
    if (labrow[k] == want && x > M) M = x;
  }
  if (!(M > 0.0f)) return -1;
  uint32_t cnt[5] = {0, 0, 0, 0, 0}, m = 0;
  for (int c = 0; c < 5; ++c) {
    for (int64_t k = 0; k < d; ++k) {
      if (labrow[k] != want) continue;
      const float x = hrow ? hrow[k] : 1.0f;
      int ck = 0;
      float t = 0.5f * M;
      while (ck < 4 && !(x > t)) {
        ++ck;
        t = 0.5f * t;
      }
      if (ck == c) {
        ord[m++] = (int32_t)k;
        cnt[c]++;
      }
    }
  }
  uint32_t slots = 0;
  for (int c = 0; c < 5; ++c) slots += (16u >> c) * cnt[c];
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t t = 0;; ++t) {
    const uint32_t ctr[4] = {wid, hop, 1u, t};
    uint32_t x[4], sl;
    or_philox4x32_10(ctr, key, x);
    ++*trials;
    if (!lemire_index(x[0], slots, &sl) && !lemire_index(x[1], slots, &sl)) continue;
    uint32_t base = 0;
    int c = 0;
    float bound = M;
    while (sl >= (16u >> c) * cnt[c]) {
      sl -= (16u >> c) * cnt[c];
      base += cnt[c];
      ++c;
      bound = 0.5f * bound;
    }
    const int64_t k = ord[base + sl / (16u >> c)];
    const float U = (float)(x[2] >> 8) * 0x1.0p-24f;
    if (U * bound < (hrow ? hrow[k] : 1.0f)) return k;
  }
}

static int64_t walk_impl(const int32_t *offsets, const int32_t *cols, const float *h,
                         const uint8_t *labels, int32_t n, const int32_t *starts, int32_t num_walkers,
                         int32_t len, int32_t algo, float p, float q, float gamma, const uint8_t *schema,
                         int32_t schema_len, uint64_t seed, uint32_t walker_base, const uint32_t *ids,
                         int32_t sampler, int32_t *out, int32_t nthreads, int64_t *trials_out) {
  if (!offsets || !cols || !starts || !out || num_walkers < 0 || len < 0 || n < 0) return -1;
  for (int32_t i = 0; i < num_walkers; ++i)
    if (starts[i] < 0 || starts[i] >= n) return -1;
  if (algo == OR_NODE2VEC && !(p > 0 && q > 0 && isfinite(p) && isfinite(q))) return -1;
  if (algo == OR_METAPATH && (!labels || !schema || schema_len < 1)) return -1;
  if (algo == OR_PAGERANK2 && !(gamma >= 0.0f && gamma <= 1.0f)) return -1;
  int32_t maxd = 0;
  for (int32_t v = 0; v < n; ++v)
    if (offsets[v + 1] - offsets[v] > maxd) maxd = offsets[v + 1] - offsets[v];
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  int64_t hops = 0, trials = 0;
  int failed = 0;
#pragma omp parallel reduction(+ : hops, trials)
  {
    float *wt = (float *)malloc((size_t)(maxd > 0 ? maxd : 1) * sizeof(float));
    int32_t *ord = (int32_t *)malloc((size_t)(maxd > 0 ? maxd : 1) * sizeof(int32_t));
    if (!wt || !ord) {
#pragma omp atomic write
      failed = 1;
    }
#pragma omp for schedule(dynamic, 64)
    for (int32_t i = 0; i < num_walkers; ++i) {
      if (!wt || !ord) continue;
      int32_t *row = out + (int64_t)i * (len + 1);
      int32_t cur = starts[i], prev = -1;
      row[0] = cur;
      int32_t j = 0;
      for (; j < len; ++j) {
        int64_t d = or_transition_weights(offsets, cols, h, labels, n, cur, prev, j, algo, p, q, gamma,
                                          schema, schema_len, wt);
        const uint32_t wid = ids ? ids[i] : walker_base + (uint32_t)i;
        int64_t k;
        if (sampler == 0) {
          k = or_icdf_pick(wt, d, or_exact_uniform(seed, wid, (uint32_t)j));
        } else if (sampler == 2 && algo == OR_METAPATH) {
          k = rjs_pick_label(h ? h + offsets[cur] : NULL, labels + offsets[cur], schema[j % schema_len], d, ord, seed,
                             wid, (uint32_t)j, &trials);
        } else {
          float hmax = 0.0f, B;
          for (int64_t e = offsets[cur]; e < offsets[cur + 1]; ++e) {
            const float x = h ? h[e] : 1.0f;
            if (x > hmax) hmax = x;
          }
          const int32_t dprev = prev >= 0 ? offsets[prev + 1] - offsets[prev] : 0;
          if (d == 0 || or_step_plan(hmax, 0.0f, prev >= 0, (int32_t)d, dprev, algo, p, q, gamma, 1.0f, &B, NULL) < 0)
            break;
          k = rjs_pick(wt, d, B, sampler == 2 ? h + offsets[cur] : NULL, hmax, ord, seed, wid, (uint32_t)j, &trials);
        }
        if (k < 0) break;
        int32_t nxt = cols[offsets[cur] + k];
        row[j + 1] = nxt;
        prev = cur;
        cur = nxt;
        hops++;
      }
      for (int32_t r = j + 1; r <= len; ++r) row[r] = -1;
    }
    free(wt);
    free(ord);
  }
  if (trials_out) *trials_out = trials;
  return failed ? -1 : hops;
}

/* Per-node reductions of the property weights (Sec. 4.2, preprocess()):
 * h_MAX[v] = max_k h (FP32, exact), h_SUM[v] = sum_k h in fp64.  h == NULL
 * means h = 1.  Nodes without neighbours get 0 for both. */
int or_node_stats(const int32_t *offsets, const float *h, int32_t n, float *hmax, double *hsum) {
  if (!offsets || n < 0 || !hmax || !hsum) return -1;
  for (int32_t v = 0; v < n; ++v) {
    float m = 0.0f;
    double s = 0.0;
    for (int64_t i = offsets[v]; i < offsets[v + 1]; ++i) {
      float x = h ? h[i] : 1.0f;
      if (x > m) m = x;
      s += (double)x;
    }
    hmax[v] = m;
    hsum[v] = s;
  }
  return 0;
}

/*
 * The per-step plan of the runtime (Sec. 3.3 bound, Sec. 4.1 cost model,
 * Sec. 4.2 helper functions), for one walker at v of degree dv with
 * previous node of degree dprev (has_prev = 0 when there is no previous
 * node, i.e. on hop 0):
 *   B       = max(w) * h_MAX[v]        (FP32 product; max(w) of the algorithm)
 *   sum_hat = h_SUM[v] * mean_w        (FP32 product; mean of the distinct return
 *                                       expressions of get_weight, Eq. (sum_estimation))
 *   mode    = eRJS iff r * B < sum_hat (FP32), else eRVS   (Eq. (runtime))
 * Distinct return expressions: node2vec {h/a, h, h/b} (3; without v': {h}),
 * metapath {h, 0} (2), weighted {h} (1), second-order PageRank {w1 h, w2 h}
 * (2; without v': {h}).  The node2vec mean is taken in double and rounded
 * once to FP32; the PageRank one is (w1 + w2) * 0.5 in FP32.  With h = 1
 * (unweighted) h_MAX = 1 and h_SUM = d(v), which is the paper's PER_KERNEL
 * rule (mean times degree).
 */
int or_step_plan(float hmax, float hsum, int32_t has_prev, int32_t dv, int32_t dprev, int32_t algo, float p,
                 float q, float gamma, float r, float *bound, float *sum_hat) {
  float wmax, wmean;
  if (algo == OR_NODE2VEC) {
    if (!(p > 0 && q > 0)) return -1;
    const float ip = or_recip(p), iq = or_recip(q);
    if (!has_prev) {
      wmax = 1.0f;
      wmean = 1.0f;
    } else {
      wmax = ip > 1.0f ? ip : 1.0f;
      if (iq > wmax) wmax = iq;
      wmean = (float)(((double)ip + 1.0 + (double)iq) / 3.0);
    }
  } else if (algo == OR_PAGERANK2) {
    if (!has_prev) {
      wmax = 1.0f;
      wmean = 1.0f;
    } else {
      if (dv < 1 || dprev < 1) return -1;
      const float fv = (float)dv, fp = (float)dprev;
      const float t1 = (1.0f - gamma) / fv;
      const float t2 = gamma / fp;
      const float m = fv > fp ? fv : fp;
      const float w1 = (t1 + t2) * m, w2 = t1 * m;
      wmax = w1;
      wmean = (w1 + w2) * 0.5f;
    }
  } else if (algo == OR_METAPATH) {
    wmax = 1.0f;
    wmean = 0.5f;
  } else if (algo == OR_WEIGHTED) {
    wmax = 1.0f;
    wmean = 1.0f;
  } else {
    return -1;
  }
  const float B = wmax * hmax;
  const float S = hsum * wmean;
  if (bound) *bound = B;
  if (sum_hat) *sum_hat = S;
  return (r * B < S) ? OR_MODE_RJS : OR_MODE_RVS;
}

/* Per-label node statistics (the Sec. 4.2 preprocessing of h restricted to
 * the edges of one label): for node v and label l in [0, 8), the maximum
 * (FP32, exact) and the sum (fp64) of h over the edges of v labelled l;
 * h == NULL means h = 1.  Returns -1 if a label >= 8 occurs. */
int or_label_stats(const int32_t *offsets, const float *h, const uint8_t *labels, int32_t n, float *lmax,
                   double *lsum) {
  if (!offsets || !labels || n < 0 || !lmax || !lsum) return -1;
  for (int32_t v = 0; v < n; ++v) {
    for (int l = 0; l < 8; ++l) {
      lmax[v * 8 + l] = 0.0f;
      lsum[v * 8 + l] = 0.0;
    }
    for (int64_t i = offsets[v]; i < offsets[v + 1]; ++i) {
      const int l = labels[i];
      if (l >= 8) return -1;
      const float x = h ? h[i] : 1.0f;
      if (x > lmax[v * 8 + l]) lmax[v * 8 + l] = x;
      lsum[v * 8 + l] += (double)x;
    }
  }
  return 0;
}

/* 8-bit property weights (Sec. 6.2 names low-precision weights as an
 * extension; the format is this reading): one FP32 scale per node, from the
 * node's own row, s_v = (max over the row of v of h) / 255; each weight
 * h(v,u) is stored as the nearest integer multiple of s_v (ties to even),
 * kept within 1..255 so that no edge loses its weight, and read back as
 * code * s_v.  Every row's largest weight gets code 255, so every row keeps
 * its distribution to within half a code step of its own maximum.  FP32
 * throughout, each operation rounded once.  codes / scales / hq may be NULL;
 * rows without entries get scale 0.  Returns 0, or -1 on bad arguments. */
int or_quantize_weights(const int32_t *offsets, int32_t n, const float *h, uint8_t *codes, float *scales,
                        float *hq) {
  if (!offsets || n < 0 || (!h && offsets[n] > 0)) return -1;
  for (int32_t v = 0; v < n; ++v) {
    float row_max = 0.0f;
    for (int64_t i = offsets[v]; i < offsets[v + 1]; ++i)
      if (h[i] > row_max) row_max = h[i];
    const float s = row_max / 255.0f;
    if (scales) scales[v] = s;
    for (int64_t i = offsets[v]; i < offsets[v + 1]; ++i) {
      float c = rintf(h[i] / s);
      if (c < 1.0f) c = 1.0f;
      if (c > 255.0f) c = 255.0f;
      if (codes) codes[i] = (uint8_t)c;
      if (hq) hq[i] = c * s;
    }
  }
  return 0;
}
