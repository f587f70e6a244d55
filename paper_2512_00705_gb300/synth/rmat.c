/*
 * Seeded synthetic inputs for dynamic random walks: R-MAT graphs in sorted,
 * symmetric int32 CSR form, plus per-undirected-edge property weights h and
 * edge labels.
 *
 * This file holds input generation only.  It contains none of the walk
 * method's arithmetic (no transition weights, no sampling); both the CPU
 * oracle's tests and the GPU path's tests and benchmark draw their inputs
 * from here.
 *
 * R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004), Graph500 style: every edge
 * picks one of four quadrants per recursion level with probabilities
 * (a, b, c, 1-a-b-c); no noise.  Vertex ids are then relabelled by a seeded
 * random permutation (optional), the edge list is symmetrised, self-loops and
 * duplicate edges are removed and every row is sorted ascending.
 *
 * Every random draw is a pure function of (seed, index) through the
 * SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014), so the output does
 * not depend on the number of threads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN64 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z += GOLDEN64;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* uniform in [0,1) with 53 bits */
static inline double u53(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

typedef struct {
  int32_t n;
  int64_t e;
  int32_t *offsets; /* n+1 */
  int32_t *cols;    /* e   */
} fws_graph;

static int set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

static int cmp_i32(const void *x, const void *y) {
  int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
  return (a > b) - (a < b);
}

/* LSD radix sort of non-negative int32 keys (used for long rows). */
static void radix_sort_u32(uint32_t *k, uint32_t *tmp, int64_t n) {
  int64_t cnt[256];
  for (int pass = 0; pass < 4; ++pass) {
    int sh = pass * 8;
    memset(cnt, 0, sizeof(cnt));
    for (int64_t i = 0; i < n; ++i) cnt[(k[i] >> sh) & 255]++;
    int64_t s = 0;
    for (int b = 0; b < 256; ++b) { int64_t c = cnt[b]; cnt[b] = s; s += c; }
    for (int64_t i = 0; i < n; ++i) tmp[cnt[(k[i] >> sh) & 255]++] = k[i];
    memcpy(k, tmp, (size_t)n * sizeof(uint32_t));
  }
}

/*
 * Build a symmetric R-MAT graph with 2^scale vertices and edge_factor*2^scale
 * generated (directed) edges before symmetrisation.
 * Returns 0 on success, -1 on bad arguments, -2 on allocation failure,
 * -3 if the symmetrised edge count does not fit int32 offsets.
 */
int fws_rmat_build(int32_t scale, int32_t edge_factor, double a, double b, double c,
                   uint64_t seed, int32_t permute, int32_t nthreads, void **handle,
                   int32_t *n_out, int64_t *e_out) {
  if (scale < 1 || scale > 30 || edge_factor < 1 || a < 0 || b < 0 || c < 0 ||
      a + b + c > 1.0 || !handle)
    return -1;
  set_threads(nthreads);
  const int64_t n = (int64_t)1 << scale;
  const int64_t m = (int64_t)edge_factor * n;
  const double ab = a + b, abc = a + b + c;

  int32_t *src = (int32_t *)malloc((size_t)m * sizeof(int32_t));
  int32_t *dst = (int32_t *)malloc((size_t)m * sizeof(int32_t));
  int32_t *perm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!src || !dst || !perm) { free(src); free(dst); free(perm); return -2; }

  /* 1. quadrant recursion per edge */
  const uint64_t gseed = mix64(seed ^ 0x52A7C0DEULL);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    uint64_t st = mix64(gseed + (uint64_t)i * GOLDEN64);
    int64_t r = 0, cc = 0;
    for (int lvl = 0; lvl < scale; ++lvl) {
      if (lvl > 0 && (lvl & 1) == 0) st = mix64(st);
      uint32_t bits = (lvl & 1) ? (uint32_t)(st >> 32) : (uint32_t)st;
      double u = (double)bits * 0x1.0p-32;
      int rb, cb;
      if (u < a) { rb = 0; cb = 0; }
      else if (u < ab) { rb = 0; cb = 1; }
      else if (u < abc) { rb = 1; cb = 0; }
      else { rb = 1; cb = 1; }
      r = (r << 1) | rb;
      cc = (cc << 1) | cb;
    }
    src[i] = (int32_t)r;
    dst[i] = (int32_t)cc;
  }

  /* 2. seeded vertex permutation (Fisher-Yates) */
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  if (permute) {
    uint64_t ps = mix64(seed ^ 0x9E12A5E7ULL);
    for (int64_t i = n - 1; i > 0; --i) {
      ps = mix64(ps);
      int64_t j = (int64_t)(u53(ps) * (double)(i + 1));
      if (j > i) j = i;
      int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
  }

  /* 3. degrees of the symmetrised multigraph without self-loops */
  int64_t *rowstart = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t *cursor = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  if (!rowstart || !cursor) { free(src); free(dst); free(perm); free(rowstart); free(cursor); return -2; }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    int32_t u = perm[src[i]], v = perm[dst[i]];
    src[i] = u; dst[i] = v;
    if (u != v) {
#pragma omp atomic
      rowstart[u + 1]++;
#pragma omp atomic
      rowstart[v + 1]++;
    }
  }
  free(perm);
  for (int64_t i = 0; i < n; ++i) rowstart[i + 1] += rowstart[i];
  const int64_t m2 = rowstart[n];
  int32_t *tmp = (int32_t *)malloc((size_t)(m2 > 0 ? m2 : 1) * sizeof(int32_t));
  if (!tmp) { free(src); free(dst); free(rowstart); free(cursor); return -2; }
  memcpy(cursor, rowstart, (size_t)n * sizeof(int64_t));

  /* 4. scatter both directions */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    int32_t u = src[i], v = dst[i];
    if (u == v) continue;
    int64_t pu, pv;
#pragma omp atomic capture
    pu = cursor[u]++;
#pragma omp atomic capture
    pv = cursor[v]++;
    tmp[pu] = v;
    tmp[pv] = u;
  }
  free(src);
  free(dst);

  /* 5. sort + dedupe every row in place; cursor[v] := deduped degree */
#pragma omp parallel
  {
    uint32_t *scratch = NULL;
    int64_t scap = 0;
#pragma omp for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; ++v) {
      int64_t s = rowstart[v], len = rowstart[v + 1] - s;
      int32_t *row = tmp + s;
      if (len > 4096) {
        if (len > scap) { free(scratch); scap = len; scratch = (uint32_t *)malloc((size_t)scap * 4); }
        radix_sort_u32((uint32_t *)row, scratch, len);
      } else if (len > 1) {
        qsort(row, (size_t)len, sizeof(int32_t), cmp_i32);
      }
      int64_t k = 0;
      for (int64_t i = 0; i < len; ++i)
        if (k == 0 || row[i] != row[k - 1]) row[k++] = row[i];
      cursor[v] = k;
    }
    free(scratch);
  }

  /* 6. compact */
  int64_t total = 0;
  for (int64_t v = 0; v < n; ++v) total += cursor[v];
  if (total > 2147483647LL) { free(tmp); free(rowstart); free(cursor); return -3; }
  fws_graph *g = (fws_graph *)calloc(1, sizeof(fws_graph));
  if (!g) { free(tmp); free(rowstart); free(cursor); return -2; }
  g->n = (int32_t)n;
  g->e = total;
  g->offsets = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
  g->cols = (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  if (!g->offsets || !g->cols) {
    free(g->offsets); free(g->cols); free(g); free(tmp); free(rowstart); free(cursor);
    return -2;
  }
  int64_t acc = 0;
  for (int64_t v = 0; v < n; ++v) { g->offsets[v] = (int32_t)acc; acc += cursor[v]; }
  g->offsets[n] = (int32_t)acc;
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t v = 0; v < n; ++v)
    memcpy(g->cols + g->offsets[v], tmp + rowstart[v], (size_t)cursor[v] * sizeof(int32_t));
  free(tmp);
  free(rowstart);
  free(cursor);
  *handle = g;
  if (n_out) *n_out = g->n;
  if (e_out) *e_out = g->e;
  return 0;
}

int fws_rmat_copy(void *handle, int32_t *offsets, int32_t *cols) {
  fws_graph *g = (fws_graph *)handle;
  if (!g || !offsets || !cols) return -1;
  memcpy(offsets, g->offsets, (size_t)(g->n + 1) * sizeof(int32_t));
  memcpy(cols, g->cols, (size_t)g->e * sizeof(int32_t));
  return 0;
}

void fws_rmat_free(void *handle) {
  fws_graph *g = (fws_graph *)handle;
  if (!g) return;
  free(g->offsets);
  free(g->cols);
  free(g);
}

/* Key of the undirected edge {u, v}: identical for (u,v) and (v,u). */
static inline uint64_t undirected_key(int32_t u, int32_t v, uint64_t seed) {
  uint32_t lo = (uint32_t)(u < v ? u : v), hi = (uint32_t)(u < v ? v : u);
  return mix64(seed ^ mix64(((uint64_t)lo << 32) | hi));
}

enum {
  FWS_W_UNIFORM01 = 0,  /* h = 1 - U, U ~ U[0,1) on a 2^-24 grid: h in (0,1]   */
  FWS_W_LOGNORMAL = 1,  /* h = exp(sigma * Z), Z ~ N(0,1) by Box-Muller      */
  FWS_W_PARETO = 2,     /* h = (1-U)^(-1/alpha): classical Pareto, x_m = 1    */
  FWS_W_UNIFORM15 = 3,  /* h = 1 + 4U on a 2^-24 grid: h in [1,5)             */
};

/*
 * Fill h[e] for every CSR entry, one value per undirected edge (mirrored
 * entries get the same value).  Returns 0, or -1 on bad arguments.
 */
int fws_edge_weights(const int32_t *offsets, const int32_t *cols, int32_t n, int32_t kind,
                     double param, uint64_t seed, float *out, int32_t nthreads) {
  if (!offsets || !cols || !out || n < 0) return -1;
  if (kind == FWS_W_PARETO && !(param > 0)) return -1;
  set_threads(nthreads);
  const uint64_t s = mix64(seed ^ 0x57E16A7ULL);
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t v = 0; v < n; ++v) {
    for (int64_t i = offsets[v]; i < offsets[v + 1]; ++i) {
      uint64_t k = undirected_key((int32_t)v, cols[i], s);
      float h;
      if (kind == FWS_W_UNIFORM01) {
        h = 1.0f - (float)(k >> 40) * 0x1.0p-24f;
      } else if (kind == FWS_W_UNIFORM15) {
        h = 1.0f + 4.0f * ((float)(k >> 40) * 0x1.0p-24f);
      } else if (kind == FWS_W_LOGNORMAL) {
        double u1 = 1.0 - u53(k);             /* (0,1] */
        double u2 = u53(mix64(k ^ 0xB0C5ULL)); /* [0,1) */
        double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
        h = (float)exp(param * z);
        if (!(h > 0.0f)) h = 0x1.0p-126f;
      } else if (kind == FWS_W_PARETO) {
        double u = u53(k); /* [0,1) */
        h = (float)pow(1.0 - u, -1.0 / param);
        if (!(h < 3.0e38f)) h = 3.0e38f;
      } else {
        h = 1.0f;
      }
      out[i] = h;
    }
  }
  return 0;
}

/* Fill labels[e] uniform in {0..nlabels-1}, one value per undirected edge. */
int fws_edge_labels(const int32_t *offsets, const int32_t *cols, int32_t n, int32_t nlabels,
                    uint64_t seed, uint8_t *out, int32_t nthreads) {
  if (!offsets || !cols || !out || n < 0 || nlabels < 1 || nlabels > 256) return -1;
  set_threads(nthreads);
  const uint64_t s = mix64(seed ^ 0x1AB31ULL);
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t v = 0; v < n; ++v)
    for (int64_t i = offsets[v]; i < offsets[v + 1]; ++i) {
      uint64_t k = undirected_key((int32_t)v, cols[i], s);
      out[i] = (uint8_t)(((k >> 32) * (uint64_t)nlabels) >> 32);
    }
  return 0;
}
