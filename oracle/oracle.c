/*
 * oracle.c -- plain, slow, CPU reference of exact k-NN search over iSAX-summarised,
 * z-normalised data series (MESSI, Peng, Fatourou, Palpanas).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or load this
 * file: only the tests, the smoke check and the benchmark's CPU-baseline leg do.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Precision: distances, lower bounds and breakpoints are computed in FP64 (long
 * double for the breakpoint search). The summarisation (z-normalisation, PAA) is
 * computed in the single-precision arithmetic the GPU kernels use, in the fixed
 * order spelled out below, because the SAX symbols are integers decided by those
 * fp32 values and must agree bit for bit; every operation is one IEEE-754 rounding
 * (built with -ffp-contract=off; fmaf is a single rounding by definition).
 *
 * Canonical fp32 order (the "lane" of point t is (t/4) mod 32):
 *   S1   : 32 lane partials, each summing its points in increasing t, combined by
 *          a pairwise tree in lane order ((a0+a1)+(a2+a3))+... ;
 *   mu   = S1 / n;   V: same layout over fmaf(d, d, acc) with d = x_t - mu;
 *   sigma= sqrt(V / n); constant series (sigma < 1e-30 or sigma <= 1e-6 |mu|) -> z = 0;
 *   z_t  = (x_t - mu) * (1 / sigma);
 *   PAA_j: if s = n/w is 4 * 2^m, groups of 4 consecutive points summed in order,
 *          the groups combined by a pairwise tree in group order; otherwise a
 *          sequential sum; then divided by s.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ breakpoints
 * iSAX divides the value axis into c regions (Section II-B); following the iSAX
 * papers it builds on, the regions are equiprobable under N(0,1):
 * beta_i = Phi^{-1}(i/c), i = 1..c-1. Phi^{-1} by bisection on
 * Phi(x) = erfc(-x / sqrt 2) / 2 in long double, to the last bit. */
static long double orc_phi(long double x) { return 0.5L * erfcl(-x / sqrtl(2.0L)); }

static long double orc_phi_inv(long double p) {
  long double lo = -40.0L, hi = 40.0L;
  for (int it = 0; it < 400; ++it) {
    long double mid = 0.5L * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (orc_phi(mid) < p) lo = mid; else hi = mid;
  }
  return 0.5L * (lo + hi);
}

/* beta[0..c-2] = Phi^{-1}(i/c), i = 1..c-1 (as double). The middle breakpoint of an
 * even cardinality is exactly 0 by symmetry. */
void orc_breakpoints(int32_t c, double* beta) {
  for (int32_t i = 1; i < c; ++i) {
    if (2 * i == c) { beta[i - 1] = 0.0; continue; }
    beta[i - 1] = (double)orc_phi_inv((long double)i / (long double)c);
  }
}

/* t[0..c-2]: smallest fp32 value >= beta_i, so that for any fp32 value p,
 * p >= t_i exactly when p >= beta_i. */
void orc_thresholds(int32_t c, float* t) {
  for (int32_t i = 1; i < c; ++i) {
    long double b = (2 * i == c) ? 0.0L : orc_phi_inv((long double)i / (long double)c);
    float f = (float)b;
    while ((long double)f < b) f = nextafterf(f, INFINITY);
    while ((long double)nextafterf(f, -INFINITY) >= b) f = nextafterf(f, -INFINITY);
    t[i - 1] = f;
  }
}

/* ----------------------------------------------------------- z-normalisation
 * Section II-A: series are compared after z-normalisation (mean 0, standard
 * deviation 1); population moments. Canonical fp32 order as in the header. */
static float orc_lane_tree(float a[32]) {
  for (int off = 1; off < 32; off <<= 1) {
    float b[32];
    for (int l = 0; l < 32; ++l) b[l] = a[l] + a[l ^ off];
    memcpy(a, b, sizeof b);
  }
  return a[0];
}

/* Returns 1 if the series is constant (z set to 0), 0 otherwise, -1 if non-finite. */
int32_t orc_znorm(const float* x, int32_t n, float* z, float* mu_out, float* rsig_out) {
  float acc[32] = {0};
  for (int32_t t = 0; t < n; ++t) acc[(t >> 2) & 31] = acc[(t >> 2) & 31] + x[t];
  const float s1 = orc_lane_tree(acc);
  const float mu = s1 / (float)n;
  float acc2[32] = {0};
  for (int32_t t = 0; t < n; ++t) {
    const float d = x[t] - mu;
    acc2[(t >> 2) & 31] = fmaf(d, d, acc2[(t >> 2) & 31]);
  }
  const float v = orc_lane_tree(acc2);
  const float sigma = sqrtf(v / (float)n);
  if (!isfinite(mu) || !isfinite(sigma)) {
    for (int32_t t = 0; t < n; ++t) z[t] = 0.0f;
    return -1;
  }
  if (sigma < 1e-30f || sigma <= 1e-6f * fabsf(mu)) {
    for (int32_t t = 0; t < n; ++t) z[t] = 0.0f;
    if (mu_out) *mu_out = mu;
    if (rsig_out) *rsig_out = 0.0f;
    return 1;
  }
  const float r = 1.0f / sigma;
  for (int32_t t = 0; t < n; ++t) z[t] = (x[t] - mu) * r;
  if (mu_out) *mu_out = mu;
  if (rsig_out) *rsig_out = r;
  return 0;
}

/* ------------------------------------------------------------------------ PAA
 * Section II-B: w segments of equal length s = n / w, each summarised by the mean
 * of its points. */
static int orc_is_pow2(int32_t v) { return v > 0 && (v & (v - 1)) == 0; }

void orc_paa(const float* z, int32_t n, int32_t w, float* paa) {
  const int32_t s = n / w;
  for (int32_t j = 0; j < w; ++j) {
    const float* seg = z + (int64_t)j * s;
    float sum;
    if (s % 4 == 0 && orc_is_pow2(s / 4)) {
      const int32_t g = s / 4;
      float* grp = (float*)malloc(sizeof(float) * (size_t)g);
      for (int32_t i = 0; i < g; ++i)
        grp[i] = ((seg[4 * i] + seg[4 * i + 1]) + seg[4 * i + 2]) + seg[4 * i + 3];
      for (int32_t off = 1; off < g; off <<= 1)
        for (int32_t i = 0; i < g; i += 2 * off) grp[i] = grp[i] + grp[i + off];
      sum = grp[0];
      free(grp);
    } else {
      sum = seg[0];
      for (int32_t t = 1; t < s; ++t) sum = sum + seg[t];
    }
    paa[j] = sum / (float)s;
  }
}

/* ------------------------------------------------------------------------ SAX
 * Section II-B: each segment gets the symbol of the region its PAA value falls
 * into; symbol = number of breakpoints at or below the value (0 .. c-1). */
void orc_sax(const float* paa, int32_t w, int32_t c, const float* t, uint8_t* word) {
  for (int32_t j = 0; j < w; ++j) {
    int32_t sym = 0;
    for (int32_t i = 0; i < c - 1; ++i)
      if (paa[j] >= t[i]) ++sym;
    word[j] = (uint8_t)sym;
  }
}

/* Algorithm 3 (CalculateiSAXSummaries), one series at a time: z-normalise, PAA, SAX.
 * Z, paa, words may be NULL. Returns the number of non-finite series. */
int64_t orc_summarise(const float* x, int64_t N, int32_t n, int32_t w, int32_t c, float* Z,
                      float* PAA, uint8_t* words, int32_t* constant) {
  float* t = (float*)malloc(sizeof(float) * (size_t)(c - 1));
  orc_thresholds(c, t);
  int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (int64_t i = 0; i < N; ++i) {
    float* zi = (float*)malloc(sizeof(float) * (size_t)n);
    float pi[64];
    const int32_t r = orc_znorm(x + i * n, n, zi, NULL, NULL);
    if (r < 0) ++bad;
    if (constant) constant[i] = r;
    orc_paa(zi, n, w, pi);
    if (Z) memcpy(Z + i * n, zi, sizeof(float) * (size_t)n);
    if (PAA) memcpy(PAA + i * w, pi, sizeof(float) * (size_t)w);
    if (words) orc_sax(pi, w, c, t, words + i * w);
    free(zi);
  }
  free(t);
  return bad;
}

/* ------------------------------------------------------------------ mindist
 * Lower bound between a query and an iSAX region (Section II-B; used by
 * TraverseRootSubtree, Algorithm 7, and CalculateRealDistance, Algorithm 9):
 * the iSAX mindist, sqrt(s * sum_j d_j^2), d_j the gap between the query's PAA
 * value and the value range [beta_lo, beta_{hi+1}) covered by symbols lo..hi of
 * segment j (0 inside). qpaa is the query's PAA in FP64 (exact mean of its
 * z-normalised points). */
double orc_mindist(const double* qpaa, const uint8_t* lo, const uint8_t* hi, int32_t w, int32_t n,
                   int32_t c, const double* beta) {
  const double s = (double)(n / w);
  double acc = 0.0;
  for (int32_t j = 0; j < w; ++j) {
    const double lower = lo[j] == 0 ? -INFINITY : beta[lo[j] - 1];
    const double upper = hi[j] >= c - 1 ? INFINITY : beta[hi[j]];
    double d = 0.0;
    if (qpaa[j] < lower) d = lower - qpaa[j];
    else if (qpaa[j] > upper) d = qpaa[j] - upper;
    acc += d * d;
  }
  return sqrt(s * acc);
}

/* FP64 mean of each segment of a (z-normalised) fp32 series. */
void orc_paa64(const float* z, int32_t n, int32_t w, double* paa) {
  const int32_t s = n / w;
  for (int32_t j = 0; j < w; ++j) {
    double sum = 0.0;
    for (int32_t t = 0; t < s; ++t) sum += (double)z[j * s + t];
    paa[j] = sum / (double)s;
  }
}

/* ------------------------------------------------------------ exact distance
 * Section II-A: Euclidean distance. D = sum_t (z_t - q_t)^2 in FP64, the terms added
 * one after another in increasing t: the definition written out. (The GPU re-check
 * adds the same FP64 terms in another order, so the two may differ in the last
 * bits; an exact tie between identical series is a tie under any order.) */
double orc_sqdist(const float* a, const float* b, int32_t n) {
  double acc = 0.0;
  for (int32_t t = 0; t < n; ++t) {
    const double d = (double)a[t] - (double)b[t];
    acc = acc + d * d;
  }
  return acc;
}

/* (D, id) order: smaller distance first, then lower id. */
static int orc_before(double da, int64_t ia, double db, int64_t ib) {
  return da < db || (da == db && ia < ib);
}

/* Insert (d, id) into a sorted list of at most k entries. */
static void orc_topk_push(double* kd, int64_t* ki, int32_t* cnt, int32_t k, double d, int64_t id) {
  if (*cnt == k && !orc_before(d, id, kd[k - 1], ki[k - 1])) return;
  int32_t pos = (*cnt < k) ? (*cnt)++ : k - 1;
  while (pos > 0 && orc_before(d, id, kd[pos - 1], ki[pos - 1])) {
    kd[pos] = kd[pos - 1];
    ki[pos] = ki[pos - 1];
    --pos;
  }
  kd[pos] = d;
  ki[pos] = id;
}

/* Exact k-NN by serial scan (the definition; the paper's UCR Suite-P comparator,
 * Section IV, is an exact scan as well): every series' FP64 squared distance, the k
 * smallest by (D, id). Z is [N][n] z-normalised, zq one z-normalised query.
 * Outputs: ids[k], d2[k] (FP64 squared distances), ascending. */
void orc_knn_scan(const float* Z, int64_t N, int32_t n, const float* zq, int32_t k, int64_t* ids,
                  double* d2) {
  int32_t nt = 1;
#ifdef _OPENMP
  nt = omp_get_max_threads();
#endif
  double* pd = (double*)malloc(sizeof(double) * (size_t)k * (size_t)nt);
  int64_t* pi = (int64_t*)malloc(sizeof(int64_t) * (size_t)k * (size_t)nt);
  int32_t* pc = (int32_t*)calloc((size_t)nt, sizeof(int32_t));
#pragma omp parallel num_threads(nt)
  {
    int32_t me = 0;
#ifdef _OPENMP
    me = omp_get_thread_num();
#endif
#pragma omp for schedule(static)
    for (int64_t i = 0; i < N; ++i)
      orc_topk_push(pd + (int64_t)me * k, pi + (int64_t)me * k, &pc[me], k,
                    orc_sqdist(Z + i * n, zq, n), i);
  }
  int32_t cnt = 0;
  for (int32_t th = 0; th < nt; ++th)
    for (int32_t j = 0; j < pc[th]; ++j)
      orc_topk_push(d2, ids, &cnt, k, pd[(int64_t)th * k + j], pi[(int64_t)th * k + j]);
  free(pd);
  free(pi);
  free(pc);
}

/* ------------------------------------------------------- index-based search
 * The oracle's own index, a flat stand-in for the iSAX tree: series ordered by
 * their SAX word (lexicographic, then id), cut into leaves of at most `cap` series,
 * each leaf summarised by its per-segment [min, max] symbol. Exact search follows
 * Algorithms 5-9 with one priority queue: leaves in ascending lower-bound order; a
 * leaf whose bound exceeds the current k-th best distance ends the search
 * (ProcessQueue, Algorithm 8); inside a leaf each series is first tested by its own
 * lower bound, then by its real distance (CalculateRealDistance, Algorithm 9).
 * `slack` is added to the k-th best distance in both tests: the SAX symbols are
 * decided on fp32 PAA values that can sit an ulp on the other side of a breakpoint
 * from the exact mean, so the bound is exact only up to that rounding.
 * Returns the number of real distances computed. */
typedef struct { const uint8_t* words; int32_t w; int64_t id; } orc_wref;
static int32_t orc_word_w;
static int orc_word_cmp(const void* a, const void* b) {
  const orc_wref* x = (const orc_wref*)a;
  const orc_wref* y = (const orc_wref*)b;
  int r = memcmp(x->words, y->words, (size_t)orc_word_w);
  if (r) return r;
  return (x->id > y->id) - (x->id < y->id);
}
typedef struct { double lb; int64_t leaf; } orc_leaf_lb;
static int orc_leaf_cmp(const void* a, const void* b) {
  const orc_leaf_lb* x = (const orc_leaf_lb*)a;
  const orc_leaf_lb* y = (const orc_leaf_lb*)b;
  if (x->lb < y->lb) return -1;
  if (x->lb > y->lb) return 1;
  return (x->leaf > y->leaf) - (x->leaf < y->leaf);
}

/* Forward declarations of the DTW pieces (defined below). */
double orc_dtw_sq(const float* a, const float* b, int32_t n, int32_t r);
void orc_envelope(const float* q, int32_t n, int32_t r, float* U, float* L);
void orc_paa_envelope(const float* U, const float* L, int32_t n, int32_t w, double* Uh, double* Lh);
double orc_mindist_env(const double* Uh, const double* Lh, const uint8_t* lo, const uint8_t* hi, int32_t w,
                       int32_t n, int32_t c, const double* beta);

/* r < 0: Euclidean distance and the PAA mindist; r >= 0: DTW with a band of
 * half-width r and the mindist of the query's PAA envelope (see below). */
static int64_t orc_knn_index_metric(const float* Z, const uint8_t* words, int64_t N, int32_t n, int32_t w,
                                    int32_t c, int32_t cap, const float* zq, int32_t k, double slack, int32_t r,
                                    int64_t* ids, double* d2) {
  orc_wref* order = (orc_wref*)malloc(sizeof(orc_wref) * (size_t)N);
  for (int64_t i = 0; i < N; ++i) {
    order[i].words = words + i * w;
    order[i].w = w;
    order[i].id = i;
  }
  orc_word_w = w;
  qsort(order, (size_t)N, sizeof(orc_wref), orc_word_cmp);
  const int64_t L = (N + cap - 1) / cap;
  uint8_t* lo = (uint8_t*)malloc((size_t)(L * w));
  uint8_t* hi = (uint8_t*)malloc((size_t)(L * w));
  for (int64_t l = 0; l < L; ++l) {
    for (int32_t j = 0; j < w; ++j) { lo[l * w + j] = 255; hi[l * w + j] = 0; }
    for (int64_t p = l * cap; p < N && p < (l + 1) * cap; ++p)
      for (int32_t j = 0; j < w; ++j) {
        const uint8_t v = order[p].words[j];
        if (v < lo[l * w + j]) lo[l * w + j] = v;
        if (v > hi[l * w + j]) hi[l * w + j] = v;
      }
  }
  double* beta = (double*)malloc(sizeof(double) * (size_t)(c - 1));
  orc_breakpoints(c, beta);
  double qpaa[64], Uh[64], Lh[64];
  orc_paa64(zq, n, w, qpaa);
  if (r >= 0) {
    float* U = (float*)malloc(sizeof(float) * (size_t)n);
    float* Lo = (float*)malloc(sizeof(float) * (size_t)n);
    orc_envelope(zq, n, r, U, Lo);
    orc_paa_envelope(U, Lo, n, w, Uh, Lh);
    free(U);
    free(Lo);
  }
  orc_leaf_lb* queue = (orc_leaf_lb*)malloc(sizeof(orc_leaf_lb) * (size_t)L);
  for (int64_t l = 0; l < L; ++l) {
    queue[l].lb = r < 0 ? orc_mindist(qpaa, lo + l * w, hi + l * w, w, n, c, beta)
                        : orc_mindist_env(Uh, Lh, lo + l * w, hi + l * w, w, n, c, beta);
    queue[l].leaf = l;
  }
  qsort(queue, (size_t)L, sizeof(orc_leaf_lb), orc_leaf_cmp);
  int32_t cnt = 0;
  int64_t real = 0;
  for (int64_t qi = 0; qi < L; ++qi) {
    const double bsf = cnt < k ? INFINITY : sqrt(d2[k - 1]);
    if (queue[qi].lb > bsf + slack) break;
    const int64_t l = queue[qi].leaf;
    for (int64_t p = l * cap; p < N && p < (l + 1) * cap; ++p) {
      const double bsf2 = cnt < k ? INFINITY : sqrt(d2[k - 1]);
      const uint8_t* wd = order[p].words;
      const double lb = r < 0 ? orc_mindist(qpaa, wd, wd, w, n, c, beta)
                              : orc_mindist_env(Uh, Lh, wd, wd, w, n, c, beta);
      if (lb > bsf2 + slack) continue;
      ++real;
      const float* row = Z + order[p].id * n;
      orc_topk_push(d2, ids, &cnt, k, r < 0 ? orc_sqdist(row, zq, n) : orc_dtw_sq(row, zq, n, r), order[p].id);
    }
  }
  free(order);
  free(lo);
  free(hi);
  free(beta);
  free(queue);
  return real;
}

int64_t orc_knn_index(const float* Z, const uint8_t* words, int64_t N, int32_t n, int32_t w,
                      int32_t c, int32_t cap, const float* zq, int32_t k, double slack,
                      int64_t* ids, double* d2) {
  return orc_knn_index_metric(Z, words, N, n, w, c, cap, zq, k, slack, -1, ids, d2);
}

/* ------------------------------------------------------------------ DTW
 * Section IV, "MESSI with DTW": the index is left as it is; the search uses the
 * LB_Keogh envelope of the query (Keogh and Ratanamahatana 2005) for its lower
 * bounds and Dynamic Time Warping (Berndt and Clifford 1994) for its real
 * distances, with a warping window (the paper uses 10% of the series length).
 *
 * DTW^2(a, b) = D(n-1, n-1), where D(i, j) = (a_i - b_j)^2 + min(D(i-1, j-1),
 * D(i-1, j), D(i, j-1)) for |i - j| <= r (a Sakoe-Chiba band of half-width r),
 * D(-1, -1) = 0 and every other cell off the grid or outside the band is +inf.
 * Every cell is d = (double)a_i - (double)b_j, then d * d, then the sum with the
 * minimum: one rounding each; a minimum is exact, so the value of a cell does not
 * depend on the order in which the cells are visited. */
double orc_dtw_sq(const float* a, const float* b, int32_t n, int32_t r) {
  /* prev[j + 1] = D(i - 1, j), cur[j + 1] = D(i, j); index 0 is column -1 */
  double* prev = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  double* cur = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  for (int32_t j = 0; j <= n; ++j) prev[j] = INFINITY;
  prev[0] = 0.0; /* D(-1, -1) */
  for (int32_t i = 0; i < n; ++i) {
    for (int32_t j = 0; j <= n; ++j) cur[j] = INFINITY;
    const int32_t j0 = i - r > 0 ? i - r : 0;
    const int32_t j1 = i + r < n - 1 ? i + r : n - 1;
    for (int32_t j = j0; j <= j1; ++j) {
      const double d = (double)a[i] - (double)b[j];
      double m = prev[j];                  /* D(i-1, j-1) */
      if (prev[j + 1] < m) m = prev[j + 1]; /* D(i-1, j)   */
      if (cur[j] < m) m = cur[j];           /* D(i, j-1)   */
      cur[j + 1] = d * d + m;
    }
    double* t = prev;
    prev = cur;
    cur = t;
  }
  const double out = prev[n];
  free(prev);
  free(cur);
  return out;
}

/* LB_Keogh envelope of q for a warping window r: U_i = max, L_i = min of
 * q_t over |t - i| <= r (inside the series). */
void orc_envelope(const float* q, int32_t n, int32_t r, float* U, float* L) {
  for (int32_t i = 0; i < n; ++i) {
    float u = q[i], l = q[i];
    for (int32_t t = i - r; t <= i + r; ++t) {
      if (t < 0 || t >= n) continue;
      if (q[t] > u) u = q[t];
      if (q[t] < l) l = q[t];
    }
    U[i] = u;
    L[i] = l;
  }
}

/* LB_Keogh(q, b)^2 = sum_i (b_i - U_i)^2 where b_i > U_i, (L_i - b_i)^2 where
 * b_i < L_i: a lower bound of DTW^2(q, b) for the same window. */
double orc_lb_keogh(const float* U, const float* L, const float* b, int32_t n) {
  double acc = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    double d = 0.0;
    if (b[i] > U[i]) d = (double)b[i] - (double)U[i];
    else if (b[i] < L[i]) d = (double)L[i] - (double)b[i];
    acc += d * d;
  }
  return acc;
}

/* The envelope reduced per segment (Keogh's PAA envelope): Uh_j = max of U over
 * segment j, Lh_j = min of L over it. */
void orc_paa_envelope(const float* U, const float* L, int32_t n, int32_t w, double* Uh, double* Lh) {
  const int32_t s = n / w;
  for (int32_t j = 0; j < w; ++j) {
    double u = -INFINITY, l = INFINITY;
    for (int32_t t = j * s; t < (j + 1) * s; ++t) {
      if ((double)U[t] > u) u = (double)U[t];
      if ((double)L[t] < l) l = (double)L[t];
    }
    Uh[j] = u;
    Lh[j] = l;
  }
}

/* Lower bound of DTW between the query and every series whose symbols lie in
 * [lo_j, hi_j]: sqrt(s * sum_j d_j^2), d_j the gap between the value range
 * [beta_lo, beta_{hi+1}) and the segment's envelope interval [Lh_j, Uh_j] (0 when
 * they meet). A series' PAA value lies in its region; the mean of a segment's points
 * above Uh_j is at least its gap to Uh_j, and by convexity the squared gaps of the
 * points sum to at least s times the squared gap of the mean, so this bounds
 * LB_Keogh, which bounds DTW. */
double orc_mindist_env(const double* Uh, const double* Lh, const uint8_t* lo, const uint8_t* hi, int32_t w,
                       int32_t n, int32_t c, const double* beta) {
  const double s = (double)(n / w);
  double acc = 0.0;
  for (int32_t j = 0; j < w; ++j) {
    const double lower = lo[j] == 0 ? -INFINITY : beta[lo[j] - 1];
    const double upper = hi[j] >= c - 1 ? INFINITY : beta[hi[j]];
    double d = 0.0;
    if (lower > Uh[j]) d = lower - Uh[j];
    else if (upper < Lh[j]) d = Lh[j] - upper;
    acc += d * d;
  }
  return sqrt(s * acc);
}

/* Exact k-NN under DTW by serial scan: the FP64 DTW^2 of every series, the k
 * smallest by (D, id). */
void orc_knn_scan_dtw(const float* Z, int64_t N, int32_t n, const float* zq, int32_t k, int32_t r, int64_t* ids,
                      double* d2) {
  int32_t nt = 1;
#ifdef _OPENMP
  nt = omp_get_max_threads();
#endif
  double* pd = (double*)malloc(sizeof(double) * (size_t)k * (size_t)nt);
  int64_t* pi = (int64_t*)malloc(sizeof(int64_t) * (size_t)k * (size_t)nt);
  int32_t* pc = (int32_t*)calloc((size_t)nt, sizeof(int32_t));
#pragma omp parallel num_threads(nt)
  {
    int32_t me = 0;
#ifdef _OPENMP
    me = omp_get_thread_num();
#endif
#pragma omp for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i)
      orc_topk_push(pd + (int64_t)me * k, pi + (int64_t)me * k, &pc[me], k, orc_dtw_sq(Z + i * n, zq, n, r), i);
  }
  int32_t cnt = 0;
  for (int32_t th = 0; th < nt; ++th)
    for (int32_t j = 0; j < pc[th]; ++j)
      orc_topk_push(d2, ids, &cnt, k, pd[(int64_t)th * k + j], pi[(int64_t)th * k + j]);
  free(pd);
  free(pi);
  free(pc);
}

/* Exact k-NN under DTW through the oracle's flat index (the same leaves and
 * priority order as orc_knn_index, with the envelope bounds). */
int64_t orc_knn_index_dtw(const float* Z, const uint8_t* words, int64_t N, int32_t n, int32_t w, int32_t c,
                          int32_t cap, const float* zq, int32_t k, int32_t r, double slack, int64_t* ids,
                          double* d2) {
  return orc_knn_index_metric(Z, words, N, n, w, c, cap, zq, k, slack, r, ids, d2);
}
