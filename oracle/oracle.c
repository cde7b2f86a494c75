/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the FMM-corrected back projection.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file: only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or helper with the CUDA
 * library; the two meet only through the seeded synthetic inputs.
 *
 * What it computes (Wang & Jing, "A fast marching method based back projection
 * algorithm for photoacoustic tomography in heterogeneous media"):
 *
 *   1. Travel times (Sec. II-B): the eikonal equation |grad T|^2 = 1/c^2 is
 *      solved by fast marching with one point source per sensor (the paper uses
 *      the sensor as the source because ray paths are reversible).  The local
 *      update is the first-order Godunov upwind scheme; the accepted set grows
 *      one node at a time in increasing T, taken from a binary min-heap with
 *      lazy deletion, ties broken by linear index.
 *   2. Preprocessing (Sec. II-C, Eq. (BP)): per sensor signal p_k = p(k dt) the
 *      integrand b_k = 2 p_k - 2 t_k dp/dt|_k, with a central difference in the
 *      interior and one-sided differences at both ends, t_k = k dt (the initial
 *      condition of Sec. II-A puts the time origin at the laser pulse).
 *   3. Back projection (Sec. II-C, Eq. (BP)): P(r_j) = sum_i w_i b_i(t_ij) with
 *      t_ij the travel time from sensor i to pixel j; b is sampled by linear
 *      interpolation in u = t/dt; samples after the last one contribute zero.
 *
 * Readings where the paper is silent:
 *   - first-order Godunov update by default; the printed second-order stencil
 *     (order 2) uses the one-sided second-order difference on an axis where
 *     the two upwind neighbours on the same side are accepted and monotone;
 *   - off-grid point source: the 2^ndim corners of the enclosing cell are
 *     accepted with T = |x - r_s| * f(x), f = 1/c at the node;
 *   - weights w_i default to 1/N_s and the integrand carries the factor 2 of
 *     the universal back projection (the paper's Eq. (BP) is that sum times
 *     N_s/2, a pure scale);
 *   - linear interpolation of b (not of p and dp/dt separately);
 *   - the exact back projection that Eq. (BP) approximates (Sec. II-C) weighs
 *     each sensor by the solid angle its element subtends at the pixel; the
 *     sum with a weight per (sensor, pixel) pair is oracle_bp_pairs, the
 *     weights themselves are formed in the Python half of the oracle.
 *
 * Everything is double precision; no blocking, fusion or reordering beyond the
 * steps above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1
#define ORACLE_ERR_NOMEM 2

enum { FAR = 0, TRIAL = 1, KNOWN = 2 };

/* ---------------------------------------------------------------- heap --- */
/* Binary min-heap of (T, linear index) pairs.  Stale entries stay in the heap
 * and are skipped when popped (lazy deletion). */
typedef struct {
  double t;
  int64_t idx;
} hentry;

typedef struct {
  hentry* a;
  int64_t n, cap;
} heap_t;

static int hless(hentry x, hentry y) {
  if (x.t < y.t) return 1;
  if (x.t > y.t) return 0;
  return x.idx < y.idx;
}

static int heap_push(heap_t* h, double t, int64_t idx) {
  if (h->n == h->cap) {
    int64_t nc = h->cap ? 2 * h->cap : 1024;
    hentry* na = (hentry*)realloc(h->a, (size_t)nc * sizeof(hentry));
    if (!na) return ORACLE_ERR_NOMEM;
    h->a = na;
    h->cap = nc;
  }
  int64_t i = h->n++;
  hentry e = {t, idx};
  while (i > 0) {
    int64_t parent = (i - 1) / 2;
    if (!hless(e, h->a[parent])) break;
    h->a[i] = h->a[parent];
    i = parent;
  }
  h->a[i] = e;
  return ORACLE_OK;
}

static hentry heap_pop(heap_t* h) {
  hentry top = h->a[0];
  hentry last = h->a[--h->n];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    hentry best = last;
    if (l < h->n && hless(h->a[l], best)) { m = l; best = h->a[l]; }
    if (r < h->n && hless(h->a[r], best)) { m = r; }
    if (m == i) break;
    h->a[i] = h->a[m];
    i = m;
  }
  if (h->n > 0) h->a[i] = last;
  return top;
}

/* ------------------------------------------------------- grid helpers --- */
typedef struct {
  int ndim;
  int64_t n[3];      /* nodes per axis, x fastest; unused axes have n = 1 */
  int64_t stride[3]; /* linear-index stride per axis */
  int64_t total;
} grid_t;

static int grid_init(grid_t* g, int ndim, const int64_t* n) {
  if (ndim < 1 || ndim > 3) return ORACLE_ERR_ARG;
  g->ndim = ndim;
  g->total = 1;
  for (int d = 0; d < 3; ++d) {
    g->n[d] = (d < ndim) ? n[d] : 1;
    if (g->n[d] < 1) return ORACLE_ERR_ARG;
    g->stride[d] = g->total;
    g->total *= g->n[d];
  }
  return ORACLE_OK;
}

static void grid_coords(const grid_t* g, int64_t idx, int64_t* c) {
  for (int d = 0; d < 3; ++d) {
    c[d] = idx % g->n[d];
    idx /= g->n[d];
  }
}

/* --------------------------------------------------- Godunov update --- */
/* Tentative arrival time at node v from its accepted neighbours only.
 *
 * For each axis d, a_d is the smaller accepted neighbour value along d (or
 * +inf).  The first-order upwind discretisation of |grad T| = f reads
 *     sum_d max(T - a_d, 0)^2 = (h f)^2 ,
 * solved by growing the number of contributing axes in increasing a_d:
 *   one axis:    T = a1 + h f;
 *   two axes:    (T - a1)^2 + (T - a2)^2 = h^2 f^2, used when the one-axis
 *                value exceeds a2;
 *   three axes:  (T-a1)^2 + (T-a2)^2 + (T-a3)^2 = h^2 f^2, used when the
 *                two-axis value exceeds a3.
 */
static double godunov_update(const grid_t* g, const double* T, const uint8_t* state,
                             int64_t v, double hf) {
  int64_t c[3];
  grid_coords(g, v, c);
  double a[3];
  int na = 0;
  for (int d = 0; d < g->ndim; ++d) {
    double best = INFINITY;
    if (c[d] > 0) {
      int64_t w = v - g->stride[d];
      if (state[w] == KNOWN && T[w] < best) best = T[w];
    }
    if (c[d] + 1 < g->n[d]) {
      int64_t w = v + g->stride[d];
      if (state[w] == KNOWN && T[w] < best) best = T[w];
    }
    if (best < INFINITY) a[na++] = best;
  }
  if (na == 0) return INFINITY;
  /* sort the (at most three) finite axis minima ascending */
  for (int i = 1; i < na; ++i) {
    double x = a[i];
    int j = i - 1;
    while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
    a[j + 1] = x;
  }
  double t = a[0] + hf;
  if (na >= 2 && t > a[1]) {
    double diff = a[0] - a[1];
    t = 0.5 * (a[0] + a[1] + sqrt(2.0 * hf * hf - diff * diff));
    if (na >= 3 && t > a[2]) {
      double s = a[0] + a[1] + a[2];
      double q = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
      t = (s + sqrt(s * s - 3.0 * (q - hf * hf))) / 3.0;
    }
  }
  return t;
}

/* ------------------------------------------- second-order update --- */
/* Tentative arrival time at node v with the second-order one-sided difference
 * (3 T_i - 4 T_{i-1} + T_{i-2}) / (2h) of Sec. II-B where it applies.
 *
 * Per axis d the upwind side is the one whose accepted neighbour is smaller
 * (the lower-index side on a tie).  With that neighbour's value t1 and the
 * value t2 of the node beyond it on the same side: if t2 is accepted and
 * t2 <= t1 the axis contributes (9/4) (T - (4 t1 - t2)/3)^2, otherwise
 * (T - t1)^2, as the first-order scheme.  The equation
 *     sum_d alpha_d (T - a_d)^2 = (h f)^2
 * is solved by growing the set of contributing axes in increasing a_d: with k
 * axes, A = sum alpha, B = sum alpha a, C = sum alpha a^2 - (h f)^2 and
 * T = (B + sqrt(B^2 - A C)) / A; the next axis joins while T exceeds its a.
 * If including an axis makes B^2 - A C negative, the root without it stays.
 * Unlike the first-order update, the result can depend on exact ties (the
 * switch t2 <= t1 flips on the last bit): a point source at a cell centre
 * gives exactly tied neighbours, and two evaluations that differ in rounding
 * can take different branches there.
 */
static double second_order_update(const grid_t* g, const double* T, const uint8_t* state,
                                  int64_t v, double hf) {
  int64_t c[3];
  grid_coords(g, v, c);
  double a[3], w[3];
  int na = 0;
  for (int d = 0; d < g->ndim; ++d) {
    double t1 = INFINITY;
    int side = 0;
    if (c[d] > 0 && state[v - g->stride[d]] == KNOWN) {
      t1 = T[v - g->stride[d]];
      side = -1;
    }
    if (c[d] + 1 < g->n[d] && state[v + g->stride[d]] == KNOWN && T[v + g->stride[d]] < t1) {
      t1 = T[v + g->stride[d]];
      side = 1;
    }
    if (side == 0) continue;
    double alpha = 1.0, ad = t1;
    int64_t c2 = c[d] + 2 * side;
    if (c2 >= 0 && c2 < g->n[d]) {
      int64_t v2 = v + 2 * side * g->stride[d];
      if (state[v2] == KNOWN && T[v2] <= t1) {
        alpha = 9.0 / 4.0;
        ad = (4.0 * t1 - T[v2]) / 3.0;
      }
    }
    a[na] = ad;
    w[na] = alpha;
    ++na;
  }
  if (na == 0) return INFINITY;
  /* sort the axes by a ascending (insertion sort, weights follow) */
  for (int i = 1; i < na; ++i) {
    double x = a[i], y = w[i];
    int j = i - 1;
    while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; w[j + 1] = w[j]; --j; }
    a[j + 1] = x;
    w[j + 1] = y;
  }
  double A = w[0], B = w[0] * a[0], C = w[0] * a[0] * a[0] - hf * hf;
  double t = a[0] + hf / sqrt(w[0]); /* one axis: alpha0 (T - a0)^2 = (h f)^2 */
  for (int k = 1; k < na; ++k) {
    if (!(t > a[k])) break;
    double A2 = A + w[k], B2 = B + w[k] * a[k], C2 = C + w[k] * a[k] * a[k];
    double disc = B2 * B2 - A2 * C2;
    if (disc < 0.0) break;
    A = A2;
    B = B2;
    C = C2;
    t = (B + sqrt(disc)) / A;
  }
  return t;
}

/* ------------------------------------------------------ fast marching --- */
/* Fast marching from an arbitrary accepted initial set.
 *
 * speed[total]     : sound speed at the nodes (m/s), > 0
 * src_idx/src_T    : n_src nodes accepted from the start with the given T
 * T[total]         : output arrival times (s); +inf where unreachable
 * pop_order        : optional, receives the linear index of every node in the
 *                    order it was accepted from the heap (sources excluded)
 * n_popped         : optional, number of entries written to pop_order
 */
int oracle_fmm_sources(int ndim, const int64_t* n, double h, const double* speed,
                       const int64_t* src_idx, const double* src_T, int64_t n_src,
                       double* T, int64_t* pop_order, int64_t* n_popped, int order) {
  grid_t g;
  if (grid_init(&g, ndim, n) != ORACLE_OK || !(h > 0) || !speed || !T) return ORACLE_ERR_ARG;
  if (n_src < 1 || !src_idx || !src_T || (order != 1 && order != 2)) return ORACLE_ERR_ARG;
  for (int64_t i = 0; i < g.total; ++i)
    if (!(speed[i] > 0)) return ORACLE_ERR_ARG;

  if (g.total <= 0) return ORACLE_ERR_ARG;
  uint8_t* state = (uint8_t*)calloc((size_t)g.total, 1);
  if (!state) return ORACLE_ERR_NOMEM;
  heap_t heap = {0, 0, 0};
  int rc = ORACLE_OK;
  for (int64_t i = 0; i < g.total; ++i) T[i] = INFINITY;
  for (int64_t k = 0; k < n_src; ++k) {
    int64_t v = src_idx[k];
    if (v < 0 || v >= g.total) { rc = ORACLE_ERR_ARG; goto done; }
    if (state[v] != KNOWN || src_T[k] < T[v]) T[v] = src_T[k];
    state[v] = KNOWN;
  }

  /* The accepted sources hand tentative values to their neighbours. */
  for (int64_t k = 0; k < n_src; ++k) {
    int64_t v = src_idx[k];
    int64_t c[3];
    grid_coords(&g, v, c);
    for (int d = 0; d < g.ndim; ++d) {
      for (int side = -1; side <= 1; side += 2) {
        int64_t cc = c[d] + side;
        if (cc < 0 || cc >= g.n[d]) continue;
        int64_t w = v + side * g.stride[d];
        if (state[w] == KNOWN) continue;
        double t = order == 2 ? second_order_update(&g, T, state, w, h / speed[w])
                              : godunov_update(&g, T, state, w, h / speed[w]);
        if (t < T[w]) {
          T[w] = t;
          state[w] = TRIAL;
          if ((rc = heap_push(&heap, t, w)) != ORACLE_OK) goto done;
        }
      }
    }
  }

  int64_t popped = 0;
  while (heap.n > 0) {
    hentry e = heap_pop(&heap);
    int64_t v = e.idx;
    if (state[v] == KNOWN) continue;   /* stale entry */
    if (e.t != T[v]) continue;         /* superseded by a smaller value */
    state[v] = KNOWN;
    if (pop_order) pop_order[popped] = v;
    ++popped;
    int64_t c[3];
    grid_coords(&g, v, c);
    for (int d = 0; d < g.ndim; ++d) {
      for (int side = -1; side <= 1; side += 2) {
        int64_t cc = c[d] + side;
        if (cc < 0 || cc >= g.n[d]) continue;
        int64_t w = v + side * g.stride[d];
        if (state[w] == KNOWN) continue;
        double t = order == 2 ? second_order_update(&g, T, state, w, h / speed[w])
                              : godunov_update(&g, T, state, w, h / speed[w]);
        if (t < T[w]) {
          T[w] = t;
          state[w] = TRIAL;
          if ((rc = heap_push(&heap, t, w)) != ORACLE_OK) goto done;
        }
      }
    }
  }
  if (n_popped) *n_popped = popped;

done:
  free(heap.a);
  free(state);
  return rc;
}

/* Point source at src (m).  Node i lies at origin + i*h per axis.  The corners
 * of the grid cell that holds the source are accepted with their straight
 * distance times the local slowness, then fast marching runs from them. */
int oracle_fmm_point(int ndim, const int64_t* n, double h, const double* origin,
                     const double* speed, const double* src, double* T,
                     int64_t* pop_order, int64_t* n_popped, int order) {
  grid_t g;
  if (grid_init(&g, ndim, n) != ORACLE_OK || !(h > 0) || !origin || !src) return ORACLE_ERR_ARG;
  int64_t cell[3] = {0, 0, 0};
  for (int d = 0; d < ndim; ++d) {
    if (g.n[d] < 2) return ORACLE_ERR_ARG;
    double x = (src[d] - origin[d]) / h;
    if (!(x >= 0.0) || !(x <= (double)(g.n[d] - 1))) return ORACLE_ERR_ARG;
    int64_t i = (int64_t)floor(x);
    if (i > g.n[d] - 2) i = g.n[d] - 2;
    cell[d] = i;
  }
  int ncorner = 1 << ndim;
  int64_t idx[8];
  double t0[8];
  for (int m = 0; m < ncorner; ++m) {
    int64_t v = 0;
    double dist2 = 0.0;
    for (int d = 0; d < ndim; ++d) {
      int64_t i = cell[d] + ((m >> d) & 1);
      v += i * g.stride[d];
      double dxd = origin[d] + (double)i * h - src[d];
      dist2 += dxd * dxd;
    }
    idx[m] = v;
    t0[m] = sqrt(dist2) / speed[v];
  }
  return oracle_fmm_sources(ndim, n, h, speed, idx, t0, ncorner, T, pop_order, n_popped, order);
}

/* ------------------------------------------------------ preprocessing --- */
/* b_k = 2 p_k - 2 t_k dp/dt|_k with t_k = k dt.  The derivative is the central
 * difference (p_{k+1} - p_{k-1}) / (2 dt) inside, and the one-sided differences
 * (p_1 - p_0)/dt and (p_{N-1} - p_{N-2})/dt at the two ends. */
int oracle_preprocess(const double* p, int64_t nt, double dt, double* b) {
  if (!p || !b || nt < 2 || !(dt > 0)) return ORACLE_ERR_ARG;
  for (int64_t k = 0; k < nt; ++k) {
    double dp;
    if (k == 0)
      dp = (p[1] - p[0]) / dt;
    else if (k == nt - 1)
      dp = (p[nt - 1] - p[nt - 2]) / dt;
    else
      dp = (p[k + 1] - p[k - 1]) / (2.0 * dt);
    double t = (double)k * dt;
    b[k] = 2.0 * p[k] - 2.0 * t * dp;
  }
  return ORACLE_OK;
}

/* b sampled at fractional sample index u by linear interpolation; zero after
 * the last sample (u > N-1).  The interval index is capped at N-2 so that
 * u = N-1 lands on the last sample. */
double oracle_sample(const double* b, int64_t nt, double u) {
  if (!(u >= 0.0) || u > (double)(nt - 1)) return 0.0;
  int64_t i0 = (int64_t)floor(u);
  if (i0 > nt - 2) i0 = nt - 2;
  double phi = u - (double)i0;
  return (1.0 - phi) * b[i0] + phi * b[i0 + 1];
}

/* --------------------------------------------------- back projection --- */
/* P_j = sum_s w_s b_s(T[s][j] / dt)  (Eq. (BP), with b of oracle_preprocess).
 *
 * T[ns][npix]   travel times (s) from sensor s to pixel j
 * p[ns][nt]     signals, sample k at t = k dt
 * w[ns]         weights, or NULL for 1/ns
 * out[npix]     image values at the pixels
 */
int oracle_bp(int64_t ns, int64_t npix, const double* T, double dt, int64_t nt,
              const double* p, const double* w, double* out) {
  if (ns < 1 || npix < 0 || !T || !p || !out || nt < 2 || !(dt > 0)) return ORACLE_ERR_ARG;
  double* b = (double*)malloc((size_t)(ns * nt) * sizeof(double));
  if (!b) return ORACLE_ERR_NOMEM;
  for (int64_t s = 0; s < ns; ++s) oracle_preprocess(p + s * nt, nt, dt, b + s * nt);
  for (int64_t j = 0; j < npix; ++j) {
    double acc = 0.0;
    for (int64_t s = 0; s < ns; ++s) {
      double ws = w ? w[s] : 1.0 / (double)ns;
      acc += ws * oracle_sample(b + s * nt, nt, T[s * npix + j] / dt);
    }
    out[j] = acc;
  }
  free(b);
  return ORACLE_OK;
}

/* P_j = sum_s W[s][j] b_s(T[s][j] / dt): Eq. (BP) with one weight per
 * (sensor, pixel) pair, the sensors summed in order.  With W[s][j] = w_s for
 * every j it is oracle_bp.
 *
 * T[ns][npix], W[ns][npix], p[ns][nt], out[npix] as in oracle_bp.
 */
int oracle_bp_pairs(int64_t ns, int64_t npix, const double* T, double dt, int64_t nt,
                    const double* p, const double* W, double* out) {
  if (ns < 1 || npix < 0 || !T || !p || !W || !out || nt < 2 || !(dt > 0)) return ORACLE_ERR_ARG;
  double* b = (double*)malloc((size_t)(ns * nt) * sizeof(double));
  if (!b) return ORACLE_ERR_NOMEM;
  for (int64_t s = 0; s < ns; ++s) oracle_preprocess(p + s * nt, nt, dt, b + s * nt);
  for (int64_t j = 0; j < npix; ++j) {
    double acc = 0.0;
    for (int64_t s = 0; s < ns; ++s)
      acc += W[s * npix + j] * oracle_sample(b + s * nt, nt, T[s * npix + j] / dt);
    out[j] = acc;
  }
  free(b);
  return ORACLE_OK;
}
