/*
 * kl_oracle.c -- plain, slow, FP64 CPU oracle for the indexed renderer of the
 * limit set of a once-punctured-torus group (Rosa, "A new indexed approach to
 * render the attractors of Kleinian groups", arXiv:1709.08018).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  It shares no code,
 * header, table or constant with the CUDA library, and the library never
 * calls it.
 *
 * Compile with -O2 -ffp-contract=off: every floating-point operation below
 * is meant to be executed exactly as written, in the order written, with no
 * fused multiply-add, so that the per-word and the tree-walk enumerations give
 * bit-identical word values.
 *
 * What is computed, and where the paper fixes it:
 *  - letters a, b, A, B with codes 0, 1, 2, 3 (the order of the rows and
 *    columns of the Cayley table of Sec. "Once-punctured torus groups",
 *    minus one); A = a^-1, B = b^-1, so inv(x) = (x + 2) mod 4.
 *  - a word w_1 ... w_d is reduced when no neighbouring pair is an inverse
 *    pair (the crash words aA, Aa, bB, Bb of the same section).
 *  - the word value is the last element of the orbit of the seed when the
 *    letters are applied right to left: w_d first, w_1 last (Sec.
 *    "Introduction", the abA example).
 *  - each map is the linear-fractional map (p z + q)/(r z + s) (Sec.
 *    "Once-punctured torus groups").
 *  - the index of a reduced word is its rank in the order in which the
 *    base-4 scan of Sec. "Implementation" meets reduced words: a base-4
 *    string with w_1 as its most significant digit.  Among reduced words this
 *    rank is the mixed-radix number with digit w_1 in base 4 followed by d-1
 *    base-3 digits (the rank of w_k among the three letters allowed after
 *    w_{k-1}); the tests check this against the brute-force scan.
 *  - generators from traces: Grandma's two-generator recipe (the book the
 *    paper builds on, Mumford-Series-Wright, "Indra's Pearls", ch. 8); seeds:
 *    the attracting fixed point of the first-applied letter.
 *  - "draw": a pixel of a uint32 hit image, column floor((x - x0) W/(x1-x0)),
 *    row floor((y1 - y) H/(y1-y0)), half-open window; non-finite and
 *    out-of-window values are dropped and counted.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EXPORT __attribute__((visibility("default")))

typedef struct { double re, im; } cx;

static cx cx_make(double re, double im) { cx z; z.re = re; z.im = im; return z; }
static cx cx_add(cx a, cx b) { return cx_make(a.re + b.re, a.im + b.im); }
static cx cx_sub(cx a, cx b) { return cx_make(a.re - b.re, a.im - b.im); }
static cx cx_mul(cx a, cx b) {
  return cx_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
static cx cx_scale(cx a, double s) { return cx_make(a.re * s, a.im * s); }
/* n / m as (n * conj(m)) / |m|^2 */
static cx cx_div(cx n, cx m) {
  double den = m.re * m.re + m.im * m.im;
  return cx_make((n.re * m.re + n.im * m.im) / den, (n.im * m.re - n.re * m.im) / den);
}
static double cx_abs(cx a) { return hypot(a.re, a.im); }
/* principal square root */
static cx cx_sqrt(cx a) {
  double r = cx_abs(a);
  if (r == 0.0) return cx_make(0.0, 0.0);
  double t = sqrt(0.5 * (r + fabs(a.re)));
  if (a.re >= 0.0) return cx_make(t, a.im / (2.0 * t));
  return cx_make(fabs(a.im) / (2.0 * t), a.im >= 0.0 ? t : -t);
}

/* A 2x2 complex matrix [[p, q], [r, s]] acting as z -> (p z + q)/(r z + s). */
typedef struct { cx p, q, r, s; } mat2;

static void mat_store(const mat2* m, double* out8) {
  out8[0] = m->p.re; out8[1] = m->p.im; out8[2] = m->q.re; out8[3] = m->q.im;
  out8[4] = m->r.re; out8[5] = m->r.im; out8[6] = m->s.re; out8[7] = m->s.im;
}
static mat2 mat_load(const double* in8) {
  mat2 m;
  m.p = cx_make(in8[0], in8[1]); m.q = cx_make(in8[2], in8[3]);
  m.r = cx_make(in8[4], in8[5]); m.s = cx_make(in8[6], in8[7]);
  return m;
}

/* Inverse of a determinant-one matrix: the adjugate [[s, -q], [-r, p]]. */
static mat2 mat_inverse_unimodular(mat2 m) {
  mat2 o;
  o.p = m.s; o.q = cx_make(-m.q.re, -m.q.im);
  o.r = cx_make(-m.r.re, -m.r.im); o.s = m.p;
  return o;
}

/* One linear-fractional map applied to a point. */
static cx mobius(const mat2* m, cx z) {
  cx num = cx_add(cx_mul(m->p, z), m->q);
  cx den = cx_add(cx_mul(m->r, z), m->s);
  return cx_div(num, den);
}

/*
 * Grandma's two-generator recipe (Indra's Pearls, ch. 8): given the traces
 * ta = tr a and tb = tr b, tab = tr ab is the root of
 *   tab^2 - ta tb tab + ta^2 + tb^2 = 0
 * (the once-punctured-torus condition tr(a b a^-1 b^-1) = -2) taken with the
 * minus sign, z0 = (tab - 2) tb / (tb tab - 2 ta + 2 i tab), and
 *   a = [[ta/2, (ta tab - 2 tb + 4i) / ((2 tab + 4) z0)],
 *        [(ta tab - 2 tb - 4i) z0 / (2 tab - 4), ta/2]]
 *   b = [[(tb - 2i)/2, tb/2], [tb/2, (tb + 2i)/2]].
 * out: 32 doubles = a, b, A, B, each (p, q, r, s) as (re, im) pairs.
 * Returns 0, or -1 when a denominator of the recipe vanishes.
 */
OR_EXPORT int or_grandma(double ta_re, double ta_im, double tb_re, double tb_im, double* out) {
  cx ta = cx_make(ta_re, ta_im), tb = cx_make(tb_re, tb_im);
  cx i1 = cx_make(0.0, 1.0);
  cx tatb = cx_mul(ta, tb);
  cx disc = cx_sub(cx_mul(tatb, tatb),
                   cx_add(cx_scale(cx_mul(ta, ta), 4.0), cx_scale(cx_mul(tb, tb), 4.0)));
  cx tab = cx_scale(cx_sub(tatb, cx_sqrt(disc)), 0.5);
  cx z0den = cx_add(cx_sub(cx_mul(tb, tab), cx_scale(ta, 2.0)), cx_scale(cx_mul(i1, tab), 2.0));
  cx z0num = cx_mul(cx_sub(tab, cx_make(2.0, 0.0)), tb);
  cx d1 = cx_mul(cx_add(cx_scale(tab, 2.0), cx_make(4.0, 0.0)), cx_make(1.0, 0.0));
  cx d2 = cx_sub(cx_scale(tab, 2.0), cx_make(4.0, 0.0));
  if (cx_abs(z0den) == 0.0 || cx_abs(d2) == 0.0) return -1;
  cx z0 = cx_div(z0num, z0den);
  cx d1z0 = cx_mul(d1, z0);
  if (cx_abs(d1z0) == 0.0) return -1;
  cx tatab = cx_mul(ta, tab);
  cx base = cx_sub(tatab, cx_scale(tb, 2.0));
  mat2 a, b;
  a.p = cx_scale(ta, 0.5);
  a.q = cx_div(cx_add(base, cx_make(0.0, 4.0)), d1z0);
  a.r = cx_div(cx_mul(cx_sub(base, cx_make(0.0, 4.0)), z0), d2);
  a.s = cx_scale(ta, 0.5);
  b.p = cx_scale(cx_sub(tb, cx_make(0.0, 2.0)), 0.5);
  b.q = cx_scale(tb, 0.5);
  b.r = cx_scale(tb, 0.5);
  b.s = cx_scale(cx_add(tb, cx_make(0.0, 2.0)), 0.5);
  mat2 A = mat_inverse_unimodular(a), B = mat_inverse_unimodular(b);
  mat_store(&a, out); mat_store(&b, out + 8); mat_store(&A, out + 16); mat_store(&B, out + 24);
  return 0;
}

/*
 * Attracting fixed point of z -> (p z + q)/(r z + s).  With r != 0 the fixed
 * points solve r z^2 + (s - p) z - q = 0: z = ((p - s) +- sqrt((p - s)^2 + 4 q r)) / (2 r).
 * |M'(z)| = 1 / |r z + s|^2 for a determinant-one matrix, so the attracting one
 * has the larger |r z + s|; a tie (parabolic map) takes the + root.  With r = 0
 * the finite fixed point is q / (s - p), and the map must contract there
 * (|p/s| < 1 fails -> infinity attracts -> error).
 * out: 8 doubles = seeds of a, b, A, B as (re, im).  Returns 0 or -1.
 */
OR_EXPORT int or_seeds(const double* gens, double* out) {
  for (int x = 0; x < 4; ++x) {
    mat2 m = mat_load(gens + 8 * x);
    cx z;
    if (m.r.re == 0.0 && m.r.im == 0.0) {
      cx sp = cx_sub(m.s, m.p);
      if (cx_abs(sp) == 0.0) return -1;
      if (!(cx_abs(m.p) < cx_abs(m.s))) return -1;
      z = cx_div(m.q, sp);
    } else {
      cx pms = cx_sub(m.p, m.s);
      cx root = cx_sqrt(cx_add(cx_mul(pms, pms), cx_scale(cx_mul(m.q, m.r), 4.0)));
      cx twor = cx_scale(m.r, 2.0);
      cx zp = cx_div(cx_add(pms, root), twor);
      cx zm = cx_div(cx_sub(pms, root), twor);
      double kp = cx_abs(cx_add(cx_mul(m.r, zp), m.s));
      double km = cx_abs(cx_add(cx_mul(m.r, zm), m.s));
      z = (km > kp) ? zm : zp;
    }
    out[2 * x] = z.re; out[2 * x + 1] = z.im;
  }
  return 0;
}

/* N_d = 4 * 3^(d-1): reduced words of length exactly d; 0 if d < 1 or overflow. */
OR_EXPORT uint64_t or_word_count(int d) {
  if (d < 1) return 0;
  uint64_t n = 4;
  for (int k = 1; k < d; ++k) {
    if (n > UINT64_MAX / 3) return 0;
    n *= 3;
  }
  return n;
}

static uint64_t pow3(int e) { uint64_t v = 1; while (e-- > 0) v *= 3; return v; }

/*
 * Index -> reduced word (letters w_1 .. w_d, codes 0..3).  The leading digit
 * c_1 = floor(i / 3^(d-1)) is w_1; each following base-3 digit c_k picks the
 * c_k-th smallest letter different from inv(w_{k-1}).
 * Returns 0, or -1 when i >= N_d or d is out of range.
 */
OR_EXPORT int or_decode(int d, uint64_t i, uint8_t* letters) {
  uint64_t n = or_word_count(d);
  if (n == 0 || i >= n) return -1;
  uint64_t place = pow3(d - 1);
  int prev = (int)(i / place);
  uint64_t rest = i % place;
  letters[0] = (uint8_t)prev;
  for (int k = 1; k < d; ++k) {
    place /= 3;
    int c = (int)(rest / place);
    rest %= place;
    int banned = (prev + 2) & 3;
    /* the letters other than `banned`, in increasing order */
    int seen = -1, w = -1;
    for (int x = 0; x < 4; ++x) {
      if (x == banned) continue;
      if (++seen == c) { w = x; break; }
    }
    letters[k] = (uint8_t)w;
    prev = w;
  }
  return 0;
}

/* Word value: z = seed[w_d]; then z <- M_{w_k}(z) for k = d, d-1, ..., 1. */
static cx word_value(const mat2* g, const cx* seeds, const uint8_t* w, int d) {
  cx z = seeds[w[d - 1]];
  for (int k = d - 1; k >= 0; --k) z = mobius(&g[w[k]], z);
  return z;
}

static void load_group(const double* gens, const double* seeds8, mat2* g, cx* seeds) {
  for (int x = 0; x < 4; ++x) {
    g[x] = mat_load(gens + 8 * x);
    seeds[x] = cx_make(seeds8[2 * x], seeds8[2 * x + 1]);
  }
}

/* Word values of the given indices, sequentially per word.  out: 2n doubles. */
OR_EXPORT int or_eval(const double* gens, const double* seeds8, int d,
                      const uint64_t* idx, uint64_t n, double* out) {
  mat2 g[4]; cx seeds[4];
  load_group(gens, seeds8, g, seeds);
  uint8_t w[64];
  if (d < 1 || d > 40) return -1;
  for (uint64_t t = 0; t < n; ++t) {
    if (or_decode(d, idx[t], w) != 0) return -1;
    cx z = word_value(g, seeds, w, d);
    out[2 * t] = z.re; out[2 * t + 1] = z.im;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Rendering                                                                */

typedef struct {
  double x0, x1, y0, y1;
  int width, height;
  double sx, sy;       /* W / (x1 - x0), H / (y1 - y0) */
  double eta;          /* edge band, in pixels */
} view_t;

static view_t make_view(const double* win, int width, int height, double eta) {
  view_t v;
  v.x0 = win[0]; v.x1 = win[1]; v.y0 = win[2]; v.y1 = win[3];
  v.width = width; v.height = height;
  v.sx = (double)width / (v.x1 - v.x0);
  v.sy = (double)height / (v.y1 - v.y0);
  v.eta = eta;
  return v;
}

/* distance from t to the nearest integer */
static double frac_dist(double t) { double f = t - floor(t); return f < 0.5 ? f : 1.0 - f; }

typedef struct {
  uint32_t* image;              /* H*W, row-major, row 0 = top */
  uint64_t in_window, dropped;  /* per worker, summed at the end */
  uint64_t* edge_idx;           /* capacity edge_cap; shared */
  double* edge_uv;              /* 2 * edge_cap; shared */
  uint64_t edge_cap;
  uint64_t* edge_count;         /* shared, atomically incremented */
} sink_t;

/* Bin one word value.  Edge words (a pixel coordinate within eta of an
 * integer, inside or at the border of the window) are logged with (u, v). */
static void splat(const view_t* v, sink_t* s, uint64_t index, cx z) {
  double u = (z.re - v->x0) * v->sx;
  double w = (v->y1 - z.im) * v->sy;
  if (v->eta > 0.0 && u == u && w == w && fabs(u) < 1e15 && fabs(w) < 1e15) {
    int near_u = frac_dist(u) < v->eta && u > -1.0 && u < v->width + 1.0;
    int near_w = frac_dist(w) < v->eta && w > -1.0 && w < v->height + 1.0;
    int in_u = u > -1.0 && u < v->width + 1.0;
    int in_w = w > -1.0 && w < v->height + 1.0;
    if ((near_u && in_w) || (near_w && in_u)) {
      uint64_t k = __atomic_fetch_add(s->edge_count, 1, __ATOMIC_RELAXED);
      if (k < s->edge_cap) {
        s->edge_idx[k] = index;
        s->edge_uv[2 * k] = u;
        s->edge_uv[2 * k + 1] = w;
      }
    }
  }
  if (!(u >= 0.0 && u < (double)v->width && w >= 0.0 && w < (double)v->height)) {
    s->dropped++;
    return;
  }
  int col = (int)floor(u), row = (int)floor(w);
  __atomic_fetch_add(&s->image[(uint64_t)row * (uint64_t)v->width + (uint64_t)col], 1u,
                     __ATOMIC_RELAXED);
  s->in_window++;
}

/*
 * Per-word render (the definition, "mode A"): for every index in [i0, i1),
 * decode, evaluate sequentially, bin.  counters[0] += in-window words,
 * counters[1] += dropped words.  edge_* may be NULL with edge_cap = 0.
 */
OR_EXPORT int or_render_indexed(const double* gens, const double* seeds8, int d,
                                const double* window, int width, int height,
                                uint64_t i0, uint64_t i1, uint32_t* image, uint64_t* counters,
                                double eta, uint64_t* edge_idx, double* edge_uv,
                                uint64_t edge_cap, uint64_t* edge_count) {
  mat2 g[4]; cx seeds[4];
  load_group(gens, seeds8, g, seeds);
  uint64_t n = or_word_count(d);
  if (n == 0 || d > 40 || i1 > n || i0 > i1 || width <= 0 || height <= 0) return -1;
  view_t v = make_view(window, width, height, eta);
  uint64_t dummy = 0;
  sink_t s = {image, 0, 0, edge_idx, edge_uv, edge_cap, edge_count ? edge_count : &dummy};
  uint8_t w[64];
  for (uint64_t i = i0; i < i1; ++i) {
    or_decode(d, i, w);
    splat(&v, &s, i, word_value(g, seeds, w, d));
  }
  counters[0] += s.in_window;
  counters[1] += s.dropped;
  return 0;
}

/*
 * Sharded render (one process per GPU renders a share of the words and the
 * shares' images are summed).  The paper's loop runs over one index range on
 * one machine; its words are independent of one another (each is pulled out
 * of its own integer, Sec. "The revised deterministic approach"), which is
 * what allows any partition.  The library's partition is by prefix slot: with
 * prefix length p, the prefix slot of w_1 .. w_d is
 *     r = sum_{k=1}^{p-1} rank_k 3^(k-1),
 * rank_k = the position of w_k among the three letters other than the inverse
 * of its right neighbour w_{k+1}, in increasing order (so w_{p-1} is the most
 * significant digit).  Shard k of n holds the words with
 *     floor(k 3^(p-1) / n) <= r < floor((k+1) 3^(p-1) / n).
 */
static uint64_t prefix_rank(const uint8_t* w, int p) {
  uint64_t r = 0, place = 1;
  for (int k = 0; k + 1 < p; ++k) {   /* k = 0 is w_1 (weight 3^0) */
    int banned = (w[k + 1] + 2) & 3;
    int rank = -1, seen = -1;
    for (int x = 0; x < 4; ++x) {
      if (x == banned) continue;
      ++seen;
      if (x == w[k]) { rank = seen; break; }
    }
    r += (uint64_t)rank * place;
    place *= 3;
  }
  return r;
}

/* Prefix slot ranks of n word indices at prefix length p (1 <= p <= d). */
OR_EXPORT int or_prefix_rank(int d, int p, const uint64_t* idx, uint64_t n, uint64_t* out) {
  if (or_word_count(d) == 0 || p < 1 || p > d) return -1;
  uint8_t w[64];
  for (uint64_t t = 0; t < n; ++t) {
    if (or_decode(d, idx[t], w) != 0) return -1;
    out[t] = prefix_rank(w, p);
  }
  return 0;
}

/* Per-word render of shard k of n (see above) of the words of length d. */
OR_EXPORT int or_render_shard(const double* gens, const double* seeds8, int d,
                              const double* window, int width, int height, int p, int shard,
                              int n_shards, uint32_t* image, uint64_t* counters, double eta,
                              uint64_t* edge_idx, double* edge_uv, uint64_t edge_cap,
                              uint64_t* edge_count) {
  mat2 g[4]; cx seeds[4];
  load_group(gens, seeds8, g, seeds);
  uint64_t n = or_word_count(d);
  if (n == 0 || d > 40 || p < 1 || p > d || n_shards < 1 || shard < 0 || shard >= n_shards ||
      width <= 0 || height <= 0)
    return -1;
  uint64_t np = pow3(p - 1);
  uint64_t lo = (uint64_t)shard * np / (uint64_t)n_shards;
  uint64_t hi = (uint64_t)(shard + 1) * np / (uint64_t)n_shards;
  view_t v = make_view(window, width, height, eta);
  uint64_t dummy = 0;
  sink_t s = {image, 0, 0, edge_idx, edge_uv, edge_cap, edge_count ? edge_count : &dummy};
  uint8_t w[64];
  for (uint64_t i = 0; i < n; ++i) {
    or_decode(d, i, w);
    uint64_t r = prefix_rank(w, p);
    if (r < lo || r >= hi) continue;
    splat(&v, &s, i, word_value(g, seeds, w, d));
  }
  counters[0] += s.in_window;
  counters[1] += s.dropped;
  return 0;
}

/*
 * Tree-walk render ("mode B"): the same word values, reached from the inside
 * out.  A node at level k holds the value of its k innermost letters
 * (w_{d-k+1} .. w_d) applied to the seed of w_d; its children prepend one
 * outer letter, so value(x U) = M_x(value(U)).  Every word performs the same
 * maps, in the same order, on the same operands as the per-word definition,
 * hence bit-identical values at about 1.5 maps per word.  The index of each
 * leaf is accumulated digit by digit as outer letters are chosen.
 */
typedef struct {
  const mat2* g; const cx* seeds; int d;
  const view_t* view;
  uint64_t p3[64];
} walk_t;

static void walk(const walk_t* t, sink_t* s, int level, int inner_letter, cx z, uint64_t idx_acc) {
  /* `level` letters chosen so far; inner_letter = the outermost of them
   * (w_{d-level+1}); z = value of those letters. */
  if (level == t->d) {
    splat(t->view, s, idx_acc + (uint64_t)inner_letter * t->p3[t->d - 1], z);
    return;
  }
  int pos = t->d - level;  /* 1-based position of the letter chosen now: w_pos */
  int banned = (inner_letter + 2) & 3;  /* the new outer letter may not be inv(inner) */
  for (int y = 0; y < 4; ++y) {
    if (y == banned) continue;
    /* digit of w_{pos+1} = inner_letter given its outer neighbour y */
    int ban_after_y = (y + 2) & 3;
    int c = inner_letter - (inner_letter > ban_after_y ? 1 : 0);
    uint64_t acc = idx_acc + (uint64_t)c * t->p3[t->d - pos - 1];
    walk(t, s, level + 1, y, mobius(&t->g[y], z), acc);
  }
}

typedef struct {
  walk_t wt;
  sink_t sink;
  int* next_job;       /* shared */
  int n_jobs;          /* one past the last job to run */
} worker_arg_t;

/* jobs: the 4 * 3^(J-1) subtrees of the J = min(d, 5) innermost letters,
 * all of equal size N_d / (4 * 3^(J-1)); job = x + 4 * (base-3 digits of the
 * next J-1 letters' ranks, innermost first). */
static int job_levels(int d) { return d < 5 ? d : 5; }

static void run_job(worker_arg_t* a, int job) {
  const walk_t* t = &a->wt;
  int d = t->d;
  int roots = job_levels(d);
  int x = job % 4, j = job / 4;  /* innermost letter x = w_d */
  cx z = mobius(&t->g[x], t->seeds[x]);
  int level = 1, inner = x;
  uint64_t acc = 0;
  for (int r = 1; r < roots; ++r) {
    int k = j % 3; j /= 3;
    int banned = (inner + 2) & 3;
    int y = -1, seen = -1;
    for (int cand = 0; cand < 4; ++cand) {
      if (cand == banned) continue;
      if (++seen == k) { y = cand; break; }
    }
    int pos = d - level;
    int ban_after_y = (y + 2) & 3;
    int c = inner - (inner > ban_after_y ? 1 : 0);
    acc += (uint64_t)c * t->p3[d - pos - 1];
    z = mobius(&t->g[y], z);
    inner = y;
    level++;
  }
  walk(t, &a->sink, level, inner, z, acc);
}

static void* worker(void* p) {
  worker_arg_t* a = (worker_arg_t*)p;
  for (;;) {
    int job = __atomic_fetch_add(a->next_job, 1, __ATOMIC_RELAXED);
    if (job >= a->n_jobs) break;
    run_job(a, job);
  }
  return NULL;
}

/* Number of equal-size jobs of the tree walk at depth d. */
OR_EXPORT int or_tree_jobs(int d) {
  int j = 4;
  for (int k = 1; k < job_levels(d); ++k) j *= 3;
  return j;
}

/* Tree-walk render of the jobs [job0, job1) (all jobs: 0, or_tree_jobs(d)). */
OR_EXPORT int or_render_tree(const double* gens, const double* seeds8, int d,
                             const double* window, int width, int height, int n_threads,
                             int job0, int job1,
                             uint32_t* image, uint64_t* counters, double eta,
                             uint64_t* edge_idx, double* edge_uv, uint64_t edge_cap,
                             uint64_t* edge_count) {
  mat2 g[4]; cx seeds[4];
  load_group(gens, seeds8, g, seeds);
  if (or_word_count(d) == 0 || d > 40 || width <= 0 || height <= 0) return -1;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  view_t v = make_view(window, width, height, eta);
  uint64_t dummy = 0;
  int n_jobs = or_tree_jobs(d);
  if (job0 < 0 || job1 > n_jobs || job0 > job1) return -1;
  int next_job = job0;
  n_jobs = job1;
  worker_arg_t* args = (worker_arg_t*)calloc((size_t)n_threads, sizeof(worker_arg_t));
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!args || !th) { free(args); free(th); return -1; }
  for (int k = 0; k < n_threads; ++k) {
    args[k].wt.g = g; args[k].wt.seeds = seeds; args[k].wt.d = d; args[k].wt.view = &v;
    for (int e = 0; e < 64; ++e) args[k].wt.p3[e] = e < 41 ? pow3(e) : 0;
    sink_t s = {image, 0, 0, edge_idx, edge_uv, edge_cap, edge_count ? edge_count : &dummy};
    args[k].sink = s;
    args[k].next_job = &next_job;
    args[k].n_jobs = n_jobs;
  }
  int started = 0;
  for (int k = 1; k < n_threads; ++k) {
    if (pthread_create(&th[k], NULL, worker, &args[k]) != 0) break;
    started = k;
  }
  worker(&args[0]);
  for (int k = 1; k <= started; ++k) pthread_join(th[k], NULL);
  for (int k = 0; k < n_threads; ++k) {
    counters[0] += args[k].sink.in_window;
    counters[1] += args[k].sink.dropped;
  }
  free(args); free(th);
  return 0;
}

/* or_decode for n indices: out[t*d .. t*d + d - 1]; an index >= N_d gives
 * letters 0xFF (and the call still returns 0). */
OR_EXPORT int or_decode_many(int d, const uint64_t* idx, uint64_t n, uint8_t* out) {
  if (or_word_count(d) == 0) return -1;
  for (uint64_t t = 0; t < n; ++t) {
    if (or_decode(d, idx[t], out + t * (uint64_t)d) != 0)
      memset(out + t * (uint64_t)d, 0xFF, (size_t)d);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* General presentations (Sec. "Cayley Multiplication Tables", Sec.         */
/* "Implementation"): the paper's own scan over every index n of the        */
/* unpruned m-ary tree of depth d.  n is written as d base-m digits, most   */
/* significant first, each plus one (symbols 1 .. m; 0 is the identity);    */
/* the string is kept if the run of the indexed Cayley table over it, read  */
/* right to left from state 0, never reaches the crash state 0.  A kept     */
/* string w_1 .. w_d (letter code = symbol - 1) is drawn at its word value: */
/* the seed of w_d, then the maps of w_d, ..., w_1.                         */

#define OR_FSA_MAX 9

/* 1 if the symbols s[0..d-1] survive the table run, else 0. */
static int fsa_run(int m, const uint8_t* table, const uint8_t* s, int d) {
  int state = 0;
  for (int k = d - 1; k >= 0; --k) {
    state = table[state * (m + 1) + s[k]];
    if (state == 0) return 0;
  }
  return 1;
}

/* Kept strings of the scan (counted by scanning; m^d <= 2^40). */
OR_EXPORT int or_fsa_count(int m, const uint8_t* table, int d, uint64_t* out) {
  if (m < 1 || m > OR_FSA_MAX || d < 1 || d > 40) return -1;
  double total = pow((double)m, (double)d);
  if (total > 1099511627776.0) return -1;
  uint64_t n_idx = 1;
  for (int k = 0; k < d; ++k) n_idx *= (uint64_t)m;
  uint8_t s[64];
  uint64_t kept = 0;
  for (uint64_t n = 0; n < n_idx; ++n) {
    uint64_t r = n;
    for (int k = d - 1; k >= 0; --k) { s[k] = (uint8_t)(r % (uint64_t)m + 1); r /= (uint64_t)m; }
    kept += (uint64_t)fsa_run(m, table, s, d);
  }
  *out = kept;
  return 0;
}

/* Render of the kept strings of the scan of indices [i0, i1).  gens: m
 * matrices of 8 doubles, seeds: m points of 2 doubles.  counters[0] +=
 * in-window words, counters[1] += dropped kept words; edge words as in
 * or_render_indexed, logged with their scan index n. */
OR_EXPORT int or_render_fsa(int m, const uint8_t* table, const double* gens,
                            const double* seeds2, int d, const double* window, int width,
                            int height, uint64_t i0, uint64_t i1, uint32_t* image,
                            uint64_t* counters, double eta, uint64_t* edge_idx,
                            double* edge_uv, uint64_t edge_cap, uint64_t* edge_count) {
  if (m < 1 || m > OR_FSA_MAX || d < 1 || d > 40 || width <= 0 || height <= 0) return -1;
  for (int k = 0; k < (m + 1) * (m + 1); ++k)
    if (table[k] > m) return -1;
  uint64_t n_idx = 1;
  for (int k = 0; k < d; ++k) {
    if (n_idx > (1ull << 40) / (uint64_t)m) return -1;
    n_idx *= (uint64_t)m;
  }
  if (i1 > n_idx || i0 > i1) return -1;
  mat2 g[OR_FSA_MAX]; cx seeds[OR_FSA_MAX];
  for (int x = 0; x < m; ++x) {
    g[x] = mat_load(gens + 8 * x);
    seeds[x] = cx_make(seeds2[2 * x], seeds2[2 * x + 1]);
  }
  view_t v = make_view(window, width, height, eta);
  uint64_t dummy = 0;
  sink_t sk = {image, 0, 0, edge_idx, edge_uv, edge_cap, edge_count ? edge_count : &dummy};
  uint8_t s[64], w[64];
  for (uint64_t n = i0; n < i1; ++n) {
    uint64_t r = n;
    for (int k = d - 1; k >= 0; --k) { s[k] = (uint8_t)(r % (uint64_t)m + 1); r /= (uint64_t)m; }
    if (!fsa_run(m, table, s, d)) continue;
    for (int k = 0; k < d; ++k) w[k] = (uint8_t)(s[k] - 1);
    splat(&v, &sk, n, word_value(g, seeds, w, d));
  }
  counters[0] += sk.in_window;
  counters[1] += sk.dropped;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Maskit's slice ("Indra's Pearls", ch. 9), the group of the paper's       */
/* example: a(z) = mu + 1/z and b(z) = z + 2.  As matrices of determinant   */
/* one: a = i [[mu, 1], [1, 0]] and b = [[1, 2], [0, 1]]; A, B their        */
/* inverses.  Seeds: a and A by or_seeds' rule; b and B fix only infinity,  */
/* so they take the fixed point of the parabolic commutator a b A B, a     */
/* finite limit point.                                                     */

static mat2 mat_mul(mat2 x, mat2 y) {
  mat2 o;
  o.p = cx_add(cx_mul(x.p, y.p), cx_mul(x.q, y.r));
  o.q = cx_add(cx_mul(x.p, y.q), cx_mul(x.q, y.s));
  o.r = cx_add(cx_mul(x.r, y.p), cx_mul(x.s, y.r));
  o.s = cx_add(cx_mul(x.r, y.q), cx_mul(x.s, y.s));
  return o;
}

OR_EXPORT int or_maskit(double mu_re, double mu_im, double* gens, double* seeds) {
  cx i = cx_make(0.0, 1.0), mu = cx_make(mu_re, mu_im);
  mat2 a, b;
  a.p = cx_mul(i, mu); a.q = i; a.r = i; a.s = cx_make(0.0, 0.0);
  b.p = cx_make(1.0, 0.0); b.q = cx_make(2.0, 0.0); b.r = cx_make(0.0, 0.0);
  b.s = cx_make(1.0, 0.0);
  mat2 all[4];
  all[0] = a; all[1] = b; all[2] = mat_inverse_unimodular(a); all[3] = mat_inverse_unimodular(b);
  for (int x = 0; x < 4; ++x) mat_store(&all[x], gens + 8 * x);
  /* seeds of a and A: or_seeds on a generator list whose b slots repeat a */
  double tmp[32], s4[8];
  for (int x = 0; x < 4; ++x) mat_store(&all[x & 2], tmp + 8 * x);
  if (or_seeds(tmp, s4) != 0) return -1;
  seeds[0] = s4[0]; seeds[1] = s4[1]; seeds[4] = s4[4]; seeds[5] = s4[5];
  mat2 k = mat_mul(mat_mul(all[0], all[1]), mat_mul(all[2], all[3]));
  if (k.r.re == 0.0 && k.r.im == 0.0) return -1;
  cx zk = cx_div(cx_sub(k.p, k.s), cx_scale(k.r, 2.0));
  seeds[2] = seeds[6] = zk.re;
  seeds[3] = seeds[7] = zk.im;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Seeds for multi-seed feeding (the paper's loop over a list of fixed       */
/* points, Sec. "Implementation").  The list it cites is not in the paper;   */
/* this oracle takes the attracting fixed points of a, b, A, B and the fixed */
/* points of the four cyclic permutations of the commutator, abAB, bABa,     */
/* ABab and BabA: parabolic maps of a once-punctured torus group, whose      */
/* fixed points are the cusps of the limit set.  out: 8 points (16 doubles). */

static mat2 word_matrix4(const mat2* g, const int* w) {
  mat2 m = g[w[0]];
  for (int k = 1; k < 4; ++k) m = mat_mul(m, g[w[k]]);
  return m;
}

OR_EXPORT int or_cusp_seeds(const double* gens, double* out) {
  if (or_seeds(gens, out) != 0) return -1;
  mat2 g[4];
  for (int x = 0; x < 4; ++x) g[x] = mat_load(gens + 8 * x);
  /* a=0, b=1, A=2, B=3: abAB and its cyclic permutations */
  static const int perms[4][4] = {{0, 1, 2, 3}, {1, 2, 3, 0}, {2, 3, 0, 1}, {3, 0, 1, 2}};
  for (int c = 0; c < 4; ++c) {
    mat2 k = word_matrix4(g, perms[c]);
    if (k.r.re == 0.0 && k.r.im == 0.0) return -1;
    cx z = cx_div(cx_sub(k.p, k.s), cx_scale(k.r, 2.0)); /* double root of a parabolic map */
    out[8 + 2 * c] = z.re;
    out[8 + 2 * c + 1] = z.im;
  }
  return 0;
}
