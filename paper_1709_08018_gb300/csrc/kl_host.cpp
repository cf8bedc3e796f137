// Host-side part of the C ABI: status strings, word counts, generators from
// traces (Grandma's recipe), seeds, Maskit's slice group, the cusp seed list
// of multi-seed feeding and parameter defaults.  No GPU is needed for
// anything in this file.
#include <cmath>
#include <complex>
#include <cstring>

#include "kl.h"

namespace {

using cplx = std::complex<double>;

struct Mobius {
  cplx p, q, r, s;  // z -> (p z + q) / (r z + s)
};

void put(const Mobius& m, double* dst) {
  const cplx v[4] = {m.p, m.q, m.r, m.s};
  for (int k = 0; k < 4; ++k) {
    dst[2 * k] = v[k].real();
    dst[2 * k + 1] = v[k].imag();
  }
}

Mobius get(const double* src) {
  Mobius m;
  m.p = cplx(src[0], src[1]);
  m.q = cplx(src[2], src[3]);
  m.r = cplx(src[4], src[5]);
  m.s = cplx(src[6], src[7]);
  return m;
}

// For a matrix of determinant one the inverse map is the adjugate.
Mobius inverse(const Mobius& m) { return Mobius{m.s, -m.q, -m.r, m.p}; }

bool finite(cplx z) { return std::isfinite(z.real()) && std::isfinite(z.imag()); }

}  // namespace

extern "C" const char* kl_status_string(int status) {
  switch (status) {
    case KL_OK: return "ok";
    case KL_EINVAL: return "invalid argument";
    case KL_ERANGE: return "value out of range";
    case KL_ECUDA: return "CUDA error";
    case KL_ENOSPACE: return "workspace too small";
    case KL_EDEGENERATE: return "degenerate group";
    default: return "unknown status";
  }
}

extern "C" uint64_t kl_word_count(uint32_t depth) {
  if (depth < 1 || depth > KL_MAX_DEPTH) return 0;
  uint64_t n = 4;
  for (uint32_t k = 1; k < depth; ++k) n *= 3;
  return n;
}

// Grandma's recipe.  tr(ab) = tab solves tab^2 - ta tb tab + ta^2 + tb^2 = 0,
// which is what makes the commutator trace -2 (a once-punctured torus); the
// root with the minus sign is taken.  With z0 = (tab - 2) tb / (tb tab - 2 ta + 2i tab):
//   a = [[ta/2, (ta tab - 2 tb + 4i) / ((2 tab + 4) z0)],
//        [(ta tab - 2 tb - 4i) z0 / (2 tab - 4), ta/2]],
//   b = [[(tb - 2i)/2, tb/2], [tb/2, (tb + 2i)/2]].
extern "C" int kl_grandma(double ta_re, double ta_im, double tb_re, double tb_im,
                          double* gens_out) {
  if (!gens_out) return KL_EINVAL;
  const cplx ta(ta_re, ta_im), tb(tb_re, tb_im);
  if (!finite(ta) || !finite(tb)) return KL_EINVAL;
  const cplx I(0.0, 1.0);
  const cplx disc = ta * ta * tb * tb - 4.0 * (ta * ta + tb * tb);
  const cplx tab = 0.5 * (ta * tb - std::sqrt(disc));
  const cplx z0_den = tb * tab - 2.0 * ta + 2.0 * I * tab;
  const cplx lower_den = 2.0 * tab - 4.0;
  if (std::abs(z0_den) == 0.0 || std::abs(lower_den) == 0.0) return KL_EDEGENERATE;
  const cplx z0 = (tab - 2.0) * tb / z0_den;
  const cplx upper_den = (2.0 * tab + 4.0) * z0;
  if (std::abs(upper_den) == 0.0) return KL_EDEGENERATE;
  const cplx k = ta * tab - 2.0 * tb;
  Mobius a{0.5 * ta, (k + 4.0 * I) / upper_den, (k - 4.0 * I) * z0 / lower_den, 0.5 * ta};
  Mobius b{0.5 * (tb - 2.0 * I), 0.5 * tb, 0.5 * tb, 0.5 * (tb + 2.0 * I)};
  const Mobius all[4] = {a, b, inverse(a), inverse(b)};
  for (int x = 0; x < 4; ++x) {
    if (!finite(all[x].p) || !finite(all[x].q) || !finite(all[x].r) || !finite(all[x].s))
      return KL_EDEGENERATE;
    put(all[x], gens_out + 8 * x);
  }
  return KL_OK;
}

namespace {

// Attracting fixed point of m.  Fixed points solve r z^2 + (s - p) z - q = 0;
// since |M'(z)| = 1 / |r z + s|^2 for det 1, the attracting one maximises
// |r z + s|.  Equal values (a parabolic map, double root) take the "+" root.
// r = 0: the finite fixed point q / (s - p), which attracts only if |p| < |s|.
int attracting_fixed_point(const Mobius& m, cplx* out) {
  cplx z;
  if (m.r == cplx(0.0, 0.0)) {
    if (!(std::abs(m.p) < std::abs(m.s))) return KL_EDEGENERATE;
    z = m.q / (m.s - m.p);
  } else {
    const cplx h = m.p - m.s;
    const cplx root = std::sqrt(h * h + 4.0 * m.q * m.r);
    const cplx plus = (h + root) / (2.0 * m.r);
    const cplx minus = (h - root) / (2.0 * m.r);
    z = std::abs(m.r * minus + m.s) > std::abs(m.r * plus + m.s) ? minus : plus;
  }
  if (!finite(z)) return KL_EDEGENERATE;
  *out = z;
  return KL_OK;
}

Mobius compose(const Mobius& x, const Mobius& y) {  // x after y
  return Mobius{x.p * y.p + x.q * y.r, x.p * y.q + x.q * y.s, x.r * y.p + x.s * y.r,
                x.r * y.q + x.s * y.s};
}

}  // namespace

extern "C" int kl_seeds(const double* gens, double* seeds_out) {
  if (!gens || !seeds_out) return KL_EINVAL;
  for (int x = 0; x < 4; ++x) {
    cplx z;
    const int st = attracting_fixed_point(get(gens + 8 * x), &z);
    if (st != KL_OK) return st;
    seeds_out[2 * x] = z.real();
    seeds_out[2 * x + 1] = z.imag();
  }
  return KL_OK;
}

// Maskit's slice (Mumford-Series-Wright, "Indra's Pearls", ch. 9): a(z) =
// mu + 1/z and b(z) = z + 2, i.e. a = [[-i mu, -i], [-i, 0]] and
// b = [[1, 2], [0, 1]], both of determinant one, with tr(a b A B) = -2 for
// every mu (a once-punctured torus group when discrete).  Seeds: a and A as
// kl_seeds; b and B fix only infinity, so their words start from the fixed
// point of the parabolic commutator a b A B instead, a finite point of the
// limit set (fixed points of parabolic elements are limit points).
extern "C" int kl_maskit(double mu_re, double mu_im, double* gens_out, double* seeds_out) {
  if (!gens_out || !seeds_out) return KL_EINVAL;
  const cplx mu(mu_re, mu_im), I(0.0, 1.0);
  if (!finite(mu)) return KL_EINVAL;
  const Mobius a{-I * mu, -I, -I, cplx(0.0, 0.0)};
  const Mobius b{cplx(1.0, 0.0), cplx(2.0, 0.0), cplx(0.0, 0.0), cplx(1.0, 0.0)};
  const Mobius all[4] = {a, b, inverse(a), inverse(b)};
  for (int x = 0; x < 4; ++x) put(all[x], gens_out + 8 * x);
  for (int x = 0; x < 4; x += 2) {
    cplx z;
    const int st = attracting_fixed_point(all[x], &z);
    if (st != KL_OK) return st;
    seeds_out[2 * x] = z.real();
    seeds_out[2 * x + 1] = z.imag();
  }
  const Mobius k = compose(compose(a, b), compose(all[2], all[3]));
  if (k.r == cplx(0.0, 0.0)) return KL_EDEGENERATE;
  const cplx zk = (k.p - k.s) / (2.0 * k.r);  // the double root of a parabolic map
  if (!finite(zk)) return KL_EDEGENERATE;
  for (int x = 1; x < 4; x += 2) {
    seeds_out[2 * x] = zk.real();
    seeds_out[2 * x + 1] = zk.imag();
  }
  return KL_OK;
}

extern "C" int kl_params_init(kl_params* p, double ta_re, double ta_im, double tb_re,
                              double tb_im, uint32_t depth, uint32_t width, uint32_t height,
                              double x0, double x1, double y0, double y1) {
  if (!p) return KL_EINVAL;
  std::memset(p, 0, sizeof(*p));
  int st = kl_grandma(ta_re, ta_im, tb_re, tb_im, p->gens);
  if (st != KL_OK) return st;
  st = kl_seeds(p->gens, p->seeds);
  if (st != KL_OK) return st;
  p->depth = depth;
  p->width = width;
  p->height = height;
  p->x0 = x0;
  p->x1 = x1;
  p->y0 = y0;
  p->y1 = y1;
  p->precision = KL_FP64;
  p->renorm_every = 8;
  p->parabolic_tol = 1e-6;
  p->prefix_len = 0;
  p->accumulate = 0;
  p->mode = KL_LIMIT_SET;
  p->cull = 0;
  return KL_OK;
}

// Seed list for multi-seed feeding: the attracting fixed points of a, b, A, B
// (as kl_seeds), then the fixed points of the commutator a b A B and of its
// cyclic permutations b A B a, A B a b, B a b A.  Those four are parabolic
// (trace -2), so each fixed point is the double root (p - s) / (2 r).
extern "C" int kl_cusp_seeds(const double* gens, double* seeds_out) {
  if (!gens || !seeds_out) return KL_EINVAL;
  int st = kl_seeds(gens, seeds_out);
  if (st != KL_OK) return st;
  Mobius m[4];
  for (int x = 0; x < 4; ++x) m[x] = get(gens + 8 * x);
  for (int c = 0; c < 4; ++c) {
    // the word of letters c, c+1, c+2, c+3 (mod 4) of a b A B
    Mobius k = m[c];
    for (int j = 1; j < 4; ++j) k = compose(k, m[(c + j) & 3]);
    if (k.r == cplx(0.0, 0.0)) return KL_EDEGENERATE;
    const cplx z = (k.p - k.s) / (2.0 * k.r);
    if (!finite(z)) return KL_EDEGENERATE;
    seeds_out[8 + 2 * c] = z.real();
    seeds_out[8 + 2 * c + 1] = z.imag();
  }
  return KL_OK;
}
