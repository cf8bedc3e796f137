// Double-float arithmetic (values as unevaluated sums hi + lo of two floats)
// on the FP32 pipe: the packed per-word map of the KL_DF64 render and the
// scalar forms used by the level-of-detail expansion.  Included at the end
// of kl_common.cuh.
#pragma once

#include "kl_common.cuh"

namespace {

// ---------------------------------------------------------------------------
// double-float per-word map (KL_DF64), two words per packed f32x2 instruction
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2
// (Dekker 1971; the "double-double" arithmetic of Hida, Li and Bailey 2001,
// here on floats): about 48 significant bits.  Sums use Knuth's two-sum and
// Dekker's fast two-sum; products use the fused multiply-add for the exact
// rounding error of hi * hi.  Every operation below is an FP32 add, multiply
// or fused multiply-add, so the map runs on the FP32 pipe.

__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// both halves negated (their sign bits flipped; an integer operation)
__device__ __forceinline__ f2 neg2(f2 a) { return a ^ 0x8000000080000000ull; }

struct DD {
  f2 hi, lo;
};

// s + e = a + b exactly (two-sum)
__device__ __forceinline__ void two_sum2(f2 a, f2 b, f2& s, f2& e) {
  s = add2(a, b);
  const f2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (fast two-sum)
__device__ __forceinline__ void fast_two_sum2(f2 a, f2 b, f2& s, f2& e) {
  s = add2(a, b);
  e = sub2(b, sub2(s, a));
}
__device__ __forceinline__ DD dd_add(const DD& a, const DD& b) {
  f2 s, e;
  two_sum2(a.hi, b.hi, s, e);
  e = add2(e, add2(a.lo, b.lo));
  DD r;
  fast_two_sum2(s, e, r.hi, r.lo);
  return r;
}
// 1/m: the hardware seed y (about 2^-23) and one Newton step y + y (1 - m y),
// with the residual 1 - m y formed from the exact product m.hi y: about 2^-46.
// The result is left as the pair (y, y (1 - m y)) without renormalising: its
// low part is below 2^-22 of the high part, which is all that its one use,
// the products of dd_fma, needs.  7 operations.
__device__ __forceinline__ DD dd_rcp(const DD& m) {
  float ma, mb;
  upk(m.hi, ma, mb);
  const f2 y = pk(rcp32(ma), rcp32(mb));
  const f2 one = 0x3F8000003F800000ull;
  const f2 p = mul2(m.hi, y);
  const f2 pe = fma2(m.hi, y, neg2(p));       // m.hi y = p + pe
  const f2 res = sub2(sub2(sub2(one, p), pe), mul2(m.lo, y));
  return DD{y, mul2(y, res)};
}

// a1 b1 + a2 b2 as one sequence: the two high products and their exact
// errors, an exact sum of the products, then the cross terms added to the
// error before one renormalisation (19 operations against 25 for two
// products and a sum; the same error order, about 2^-48 of |a1 b1| + |a2 b2|)
__device__ __forceinline__ DD dd_dot(const DD& a1, const DD& b1, const DD& a2, const DD& b2) {
  const f2 p1 = mul2(a1.hi, b1.hi), p2 = mul2(a2.hi, b2.hi);
  const f2 e1 = fma2(a1.hi, b1.hi, neg2(p1)), e2 = fma2(a2.hi, b2.hi, neg2(p2));
  f2 s, e;
  two_sum2(p1, p2, s, e);
  e = add2(e, add2(e1, e2));
  e = fma2(a1.hi, b1.lo, e);
  e = fma2(a1.lo, b1.hi, e);
  e = fma2(a2.hi, b2.lo, e);
  e = fma2(a2.lo, b2.hi, e);
  DD r;
  fast_two_sum2(s, e, r.hi, r.lo);
  return r;
}
// |w|^2 = wr^2 + wi^2 in the same way, left unrenormalised: both products are
// >= 0, so nothing cancels and the low part stays within a few ulp of the
// high part, which is all dd_rcp needs (16 operations)
__device__ __forceinline__ DD dd_norm2(const DD& wr, const DD& wi) {
  const f2 p1 = mul2(wr.hi, wr.hi), p2 = mul2(wi.hi, wi.hi);
  const f2 e1 = fma2(wr.hi, wr.hi, neg2(p1)), e2 = fma2(wi.hi, wi.hi, neg2(p2));
  f2 s, e;
  two_sum2(p1, p2, s, e);
  e = add2(e, add2(e1, e2));
  e = fma2(add2(wr.hi, wr.hi), wr.lo, e);
  e = fma2(add2(wi.hi, wi.hi), wi.lo, e);
  return DD{s, e};
}
// a + b c: the product's high part summed exactly with a.hi, its error and
// cross terms and a.lo added before one renormalisation (15 against 18)
__device__ __forceinline__ DD dd_fma(const DD& a, const DD& b, const DD& c) {
  const f2 p = mul2(b.hi, c.hi);
  f2 e = fma2(b.hi, c.hi, neg2(p));
  e = fma2(b.hi, c.lo, e);
  e = fma2(b.lo, c.hi, e);
  f2 s, f;
  two_sum2(a.hi, p, s, f);
  f = add2(f, add2(e, a.lo));
  DD r;
  fast_two_sum2(s, f, r.hi, r.lo);
  return r;
}

// Pole-form constants of a prefix as double-floats, each in both halves.
struct DfConst {
  DD k[8];  // gr, gi, ax, ay, c1, c2, c3, c4
};
__device__ __forceinline__ DfConst df_const(const PreDF& c) {
  DfConst K;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    K.k[q].hi = pk(c.h[q], c.h[q]);
    K.k[q].lo = pk(c.l[q], c.l[q]);
  }
  return K;
}

// Pixel coordinates (u, v) of two words with suffix points (vr, vi):
// u = ax + (c1 wr + c2 wi) / |w|^2, v = ay + (c3 wr + c4 wi) / |w|^2, w = v + gamma.
__device__ __forceinline__ void uv_df2(const DfConst& K, const DD& vr, const DD& vi, DD& u,
                                       DD& v) {
  const DD wr = dd_add(vr, K.k[0]);
  const DD wi = dd_add(vi, K.k[1]);
  const DD r = dd_rcp(dd_norm2(wr, wi));
  const DD tx = dd_dot(K.k[4], wr, K.k[5], wi);
  const DD ty = dd_dot(K.k[6], wr, K.k[7], wi);
  u = dd_fma(K.k[2], tx, r);
  v = dd_fma(K.k[3], ty, r);
}

// Pixel keys 0x4B400000 + floor(u) of two double-float coordinates: floor
// of u.hi from its rounding toward minus infinity after adding 1.5 2^23, less
// one where u.lo takes u below that integer.  That happens exactly when u.hi
// is an integer and u.lo < 0: a non-integral u.hi lies at least ulp(u.hi)
// from the integers on both sides, farther than |u.lo| <= ulp(u.hi)/2.  The
// tests are on the bits (u.hi equal to its floor; u.lo negative, -0 not).
// As for the mixed path, any |u| >= 2^22, infinity or NaN gives a key whose
// column or row falls outside the image.
__device__ __forceinline__ void floor_keys(const DD& u, uint32_t& ka, uint32_t& kb) {
  const f2 magic = 0x4B4000004B400000ull;
  const f2 t = add2_rm(u.hi, magic);
  const f2 fl = sub2(t, magic);  // floor(u.hi), exactly
  const bool da = ((uint32_t)fl == (uint32_t)u.hi) & ((uint32_t)u.lo > 0x80000000u);
  const bool db = ((uint32_t)(fl >> 32) == (uint32_t)(u.hi >> 32)) &
                  ((uint32_t)(u.lo >> 32) > 0x80000000u);
  ka = (uint32_t)t - (da ? 1u : 0u);
  kb = (uint32_t)(t >> 32) - (db ? 1u : 0u);
}

// One run of n words ending in the pixel of keys (cu, cv) (absolute pixel
// keys: col = cu - 0x4B400000).
__device__ __forceinline__ void flush_key(uint32_t cu, uint32_t cv, uint32_t n, const View& V,
                                          Tally& t, uint32_t* __restrict__ img) {
  const uint32_t col = cu - 0x4B400000u, row = cv - 0x4B400000u;
  if (n && col < V.W && row < V.H) {
    atomicAdd(img + row * V.W + col, n);
    ++t.atomics;
    t.in_window += n;
  }
}

// Double-float words of prefix slot `slot` on suffix point pairs [k0, k1) of
// first letter u, with the run-length splat of mixed_slot_words on pixel keys.
__device__ __forceinline__ void df64_slot_words(uint32_t slot, int u, uint32_t k0, uint32_t k1,
                                                const Plan& L, const View& V, const Tables& T,
                                                Tally& t, uint32_t& words,
                                                uint32_t* __restrict__ img) {
  const DfConst K = df_const(T.predf[slot]);
  const float4* src = T.sufdf + 2ull * (size_t)u * L.npairs;
  t.flush(img);
  t.cur = -1;
  uint32_t cu = 0, cv = 0, run = 0;  // keys (0, 0): no in-window pixel
  uint32_t e_run = k0;
  for (uint32_t e = k0; e < k1; ++e) {
    const float4 a = __ldg(src + 2 * e), b = __ldg(src + 2 * e + 1);
    const DD vr = {pk(a.x, a.y), pk(a.z, a.w)}, vi = {pk(b.x, b.y), pk(b.z, b.w)};
    DD U, Vv;
    uv_df2(K, vr, vi, U, Vv);
    uint32_t ua, ub, va, vb;
    floor_keys(U, ua, ub);
    floor_keys(Vv, va, vb);
    if (!((ua == cu) & (ub == cu) & (va == cv) & (vb == cv))) {
      const bool a_in = (ua == cu) & (va == cv);
      const bool ab = (ua == ub) & (va == vb);
      run += 2u * (e - e_run) + (a_in ? 1u : 0u);
      e_run = e + 1;
      flush_key(cu, cv, run, V, t, img);
      if (!a_in && !ab) flush_key(ua, va, 1u, V, t, img);  // word a on its own
      run = (!a_in && ab) ? 2u : 1u;
      cu = ub;
      cv = vb;
    }
  }
  run += 2u * (k1 - e_run);
  flush_key(cu, cv, run, V, t, img);
  words += min(2u * k1, L.ns) - 2u * k0;
}

// One double-float item: this thread's prefix on one chunk of suffix pairs.
template <int BT>
__device__ __forceinline__ void df64_item(uint32_t item, const Work& Wk, const Plan& L,
                                          const View& V, const Tables& T, Tally& t,
                                          uint32_t& words, uint32_t* __restrict__ img) {
  int x, u;
  uint32_t pb, c;
  item_of(item, Wk, x, u, pb, c);
  const uint32_t k = pb * BT + (threadIdx.x % BT);
  if (k >= L.nr) return;
  const uint32_t slot = (uint32_t)x * L.np + L.r0 + k;
  if (T.flags[slot] & kFallback) return;
  const uint32_t k0 = c * Wk.chunk, k1 = min(L.npairs, k0 + Wk.chunk);
  df64_slot_words(slot, u, k0, k1, L, V, T, t, words, img);
}

// ---------------------------------------------------------------------------
// scalar double-floats: one value per thread (the level-of-detail expansion,
// where each lane holds its own node matrix).  The same arithmetic as the
// packed pairs above.

struct D1 {
  float hi, lo;
};

__device__ __forceinline__ D1 d1_of(double d) {
  D1 r;
  split_df(d, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ D1 d1_neg(D1 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ void two_sum1(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ D1 fast_two_sum1(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ D1 d1_add(D1 a, D1 b) {
  float s, e;
  two_sum1(a.hi, b.hi, s, e);
  return fast_two_sum1(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ D1 d1_mul(D1 a, D1 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum1(p, e);
}
// sum of N products a_i b_i: high products and their exact errors, an exact
// running sum of the products, the cross terms, one renormalisation
template <int N>
__device__ __forceinline__ D1 d1_dot(const D1 (&a)[N], const D1 (&b)[N]) {
  float s = __fmul_rn(a[0].hi, b[0].hi);
  float e = __fmaf_rn(a[0].hi, b[0].hi, -s);
#pragma unroll
  for (int i = 1; i < N; ++i) {
    const float p = __fmul_rn(a[i].hi, b[i].hi);
    e = __fadd_rn(e, __fmaf_rn(a[i].hi, b[i].hi, -p));
    float t;
    two_sum1(s, p, s, t);
    e = __fadd_rn(e, t);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    e = __fmaf_rn(a[i].hi, b[i].lo, e);
    e = __fmaf_rn(a[i].lo, b[i].hi, e);
  }
  return fast_two_sum1(s, e);
}
// 1/m: hardware seed and one Newton step with the residual from m.hi y exactly
__device__ __forceinline__ D1 d1_rcp(D1 m) {
  const float y = rcp32(m.hi);
  const float p = __fmul_rn(m.hi, y);
  const float pe = __fmaf_rn(m.hi, y, -p);
  const float res = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), pe), __fmul_rn(m.lo, y));
  return fast_two_sum1(y, __fmul_rn(y, res));
}

struct C1 {
  D1 re, im;
};
struct M1 {
  C1 p, q, r, s;
};

__device__ __forceinline__ M1 m1_of(const M2& a) {
  return {{d1_of(a.p.re), d1_of(a.p.im)}, {d1_of(a.q.re), d1_of(a.q.im)},
          {d1_of(a.r.re), d1_of(a.r.im)}, {d1_of(a.s.re), d1_of(a.s.im)}};
}
// a b + c d (complex), each part one 4-term dot product
__device__ __forceinline__ C1 c1_mul_add(C1 a, C1 b, C1 c, C1 d) {
  const D1 xr[4] = {a.re, d1_neg(a.im), c.re, d1_neg(c.im)};
  const D1 yr[4] = {b.re, b.im, d.re, d.im};
  const D1 xi[4] = {a.re, a.im, c.re, c.im};
  const D1 yi[4] = {b.im, b.re, d.im, d.re};
  return {d1_dot<4>(xr, yr), d1_dot<4>(xi, yi)};
}
__device__ __forceinline__ M1 m1_mul(const M1& a, const M1& b) {
  return {c1_mul_add(a.p, b.p, a.q, b.r), c1_mul_add(a.p, b.q, a.q, b.s),
          c1_mul_add(a.r, b.p, a.s, b.r), c1_mul_add(a.r, b.q, a.s, b.s)};
}
// a v + b (complex)
__device__ __forceinline__ C1 c1_affine(C1 a, C1 v, C1 b) {
  const D1 one = {1.0f, 0.0f};
  const D1 xr[3] = {a.re, d1_neg(a.im), b.re};
  const D1 yr[3] = {v.re, v.im, one};
  const D1 xi[3] = {a.re, a.im, b.im};
  const D1 yi[3] = {v.im, v.re, one};
  return {d1_dot<3>(xr, yr), d1_dot<3>(xi, yi)};
}
// P(v) = (p v + q) / (r v + s) as n conj(m) / |m|^2
__device__ __forceinline__ C1 m1_apply(const M1& P, C1 v) {
  const C1 n = c1_affine(P.p, v, P.q), m = c1_affine(P.r, v, P.s);
  const D1 mm[2] = {m.re, m.im};
  const D1 k = d1_rcp(d1_dot<2>(mm, mm));
  const D1 ar[2] = {n.re, n.im}, br[2] = {m.re, m.im};
  const D1 ai[2] = {n.im, d1_neg(n.re)}, bi[2] = {m.re, m.im};
  return {d1_mul(d1_dot<2>(ar, br), k), d1_mul(d1_dot<2>(ai, bi), k)};
}

}  // namespace
