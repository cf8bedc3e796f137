// Shared device code of the indexed limit-set renderer (sm_103a): data
// layouts, the per-word arithmetic, the table builders and the per-item render
// bodies used by both the single render (kl_render.cu) and the batched render
// (kl_batch.cu).
//
// A reduced word w_1 .. w_d is split into a prefix w_1 .. w_p (the letters
// applied last) and a suffix w_{p+1} .. w_d (applied first, starting from the
// seed of w_d).  Its value is P(v): P = M_{w_1} ... M_{w_p} is the prefix
// matrix and v the suffix point.  The index of the word factors the same
// way: i = (prefix index) * 3^s + (suffix digits), so instead of decoding i
// digit by digit for every word, the kernels decode each prefix once (a table
// of prefix constants) and each suffix once (a table of suffix points) and
// enumerate the compatible pairs (suffix first letter != inverse of the prefix
// last letter, Sec. "Once-punctured torus groups").
//
// Per word the only work left is one linear-fractional map and a splat.  With
// det P = D the map is written in pole form
//     P(v) = alpha + beta / (v + gamma),
//     alpha = P00/P10, gamma = P11/P10, beta = -D/P10^2,
// and folded into pixel units, u = (Re z - x0) sx = ax + (c1 wr + c2 wi)/|w|^2,
// row coordinate v = (y1 - Im z) sy = ay + (c3 wr + c4 wi)/|w|^2, w = v + gamma:
// 13 FP64 operations and one reciprocal seed per word.  Pixel binning uses
// only integer operations.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "kl.h"

namespace {

constexpr int kMaxPrefix = 15;
constexpr int kMaxPlainSuffix = 9;  // suffix letters of the default per-word plans
constexpr int kMaxSuffix = 12;      // of culled plans and of a caller's prefix_len
constexpr int kMaxRenderDepth = kMaxPrefix + kMaxPlainSuffix;
constexpr int kDefaultThreads = 128;
constexpr int kMaxCullLevels = 8;

// Prefix flags.
constexpr uint32_t kDirect = 1u;     // P10 ~ 0: pole form invalid, use the direct map
constexpr uint32_t kNearPar = 2u;    // |tr^2 - 4 det| small: near-parabolic (cusp) prefix
constexpr uint32_t kWide = 4u;       // local FP32 frame unsafe (far or huge offsets)
constexpr uint32_t kFallback = 8u;   // KL_MIXED, KL_DF64: words of this prefix run in FP64
constexpr uint32_t kDfRange = 16u;   // a pole-form constant outside the double-float range

// FP64 fallback work unit: a chunk of this many suffix points.
constexpr uint32_t kFbChunk = 64;

struct Plan {
  int d, p, s;
  int q;         // letters of the prefix tail table (the rest, p - q, in the head table)
  int so, si;    // letters of the suffix head (matrix) and tail (point) tables
  uint32_t np;   // prefix slots per last letter: 3^(p-1)
  uint32_t ns;   // suffix points per first letter: 3^(s-1)
  uint32_t npairs;  // FP32 point pairs per first letter: ceil(ns / 2)
  // prefix slots this render draws, per last letter: [r0, r0 + nr) (a shard of
  // kl_params.shard_count > 1; else all np); tables and work cover only these
  uint32_t r0, nr;
  uint32_t p3_q1, p3_pq, p3_so1, p3_si, p3_si1;  // 3^(q-1), 3^(p-q), 3^(so-1), 3^si, 3^(si-1)
  // culling blocks (kl_params.cull): level l = 0 .. clev-1 holds aligned blocks
  // of csz[l] = 3^(cj0 + l) suffix points (one subtree each), cnb[l] = ns /
  // csz[l] of them per first letter, their disks from index cdisk[l] on
  uint32_t cj0, clev, ndisks;
  uint32_t csz[kMaxCullLevels], cnb[kMaxCullLevels], cdisk[kMaxCullLevels];
  size_t off_pre64, off_pre32, off_flags, off_suf64, off_suf32, off_fb, off_fbcount;
  size_t off_L, off_H, off_So, off_Si, off_disk32, off_disk64, off_nrm32, off_nrm64;
  size_t off_predf, off_sufdf, total;
};

struct View {
  double x0, y1, sx, sy;
  uint32_t W, H;
  uint32_t hiW, hiH;  // high words of (double)W and (double)H
};

struct Group {
  double g[32];
  double seed[8];
};

struct __align__(16) Pre64 {
  double gr, gi, ax, ay, c1, c2, c3, c4;  // pole form; or P00..P11 (re, im) if kDirect
};

struct __align__(16) Pre32 {
  float gr, gi, axf, ayf, c1, c2, c3, c4;
  int axi, ayi;  // integer part of the pixel coordinates of alpha
  int kx, ky;    // 0x4B400000 - axi, 0x4B400000 - ayi (see mixed_item)
};

// Pole-form constants of one prefix as double-floats (KL_DF64): each FP64
// constant d as hi = fl32(d), lo = fl32(d - hi), in the order gr, gi, ax,
// ay, c1, c2, c3, c4 (ax, ay: pixel coordinates of alpha, no local frame).
struct __align__(16) PreDF {
  float h[8], l[8];
};

// Disk bounding one culling block of suffix points (FP64 points).
struct __align__(16) Disk64 {
  double cr, ci, rho, pad;
};

struct dc {
  double re, im;
};

struct M2 {
  dc p, q, r, s;
};

struct __align__(16) PartM {
  M2 m;
  int edge;  // L: its outermost letter w_{p-q+1}; So: its innermost letter w_{p+so}
  int pad[3];
};

// Device tables of one render, carved from the caller's workspace.
struct Tables {
  Pre64* pre64;
  Pre32* pre32;
  uint32_t* flags;
  double2* suf64;
  float4* suf32p;
  unsigned long long* fb;  // fallback entries: (group << 32) | prefix slot
  uint32_t* fbcount;       // [0] fallback entries, [1] work-queue head
  PartM* Lt;
  M2* Ht;
  PartM* Sot;
  double2* Sit;
  float4* disk32;  // per culling block: center (x, y) and radius (z) of the FP32 points
  Disk64* disk64;  // the same for the FP64 points
  float* nrm32;    // per prefix slot: operator norm of the FP32 pole-form matrix
  double* nrm64;   // the same in FP64
  PreDF* predf;    // KL_DF64: per prefix slot, the pole-form constants as double-floats
  float4* sufdf;   // KL_DF64: per suffix point pair (a, b) two float4s:
                   // (re_hi a, re_hi b, re_lo a, re_lo b), (im_hi a, im_hi b, im_lo a, im_lo b)
};

// Work items of the persistent render kernels: item = (q, prefix block pb,
// suffix chunk c), chunk index fastest.  q = 3 x + k enumerates the 12
// compatible (prefix last letter x, suffix first letter u) pairs, u being the
// k-th letter other than inv(x); thread t of the block takes prefix slot
// (x, pb * BT + t) and the chunk's suffix points.
struct Work {
  uint32_t n_pb;      // prefix blocks per letter: ceil(np / BT)
  uint32_t n_chunks;  // suffix chunks per first letter
  uint32_t chunk;     // suffix points (FP64) or point pairs (FP32) per chunk
  uint32_t n_items;   // 12 * n_pb * n_chunks
};

// Per-prefix boxes of all words of a prefix's subtree (level-of-detail
// labels), in fixed point: pixel coordinates times 256, floored, saturated to
// +-2^30 for far words.
struct BoxRef {
  int* cmin;
  int* cmax;
  int* rmin;
  int* rmax;
};

// ---------------------------------------------------------------------------
// complex FP64 helpers (tables only; the per-word code spells out its ops)

__device__ __forceinline__ dc cadd(dc a, dc b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ dc csub(dc a, dc b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ dc cmul(dc a, dc b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ dc cdiv(dc n, dc m) {
  double den = m.re * m.re + m.im * m.im;
  return {(n.re * m.re + n.im * m.im) / den, (n.im * m.re - n.re * m.im) / den};
}
__device__ __forceinline__ double cabs1(dc a) { return fabs(a.re) + fabs(a.im); }
// principal square root
__device__ __forceinline__ dc csqrt(dc a) {
  double r = hypot(a.re, a.im);
  if (r == 0.0) return {0.0, 0.0};
  double t = sqrt(0.5 * (r + fabs(a.re)));
  if (a.re >= 0.0) return {t, a.im / (2.0 * t)};
  return {fabs(a.im) / (2.0 * t), copysign(t, a.im)};
}
// 1/z for z != 0: conj(z) / |z|^2 with one real division
__device__ __forceinline__ dc crcp(dc z) {
  const double t = 1.0 / (z.re * z.re + z.im * z.im);
  return {z.re * t, -z.im * t};
}

__device__ __forceinline__ M2 load_gen(const Group& G, int x) {
  const double* g = G.g + 8 * x;
  return {{g[0], g[1]}, {g[2], g[3]}, {g[4], g[5]}, {g[6], g[7]}};
}
__device__ __forceinline__ M2 mmul(const M2& a, const M2& b) {
  return {cadd(cmul(a.p, b.p), cmul(a.q, b.r)), cadd(cmul(a.p, b.q), cmul(a.q, b.s)),
          cadd(cmul(a.r, b.p), cmul(a.s, b.r)), cadd(cmul(a.r, b.q), cmul(a.s, b.s))};
}
__device__ __forceinline__ dc mdet(const M2& a) { return csub(cmul(a.p, a.s), cmul(a.q, a.r)); }
// divide by the principal square root of the determinant
__device__ __forceinline__ void renormalise(M2& a) {
  dc k = csqrt(mdet(a));
  if (k.re == 0.0 && k.im == 0.0) return;
  k = crcp(k);
  a.p = cmul(a.p, k); a.q = cmul(a.q, k); a.r = cmul(a.r, k); a.s = cmul(a.s, k);
}
__device__ __forceinline__ M2 identity2() {
  return {{1.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {1.0, 0.0}};
}
__device__ __forceinline__ dc mobius(const M2& m, dc z) {
  return cmul(cadd(cmul(m.p, z), m.q), crcp(cadd(cmul(m.r, z), m.s)));
}

// ---------------------------------------------------------------------------
// per-word arithmetic, shared by the render kernels and the evaluation kernel

// FP64 reciprocal: hardware seed (rcp.approx.ftz.f64) refined by one cubic
// Newton-Raphson step y <- y (1 + e + e^2), e = 1 - m y (Householder order 3).
__device__ __forceinline__ double rcp64(double m) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(m));
  double e = __fma_rn(-m, y, 1.0);
  double e2 = __fma_rn(e, e, e);
  return __fma_rn(y, e2, y);
}

__device__ __forceinline__ float rcp32(float m) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(m));
  return y;
}

__device__ __forceinline__ void uv_pole64(const Pre64& c, double vr, double vi, double& u,
                                          double& v) {
  double wr = __dadd_rn(vr, c.gr);
  double wi = __dadd_rn(vi, c.gi);
  double m = __fma_rn(wr, wr, __dmul_rn(wi, wi));
  double r = rcp64(m);
  double tx = __fma_rn(c.c1, wr, __dmul_rn(c.c2, wi));
  double ty = __fma_rn(c.c3, wr, __dmul_rn(c.c4, wi));
  u = __fma_rn(tx, r, c.ax);
  v = __fma_rn(ty, r, c.ay);
}

// Direct form for prefixes whose P10 vanishes: z = (P00 v + P01)/(P10 v + P11).
__device__ __forceinline__ void uv_direct64(const Pre64& c, double vr, double vi,
                                            const View& V, double& u, double& v) {
  dc P00 = {c.gr, c.gi}, P01 = {c.ax, c.ay}, P10 = {c.c1, c.c2}, P11 = {c.c3, c.c4};
  dc z = {vr, vi};
  dc w = cdiv(cadd(cmul(P00, z), P01), cadd(cmul(P10, z), P11));
  u = (w.re - V.x0) * V.sx;
  v = (V.y1 - w.im) * V.sy;
}

// Scalar form of the mixed per-word map (the evaluation kernel); the render
// evaluates the same operations two words at a time.
__device__ __forceinline__ void uv_pole32(const Pre32& c, float vr, float vi, float& uf,
                                          float& vf) {
  float wr = __fadd_rn(vr, c.gr);
  float wi = __fadd_rn(vi, c.gi);
  float m = __fmaf_rn(wr, wr, __fmul_rn(wi, wi));
  float r = rcp32(m);
  float tx = __fmaf_rn(c.c1, wr, __fmul_rn(c.c2, wi));
  float ty = __fmaf_rn(c.c3, wr, __fmul_rn(c.c4, wi));
  uf = __fmaf_rn(tx, r, c.axf);
  vf = __fmaf_rn(ty, r, c.ayf);
}

// floor of a double in [0, 2^20) from its high word alone
__device__ __forceinline__ uint32_t floor_hi(uint32_t h) {
  int e = (int)(h >> 20) - 1023;
  uint32_t mant = (h & 0xFFFFFu) | 0x100000u;
  return e < 0 ? 0u : (mant >> (20 - e));
}

// Pixel id (row * W + col) of pixel coordinates (u, v), or -1 if outside
// [0, W) x [0, H) or not finite.  For u >= 0, u < W iff hi(u) < hi(W) because
// the low word of an integer below 2^20 is zero; negative values, infinities
// and NaNs all have high words above hi(W).
__device__ __forceinline__ int pixel64(double u, double v, const View& V) {
  uint32_t hu = (uint32_t)__double2hiint(u);
  uint32_t hv = (uint32_t)__double2hiint(v);
  if (hu >= V.hiW || hv >= V.hiH) return -1;
  return (int)(floor_hi(hv) * V.W + floor_hi(hu));
}

// Packed FP32 pairs (Blackwell f32x2 add/mul/fma): two words per instruction,
// each half rounded exactly as the scalar operation.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float lo, float hi) {
  f2 d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void upk(f2 a, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 add2_rm(f2 a, f2 b) {
  f2 d;
  asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// ---------------------------------------------------------------------------
// words and tables

__device__ __forceinline__ int allowed_letter(int digit, int ban) {
  return digit + (digit >= ban ? 1 : 0);
}

// Index -> letters w_1 .. w_d: w_1 = i / 3^(d-1), then each base-3 digit picks
// the digit-th letter other than the inverse of the letter before it.
__device__ __forceinline__ void decode_word(uint64_t i, int d, int* w) {
  for (int k = d - 1; k >= 1; --k) {
    w[k] = (int)(i % 3u);
    i /= 3u;
  }
  w[0] = (int)i;
  for (int k = 1; k < d; ++k) w[k] = allowed_letter(w[k], (w[k - 1] + 2) & 3);
}

// Tables are built in two passes.  The parts pass builds four small tables:
//   L: prefix tails, the q innermost prefix letters w_{p-q+1} .. w_p, as a
//      matrix, slot (x = w_p, base-3 ranks of w_{p-1} .. w_{p-q+1});
//   H: prefix heads w_1 .. w_{p-q}, slot (y = the letter right of the head,
//      base-3 ranks of w_{p-q} .. w_1);
//   So: suffix heads w_{p+1} .. w_{p+so} as a matrix, slot (u = w_{p+1}, ranks);
//   Si: suffix tails w_{p+so+1} .. w_d applied to the seed of w_d, one map at a
//      time, slot (z = w_{p+so+1}, ranks).
// The combine pass then forms every prefix matrix P = H L (one 2x2 product)
// and its pole-form constants, and every suffix point v = So(Si) (one map).
// Each L, H and So matrix is renormalised to det 1 after every `renorm`
// letters (a shorter product of det-1 generators has det 1 up to rounding);
// P is not renormalised (its determinant enters beta explicitly).
// The slot numbering is the same as for a single-level decode: a prefix slot
// (x, r) has r = r_L 3^(p-q) + r_H, a suffix slot (u, j) has
// j = j_So 3^si + rank(z) 3^(si-1) + j_Si.

__host__ __device__ __forceinline__ uint32_t parts_count(const Plan& L) {
  return 4u * L.p3_q1 + (L.p > L.q ? 4u * L.p3_pq : 0u) + (L.so > 0 ? 4u * L.p3_so1 : 0u) +
         4u * L.p3_si1;
}
__host__ __device__ __forceinline__ uint32_t combine_count(const Plan& L) {
  return 4u * L.nr + 4u * L.ns;
}

__device__ void part_entry(const Group& G, const Plan& L, int renorm, uint32_t idx,
                           const Tables& T) {
  const uint32_t nL = 4u * L.p3_q1, nH = L.p > L.q ? 4u * L.p3_pq : 0u;
  const uint32_t nSo = L.so > 0 ? 4u * L.p3_so1 : 0u;
  if (idx < nL + nH) {
    // prefix part: letters taken right to left, matrix built by prepending
    const bool tail = idx < nL;
    const uint32_t slot = tail ? idx : idx - nL;
    const uint32_t per = tail ? L.p3_q1 : L.p3_pq;
    const int first = (int)(slot / per);
    const uint32_t r = slot % per;
    const int nlet = tail ? L.q - 1 : L.p - L.q;  // letters chosen by digits
    M2 P = tail ? load_gen(G, first) : identity2();
    int right = first;
    uint32_t place = per / 3u;
    int used = tail ? 1 : 0;
    for (int k = 0; k < nlet; ++k) {
      const int digit = (int)((r / place) % 3u);
      place /= 3u;
      const int w = allowed_letter(digit, (right + 2) & 3);
      P = mmul(load_gen(G, w), P);
      right = w;
      if (renorm > 0 && (++used % renorm) == 0) renormalise(P);
    }
    if (tail) {
      PartM e;
      e.m = P;
      e.edge = right;
      e.pad[0] = e.pad[1] = e.pad[2] = 0;
      T.Lt[slot] = e;
    } else {
      T.Ht[slot] = P;
    }
  } else if (idx < nL + nH + nSo) {
    // suffix head: letters left to right, matrix built by appending
    const uint32_t slot = idx - nL - nH;
    const int u = (int)(slot / L.p3_so1);
    const uint32_t j = slot % L.p3_so1;
    M2 S = load_gen(G, u);
    int left = u, used = 1;
    uint32_t place = L.p3_so1 / 3u;
    for (int k = 1; k < L.so; ++k) {
      const int digit = (int)((j / place) % 3u);
      place /= 3u;
      const int w = allowed_letter(digit, (left + 2) & 3);
      S = mmul(S, load_gen(G, w));
      left = w;
      if (renorm > 0 && (++used % renorm) == 0) renormalise(S);
    }
    PartM e;
    e.m = S;
    e.edge = left;
    e.pad[0] = e.pad[1] = e.pad[2] = 0;
    T.Sot[slot] = e;
  } else {
    // suffix tail: the orbit of the seed of w_d, innermost letter first.  A
    // plan always has at least one tail letter (si >= 1 for suffixes of one
    // or more letters); words of length 1 build no tables (their callers
    // render them directly or reject them), and a plan without tail letters
    // has no tail entries to build: w_{si-1} would not exist.
    if (L.si < 1) return;
    const uint32_t slot = idx - nL - nH - nSo;
    int w[kMaxSuffix];
    w[0] = (int)(slot / L.p3_si1);
    const uint32_t j = slot % L.p3_si1;
    uint32_t place = L.p3_si1 / 3u;
    for (int k = 1; k < L.si; ++k) {
      const int digit = (int)((j / place) % 3u);
      place /= 3u;
      w[k] = allowed_letter(digit, (w[k - 1] + 2) & 3);
    }
    const int last = w[L.si - 1];
    dc z = {G.seed[2 * last], G.seed[2 * last + 1]};
    for (int k = L.si - 1; k >= 0; --k) z = mobius(load_gen(G, w[k]), z);
    T.Sit[slot] = make_double2(z.re, z.im);
  }
}

// A double as a double-float: hi = fl32(d), lo = fl32(d - hi).
__device__ __forceinline__ void split_df(double d, float& hi, float& lo) {
  hi = __double2float_rn(d);
  lo = __double2float_rn(d - (double)hi);
}

// Combine pass entry idx (the render's prefix slots first, 4 nr of them:
// last letter x, slot r0 + k; then the suffix slots).  prec: the kl_precision
// of the render.  Fallback prefixes (KL_MIXED, KL_DF64) are appended to
// fb_list as (group << 32) | slot.
__device__ void combine_entry(const View& V, const Plan& L, double ptol, int prec,
                              uint32_t idx, const Tables& T, uint32_t group,
                              unsigned long long* __restrict__ fb_list,
                              uint32_t* __restrict__ fb_count) {
  const bool mixed = prec == KL_MIXED, df = prec == KL_DF64;
  const uint32_t nP = 4u * L.nr;
  if (idx >= nP) {
    const uint32_t slot = idx - nP;
    double2 v;
    if (L.so == 0) {
      v = T.Sit[slot];
    } else {
      const int u = (int)(slot / L.ns);
      const uint32_t j = slot % L.ns;
      const uint32_t j_so = j / L.p3_si, rem = j % L.p3_si;
      const PartM& S = T.Sot[(uint32_t)u * L.p3_so1 + j_so];
      const int z = allowed_letter((int)(rem / L.p3_si1), (S.edge + 2) & 3);
      const double2 t = T.Sit[(uint32_t)z * L.p3_si1 + rem % L.p3_si1];
      const dc r = mobius(S.m, {t.x, t.y});
      v = make_double2(r.re, r.im);
    }
    T.suf64[slot] = v;
    // pair-interleaved FP32 table: per first letter u, entry k holds
    // (re v_2k, re v_2k+1, im v_2k, im v_2k+1); an odd count is padded with NaN
    const uint32_t u = slot / L.ns, j = slot % L.ns;
    float* e = (float*)T.suf32p + 4ull * ((uint64_t)u * L.npairs + j / 2u);
    e[j & 1u] = (float)v.x;
    e[2 + (j & 1u)] = (float)v.y;
    if (j + 1u == L.ns && (L.ns & 1u)) {
      e[1] = __int_as_float(0x7FC00000);
      e[3] = __int_as_float(0x7FC00000);
    }
    if (df) {
      // pair-interleaved double-float table, padded with NaN like the FP32 one
      float* q = (float*)T.sufdf + 8ull * ((uint64_t)u * L.npairs + j / 2u);
      float rh, rl, ih, il;
      split_df(v.x, rh, rl);
      split_df(v.y, ih, il);
      q[j & 1u] = rh;
      q[2 + (j & 1u)] = rl;
      q[4 + (j & 1u)] = ih;
      q[6 + (j & 1u)] = il;
      if (j + 1u == L.ns && (L.ns & 1u))
        for (int c = 1; c < 8; c += 2) q[c] = __int_as_float(0x7FC00000);
    }
    return;
  }
  const int x = (int)(idx / L.nr);
  const uint32_t r = L.r0 + idx % L.nr;
  const uint32_t slot = (uint32_t)x * L.np + r;
  const PartM& TL = T.Lt[(uint32_t)x * L.p3_q1 + r / L.p3_pq];
  const M2 P = L.p > L.q ? mmul(T.Ht[(uint32_t)TL.edge * L.p3_pq + r % L.p3_pq], TL.m) : TL.m;
  const dc det = mdet(P);
  const dc tr = cadd(P.p, P.s);
  const double scale = fmax(fmax(cabs1(P.p), cabs1(P.q)), fmax(cabs1(P.r), cabs1(P.s)));
  uint32_t fl = 0;
  const dc tr2m4 = csub(cmul(tr, tr), {4.0 * det.re, 4.0 * det.im});
  const double t2 = tr.re * tr.re + tr.im * tr.im;
  const double lim2 = ptol * fmax(1.0, t2);
  if (tr2m4.re * tr2m4.re + tr2m4.im * tr2m4.im < lim2 * lim2) fl |= kNearPar;
  Pre64 c64;
  Pre32 c32;
  if (!(cabs1(P.r) > 1e-12 * scale)) {
    fl |= kDirect;
    c64 = {P.p.re, P.p.im, P.q.re, P.q.im, P.r.re, P.r.im, P.s.re, P.s.im};
    c32 = {};
  } else {
    const dc inv10 = crcp(P.r);
    const dc alpha = cmul(P.p, inv10);
    const dc gamma = cmul(P.s, inv10);
    const dc mbeta = cmul(det, cmul(inv10, inv10));  // -beta
    const double ax = (alpha.re - V.x0) * V.sx;
    const double ay = (V.y1 - alpha.im) * V.sy;
    const double c1 = -V.sx * mbeta.re, c2 = -V.sx * mbeta.im;
    const double c3 = V.sy * mbeta.im, c4 = -V.sy * mbeta.re;
    c64 = {gamma.re, gamma.im, ax, ay, c1, c2, c3, c4};
    const double lim = 1048576.0;  // 2^20
    if (!(fabs(ax) < lim && fabs(ay) < lim && fabs(gamma.re) < 1e15 && fabs(gamma.im) < 1e15))
      fl |= kWide;
    const double axi = floor(fmax(fmin(ax, lim), -lim));
    const double ayi = floor(fmax(fmin(ay, lim), -lim));
    c32.gr = (float)gamma.re;
    c32.gi = (float)gamma.im;
    c32.axf = (float)(ax - axi);
    c32.ayf = (float)(ay - ayi);
    c32.c1 = (float)c1;
    c32.c2 = (float)c2;
    c32.c3 = (float)c3;
    c32.c4 = (float)c4;
    c32.axi = (int)axi;
    c32.ayi = (int)ayi;
    c32.kx = 0x4B400000 - (int)axi;
    c32.ky = 0x4B400000 - (int)ayi;
  }
  if (df) {
    // the double-float constants; a constant (nonzero) outside [1e-30, 1e30]
    // would leave the float range in the per-word products
    PreDF cd;
    const double cv[8] = {c64.gr, c64.gi, c64.ax, c64.ay, c64.c1, c64.c2, c64.c3, c64.c4};
    for (int q = 0; q < 8; ++q) {
      split_df(cv[q], cd.h[q], cd.l[q]);
      const double a = fabs(cv[q]);
      if (!(a < 1e30) || (a != 0.0 && a < 1e-30)) fl |= kDfRange;
    }
    if (!(fl & kDirect)) T.predf[slot] = cd;
  }
  if ((mixed && (fl & (kDirect | kNearPar | kWide))) ||
      (df && (fl & (kDirect | kWide | kDfRange)))) {
    fl |= kFallback;
    const uint32_t k = atomicAdd(fb_count, 1u);
    fb_list[k] = ((unsigned long long)group << 32) | slot;
  }
  T.pre64[slot] = c64;
  T.pre32[slot] = c32;
  T.flags[slot] = fl;
}

// ---------------------------------------------------------------------------
// splat

// Run-length tally of one thread's words.  Consecutive words of a thread
// differ only in their innermost letters, so they usually land in the same
// pixel; a run of equal pixels becomes one atomic add.  pix < 0 marks a
// dropped word (such runs are discarded).
struct Tally {
  uint32_t in_window = 0, atomics = 0;
  int cur = -1;
  uint32_t run = 0;

  __device__ __forceinline__ void flush(uint32_t* __restrict__ img) {
    if (cur >= 0 && run) {
      atomicAdd(img + cur, run);
      ++atomics;
      in_window += run;
    }
    run = 0;
  }
  __device__ __forceinline__ void add(int pix, uint32_t* __restrict__ img) {
    if (pix != cur) {
      flush(img);
      cur = pix;
    }
    ++run;
  }
  // n words into pixel pix (-1: outside the window)
  __device__ __forceinline__ void add_n(int pix, uint32_t n, uint32_t* __restrict__ img) {
    if (pix != cur) {
      flush(img);
      cur = pix;
    }
    run += n;
  }
};

struct UnitTally {
  uint32_t words, in_window, atomics;
};

// Warp-sum the four counters and add them once per warp (all lanes must call).
__device__ __forceinline__ void publish_counts(uint32_t in_window, uint32_t words,
                                               uint32_t fp64_words, uint32_t atomics,
                                               unsigned long long* counters) {
  unsigned long long a = in_window, b = words - in_window, c = fp64_words, e = atomics;
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xFFFFFFFFu, a, o);
    b += __shfl_down_sync(0xFFFFFFFFu, b, o);
    c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    e += __shfl_down_sync(0xFFFFFFFFu, e, o);
  }
  if ((threadIdx.x & 31) == 0 && counters) {
    if (a) atomicAdd(counters + KL_CNT_IN_WINDOW, a);
    if (b) atomicAdd(counters + KL_CNT_DROPPED, b);
    if (c) atomicAdd(counters + KL_CNT_FP64_WORDS, c);
    if (e) atomicAdd(counters + KL_CNT_ATOMICS, e);
  }
}

// Programmatic dependent launch: a kernel launched with launch_dependent may
// start while the kernel before it in the stream is still running; pdl_wait
// blocks until that kernel has completed and its writes are visible, and
// must come before any read of them.  pdl_trigger lets the next dependent
// launch start early.  Launched the ordinary way, both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Image clearing carried by another launch: `words` uint32 at `img` (none if
// 0), and the counters (if not null).
struct Clear {
  uint32_t* img = nullptr;
  size_t words = 0;
  unsigned long long* counters = nullptr;
};

// Zero words [0, n) of p (4-byte aligned) with 16-byte stores; thread t of
// `threads` takes every threads-th vector.
__device__ __forceinline__ void clear_words(uint32_t* p, size_t n, size_t t, size_t threads) {
  const size_t head = (((16u - ((uintptr_t)p & 15u)) & 15u) / 4u) < n
                          ? ((16u - ((uintptr_t)p & 15u)) & 15u) / 4u
                          : n;
  if (t < head) p[t] = 0u;
  uint4* v = reinterpret_cast<uint4*>(p + head);
  const size_t nv = (n - head) / 4;
  for (size_t i = t; i < nv; i += threads) v[i] = make_uint4(0u, 0u, 0u, 0u);
  const size_t tail = head + 4 * nv;
  if (tail + t < n) p[tail + t] = 0u;
}

// Per-warp queue: lane 0 takes the next item and broadcasts it (no block
// barrier; warps proceed independently).
__device__ __forceinline__ uint32_t next_item_warp(uint32_t* queue) {
  uint32_t v = 0;
  if ((threadIdx.x & 31) == 0) v = atomicAdd(queue, 1u);
  return __shfl_sync(0xFFFFFFFFu, v, 0);
}

__device__ __forceinline__ uint32_t next_item(uint32_t* queue) {
  __shared__ uint32_t s_item;
  __syncthreads();
  if (threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
  __syncthreads();
  return s_item;
}

__device__ __forceinline__ void item_of(uint32_t item, const Work& W, int& x, int& u,
                                        uint32_t& pb, uint32_t& c) {
  c = item % W.n_chunks;
  const uint32_t t = item / W.n_chunks;
  pb = t % W.n_pb;
  const int q = (int)(t / W.n_pb);
  x = q / 3;
  u = allowed_letter(q % 3, (x + 2) & 3);
}

// Fixed-point box coordinate (1/256 pixel) of an FP64 pixel coordinate:
// floor(256 u), saturated to +-2^30; NaN is reported through `ok`.
__device__ __forceinline__ int box_coord64(double u, bool& ok) {
  ok = ok && (u == u);
  const double c = fmin(fmax(floor(256.0 * u), -1073741824.0), 1073741824.0);
  return (int)c;
}

// The same for a local-frame FP32 coordinate: 256 axi + floor(256 uf).
__device__ __forceinline__ int box_coord32(int axi, float uf) {
  const int A = 1073741824;
  if (!(fabsf(uf) < 2097152.0f)) return uf > 0.0f ? A : -A;  // |uf| >= 2^21
  return 256 * axi + (int)floorf(256.0f * uf);
}

__device__ __forceinline__ void box_merge(const BoxRef& B, uint32_t slot, int c0, int c1, int r0,
                                          int r1) {
  if (c0 > c1) return;  // no finite word
  atomicMin(B.cmin + slot, c0);
  atomicMax(B.cmax + slot, c1);
  atomicMin(B.rmin + slot, r0);
  atomicMax(B.rmax + slot, r1);
}

// FP64 words of one prefix slot on suffix points [j0, j1) of one first letter.
// BBOX: also merge the words' pixel box into the slot's box.
template <bool BBOX = false>
__device__ __forceinline__ void words64(const Pre64& k, bool direct, const double2* src,
                                        uint32_t j0, uint32_t j1, const View& V, Tally& t,
                                        uint32_t* __restrict__ img, const BoxRef* B = nullptr,
                                        uint32_t slot = 0) {
  int c0 = 0x7FFFFFFF, c1 = -0x7FFFFFFF, r0 = 0x7FFFFFFF, r1 = -0x7FFFFFFF;
  if (direct) {
    for (uint32_t j = j0; j < j1; ++j) {
      double uu, vv;
      const double2 s = __ldg(src + j);
      uv_direct64(k, s.x, s.y, V, uu, vv);
      t.add(pixel64(uu, vv, V), img);
      if (BBOX) {
        bool ok = true;
        const int cc = box_coord64(uu, ok), rr = box_coord64(vv, ok);
        if (ok) { c0 = min(c0, cc); c1 = max(c1, cc); r0 = min(r0, rr); r1 = max(r1, rr); }
      }
    }
  } else {
#pragma unroll 2
    for (uint32_t j = j0; j < j1; ++j) {
      double uu, vv;
      const double2 s = __ldg(src + j);
      uv_pole64(k, s.x, s.y, uu, vv);
      t.add(pixel64(uu, vv, V), img);
      if (BBOX) {
        bool ok = true;
        const int cc = box_coord64(uu, ok), rr = box_coord64(vv, ok);
        if (ok) { c0 = min(c0, cc); c1 = max(c1, cc); r0 = min(r0, rr); r1 = max(r1, rr); }
      }
    }
  }
  t.flush(img);
  if (BBOX) box_merge(*B, slot, c0, c1, r0, r1);
}

// One FP64 item of a plain render: words of this thread's prefix on one chunk.
template <int BT>
__device__ __forceinline__ void fp64_item(uint32_t item, const Work& Wk, const Plan& L,
                                          const View& V, const Tables& T, Tally& t,
                                          uint32_t& words, uint32_t* __restrict__ img) {
  int x, u;
  uint32_t pb, c;
  item_of(item, Wk, x, u, pb, c);
  const uint32_t k = pb * BT + threadIdx.x;
  if (k >= L.nr) return;
  const uint32_t slot = (uint32_t)x * L.np + L.r0 + k;
  const uint32_t j0 = c * Wk.chunk, j1 = min(L.ns, j0 + Wk.chunk);
  words64(T.pre64[slot], T.flags[slot] & kDirect, T.suf64 + (size_t)u * L.ns, j0, j1, V, t,
          img);
  words += j1 - j0;
}

// Mixed-mode FP64 fallback unit (kept out of line so that its registers do
// not bind the FP32 loop): (fallback prefix, one of its three suffix letters,
// a chunk of kFbChunk suffix points).  Chunks past the end are empty.
template <bool BBOX = false>
__device__ __noinline__ UnitTally fallback_unit(const Pre64* __restrict__ pre,
                                                const uint32_t* __restrict__ flags,
                                                const double2* __restrict__ suf, uint32_t slot,
                                                uint32_t k, uint32_t c, uint32_t np, uint32_t ns,
                                                View V, uint32_t* __restrict__ img,
                                                BoxRef B = BoxRef{}) {
  const int x = (int)(slot / np);
  const int u = allowed_letter((int)k, (x + 2) & 3);
  const uint32_t j0 = c * kFbChunk;
  if (j0 >= ns) return {0u, 0u, 0u};
  const uint32_t j1 = min(ns, j0 + kFbChunk);
  Tally t;
  words64<BBOX>(pre[slot], flags[slot] & kDirect, suf + (size_t)u * ns, j0, j1, V, t, img, &B,
                slot);
  return {j1 - j0, t.in_window, t.atomics};
}

// One FP32 item of a mixed render.  The per-word map runs in the prefix's
// local frame, two words per packed f32x2 instruction.
//
// Pixel ids: for |uf| < 2^22, adding 1.5 * 2^23 rounded toward minus infinity
// leaves floor(uf) in the low mantissa bits: bits(t) - 0x4B400000 = floor(uf),
// so col = bits(t) - kx with kx = 0x4B400000 - axi.  Any |uf| >= 2^22,
// infinity or NaN gives a t whose bits put col outside [0, W) (|axi| < 2^20
// and W <= 2^16), so one unsigned compare per coordinate rejects
// out-of-window and non-finite words alike.  Within one prefix kx and ky are
// fixed, so two words share a pixel exactly when their t bits agree.
//
// Runs: consecutive suffix points usually land in one pixel.  The current
// run is kept as its pixel's t bits (cu, cv), doubled into the packed CU, CV,
// so that a pair of words that both fall in it is settled by two 64-bit
// compares; the run's length is taken from the pair index when it ends, and
// only then is its pixel id formed and one atomic issued.  A run may lie
// outside the window (its words are then dropped when it ends), so words
// outside the window also take the two-compare path while they keep to one
// (virtual) pixel.  Runs start afresh for every prefix.
__device__ __forceinline__ void flush_run(uint32_t cu, uint32_t cv, uint32_t n, const Pre32& k,
                                          const View& V, Tally& t,
                                          uint32_t* __restrict__ img) {
  const int col = (int)cu - k.kx, row = (int)cv - k.ky;
  if (n && (uint32_t)col < V.W && (uint32_t)row < V.H) {
    atomicAdd(img + (uint32_t)row * V.W + (uint32_t)col, n);
    ++t.atomics;
    t.in_window += n;
  }
}

// Mixed words of prefix slot `slot` on suffix point pairs [k0, k1) of first
// letter u (see the comment above for the pixel arithmetic and the runs).
template <bool BBOX = false>
__device__ __forceinline__ void mixed_slot_words(uint32_t slot, int u, uint32_t k0, uint32_t k1,
                                                 const Plan& L, const View& V, const Tables& T,
                                                 Tally& t, uint32_t& words,
                                                 uint32_t* __restrict__ img,
                                                 const BoxRef* B = nullptr) {
  const Pre32 k = T.pre32[slot];
  const f2 GR = pk(k.gr, k.gr), GI = pk(k.gi, k.gi);
  const f2 C1 = pk(k.c1, k.c1), C2 = pk(k.c2, k.c2), C3 = pk(k.c3, k.c3), C4 = pk(k.c4, k.c4);
  const f2 AX = pk(k.axf, k.axf), AY = pk(k.ayf, k.ayf);
  const f2 magic = 0x4B4000004B400000ull;  // (1.5 * 2^23, 1.5 * 2^23)
  const float4* src = T.suf32p + (size_t)u * L.npairs;
  int bc0 = 0x7FFFFFFF, bc1 = -0x7FFFFFFF, br0 = 0x7FFFFFFF, br1 = -0x7FFFFFFF;
  t.flush(img);
  t.cur = -1;
  // the current run: its pixel's t bits, doubled, in CU and CV (the low
  // halves are the bits); `run` words before pair e_run, and every pair from
  // e_run on that matched it.  It starts as bits (0, 0) with no word (no
  // in-window word has them).
  uint32_t run = 0;
  f2 CU = 0, CV = 0;
  uint32_t e_run = k0;
#pragma unroll 4
  for (uint32_t e = k0; e < k1; ++e) {
    const float4 s = __ldg(src + e);
    const f2 wr = add2(pk(s.x, s.y), GR);
    const f2 wi = add2(pk(s.z, s.w), GI);
    const f2 m = fma2(wr, wr, mul2(wi, wi));
    float ma, mb;
    upk(m, ma, mb);
    const f2 rr = pk(rcp32(ma), rcp32(mb));
    const f2 tx = fma2(C1, wr, mul2(C2, wi));
    const f2 ty = fma2(C3, wr, mul2(C4, wi));
    const f2 TU = add2_rm(fma2(tx, rr, AX), magic);
    const f2 TV = add2_rm(fma2(ty, rr, AY), magic);
    if (!((TU == CU) & (TV == CV))) {
      const uint32_t ua = (uint32_t)TU, ub = (uint32_t)(TU >> 32);
      const uint32_t va = (uint32_t)TV, vb = (uint32_t)(TV >> 32);
      const uint32_t cu = (uint32_t)CU, cv = (uint32_t)CV;
      const bool a_in = (ua == cu) & (va == cv);
      const bool ab = (ua == ub) & (va == vb);
      run += 2u * (e - e_run) + (a_in ? 1u : 0u);
      e_run = e + 1;
      flush_run(cu, cv, run, k, V, t, img);
      if (!a_in && !ab) flush_run(ua, va, 1u, k, V, t, img);  // word a on its own
      run = (!a_in && ab) ? 2u : 1u;
      CU = TU >> 32 | (TU & 0xFFFFFFFF00000000ull);
      CV = TV >> 32 | (TV & 0xFFFFFFFF00000000ull);
    }
    if (BBOX) {
      float ua, ub, va, vb;
      upk(fma2(tx, rr, AX), ua, ub);
      upk(fma2(ty, rr, AY), va, vb);
      if (ua == ua && va == va) {
        const int cc = box_coord32(k.axi, ua), rr2 = box_coord32(k.ayi, va);
        bc0 = min(bc0, cc); bc1 = max(bc1, cc); br0 = min(br0, rr2); br1 = max(br1, rr2);
      }
      if (ub == ub && vb == vb) {
        const int cc = box_coord32(k.axi, ub), rr2 = box_coord32(k.ayi, vb);
        bc0 = min(bc0, cc); bc1 = max(bc1, cc); br0 = min(br0, rr2); br1 = max(br1, rr2);
      }
    }
  }
  run += 2u * (k1 - e_run);
  flush_run((uint32_t)CU, (uint32_t)CV, run, k, V, t, img);
  words += min(2u * k1, L.ns) - 2u * k0;
  if (BBOX) box_merge(*B, slot, bc0, bc1, br0, br1);
}

// One FP32 item of a mixed render: this thread's prefix on one chunk.
template <int BT, bool BBOX = false>
__device__ __forceinline__ void mixed_item(uint32_t item, const Work& Wk, const Plan& L,
                                           const View& V, const Tables& T, Tally& t,
                                           uint32_t& words, uint32_t* __restrict__ img,
                                           const BoxRef* B = nullptr) {
  int x, u;
  uint32_t pb, c;
  item_of(item, Wk, x, u, pb, c);
  const uint32_t k = pb * BT + (threadIdx.x % BT);
  if (k >= L.nr) return;
  const uint32_t slot = (uint32_t)x * L.np + L.r0 + k;
  if (T.flags[slot] & kFallback) return;
  const uint32_t k0 = c * Wk.chunk, k1 = min(L.npairs, k0 + Wk.chunk);
  mixed_slot_words<BBOX>(slot, u, k0, k1, L, V, T, t, words, img, B);
}

}  // namespace

// The double-float arithmetic, the culled renders and the host helpers.
#include "kl_df.cuh"
#include "kl_cull.cuh"
#include "kl_plan.cuh"
