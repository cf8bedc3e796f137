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

// ---------------------------------------------------------------------------
// culled renders (kl_params.cull), shared by the single and batched renders
//
// The suffix points of one first letter come in aligned blocks of 3^j
// consecutive points: the points of one subtree, which share all but their
// last j letters and so lie close together.  Blocks of 9 .. 729 points form a
// tree (a block's children are the three blocks of a third its size inside
// it), and the disk pass (cull_disk_unit) bounds every block by a disk.  A
// prefix in pole form, (u, v) = M (w_re, w_im) / |w|^2 + (ax, ay) with
// w = v + gamma, sends a disk D(c, rho) with |c + gamma| > rho onto a set
// inside the disk of center M (c + gamma) / q + (ax, ay) and radius
// |M| rho / q, q = |c + gamma|^2 - rho^2
// (inversion maps a disk clear of the pole onto a disk; M is linear with
// operator norm |M|).  When that disk, widened by a margin larger than the
// rounding error of the per-word map, lies inside one pixel or wholly outside
// the window, every word of the block lands there and the block is tallied
// with one add; otherwise its three children are tested, and a failing block
// of the smallest size is evaluated word by word.  Tests run 32 to a warp, one
// per lane, from a per-warp stack of (prefix, level, block) entries in shared
// memory; word-by-word blocks wait in a second per-warp queue until 32 are
// there.

constexpr int kCullStack = 384;  // per-warp test stack (entries)
constexpr int kLeafQueue = 64;   // per-warp queue of blocks left to the per-word path

// Operator norm of the 2x2 real matrix [[c1, c2], [c3, c4]] (its largest
// singular value), slightly rounded up.
__device__ __forceinline__ float opnorm32(float c1, float c2, float c3, float c4) {
  const float a = sqrtf(fmaf(c1 + c4, c1 + c4, (c2 - c3) * (c2 - c3)));
  const float b = sqrtf(fmaf(c1 - c4, c1 - c4, (c2 + c3) * (c2 + c3)));
  return 0.5f * (a + b) * (1.0f + 0x1p-16f);
}
__device__ __forceinline__ double opnorm64(double c1, double c2, double c3, double c4) {
  const double a = sqrt(fma(c1 + c4, c1 + c4, (c2 - c3) * (c2 - c3)));
  const double b = sqrt(fma(c1 - c4, c1 - c4, (c2 + c3) * (c2 + c3)));
  return 0.5 * (a + b) * (1.0 + 0x1p-40);
}

constexpr int kUncertified = -2;

// Certified pixel of a whole block under an FP32 prefix (local frame, as the
// mixed per-word map): the pixel id, -1 (every word outside the window), or
// kUncertified.  The margin, 2^-11 px + 2^-20 of the offsets from alpha's
// pixel, is far above the per-word map's rounding error; the interval ends are
// rounded outwards before flooring, so a certified block never straddles a
// pixel edge.
__device__ __forceinline__ int block_pixel32(const Pre32& k, float nrm, float4 D, const View& V) {
  const float c0r = D.x + k.gr, c0i = D.y + k.gi;
  const float n2 = fmaf(c0r, c0r, c0i * c0i), rho2 = D.z * D.z;
  if (!(4.0f * rho2 < n2)) return kUncertified;  // near the pole, or not finite
  const float rq = rcp32(n2 - rho2);
  const float X = fmaf(fmaf(k.c1, c0r, k.c2 * c0i), rq, k.axf);
  const float Y = fmaf(fmaf(k.c3, c0r, k.c4 * c0i), rq, k.ayf);
  const float R = nrm * D.z * rq;
  const float m = R + fmaf(fabsf(X) + fabsf(Y) + R, 0x1p-20f, 0x1p-11f);
  if (m < 0.5f && fabsf(X) < 0x1p21f && fabsf(Y) < 0x1p21f) {
    const float magic = 12582912.0f;  // 1.5 * 2^23: t bits - 0x4B400000 = floor
    const int xl = __float_as_int(__fadd_rd(__fsub_rd(X, m), magic));
    const int xh = __float_as_int(__fadd_rd(__fadd_ru(X, m), magic));
    const int yl = __float_as_int(__fadd_rd(__fsub_rd(Y, m), magic));
    const int yh = __float_as_int(__fadd_rd(__fadd_ru(Y, m), magic));
    if (xl == xh && yl == yh) {
      const int col = xl - k.kx, row = yl - k.ky;
      return ((uint32_t)col < V.W && (uint32_t)row < V.H) ? row * (int)V.W + col : -1;
    }
  }
  // wholly outside the window (one pixel of slack covers the rounding of the
  // absolute coordinates)
  const float Xa = X + (float)k.axi, Ya = Y + (float)k.ayi;
  if (Xa + m < -1.0f || Xa - m > (float)V.W + 1.0f || Ya + m < -1.0f ||
      Ya - m > (float)V.H + 1.0f)
    return -1;
  return kUncertified;
}

// The same in FP64 (pole-form prefixes; absolute pixel coordinates).  Margin
// 2^-30 px + 2^-44 of the offsets from alpha.
__device__ __forceinline__ int block_pixel64(const Pre64& k, double nrm, const Disk64& D,
                                             const View& V) {
  const double c0r = D.cr + k.gr, c0i = D.ci + k.gi;
  const double n2 = fma(c0r, c0r, c0i * c0i), rho2 = D.rho * D.rho;
  if (!(4.0 * rho2 < n2)) return kUncertified;
  const double rq = rcp64(n2 - rho2);
  const double ox = fma(k.c1, c0r, k.c2 * c0i) * rq, oy = fma(k.c3, c0r, k.c4 * c0i) * rq;
  const double R = nrm * D.rho * rq;
  const double m = R + fma(fabs(ox) + fabs(oy) + R, 0x1p-44, 0x1p-30);
  const double X = ox + k.ax, Y = oy + k.ay;
  if (m < 0.5 && fabs(X) < 0x1p40 && fabs(Y) < 0x1p40) {
    const double xl = floor(__dsub_rd(X, m)), xh = floor(__dadd_ru(X, m));
    const double yl = floor(__dsub_rd(Y, m)), yh = floor(__dadd_ru(Y, m));
    if (xl == xh && yl == yh)
      return (xl >= 0.0 && xl < (double)V.W && yl >= 0.0 && yl < (double)V.H)
                 ? (int)yl * (int)V.W + (int)xl
                 : -1;
  }
  if (X + m < -1.0 || X - m > (double)V.W + 1.0 || Y + m < -1.0 || Y - m > (double)V.H + 1.0)
    return -1;
  return kUncertified;
}

// One FP32 word of prefix constants k: suffix point j of the letter's pair
// table (the operations of the packed per-word loop, on one half).
__device__ __forceinline__ void mixed_single_word(const Pre32& k, const float4* src, uint32_t j,
                                                  const View& V, Tally& t,
                                                  uint32_t* __restrict__ img) {
  const float4 s = __ldg(src + j / 2u);
  const bool odd = j & 1u;
  float uf, vf;
  uv_pole32(k, odd ? s.y : s.x, odd ? s.w : s.z, uf, vf);
  const int col = __float_as_int(__fadd_rd(uf, 12582912.0f)) - k.kx;
  const int row = __float_as_int(__fadd_rd(vf, 12582912.0f)) - k.ky;
  t.add(((uint32_t)col < V.W && (uint32_t)row < V.H) ? row * (int)V.W + col : -1, img);
}

// Words of FP32 prefix slot `slot` on suffix points [j0, j0 + n) of letter u:
// the odd ends one at a time, the rest as packed pairs.
__device__ __forceinline__ void mixed_block_words(uint32_t slot, int u, uint32_t j0, uint32_t n,
                                                  const Plan& L, const View& V, const Tables& T,
                                                  Tally& t, uint32_t& words,
                                                  uint32_t* __restrict__ img) {
  const float4* src = T.suf32p + (size_t)u * L.npairs;
  uint32_t j1 = j0 + n;
  if (j0 & 1u) {
    mixed_single_word(T.pre32[slot], src, j0, V, t, img);
    ++j0;
    ++words;
  }
  if (j1 > j0 && (j1 & 1u)) {
    --j1;
    mixed_single_word(T.pre32[slot], src, j1, V, t, img);
    ++words;
  }
  if (j1 > j0) mixed_slot_words(slot, u, j0 / 2u, j1 / 2u, L, V, T, t, words, img);
}

// Disk of culling block `disk` of plan L (all lanes of a warp take part),
// from the FP32 points that the mixed per-word path reads: center = middle of
// their bounding box, radius = largest distance from it, with a relative
// allowance for the FP32 rounding of that distance.  The FP64 disk has the
// same center and a radius larger by 2^-23 of the largest coordinate, which
// covers the distance from an FP64 point to its FP32 rounding.  A block with a
// non-finite point gets an infinite radius, which no test certifies.
__device__ __forceinline__ void cull_disk(const Plan& L, const Tables& T, uint32_t disk,
                                          uint32_t lane) {
  uint32_t l = 0;
  while (l + 1 < L.clev && L.cdisk[l + 1] <= disk) ++l;
  const uint32_t rem = disk - L.cdisk[l];
  const uint32_t u = rem / L.cnb[l], j0 = (rem % L.cnb[l]) * L.csz[l], j1 = j0 + L.csz[l];
  const float* s32 = reinterpret_cast<const float*>(T.suf32p + (size_t)u * L.npairs);
  const float inf = __int_as_float(0x7F800000);
  float x0 = inf, y0 = inf, x1 = -inf, y1 = -inf, amax = 0.0f;
  bool finite = true;
  for (uint32_t j = j0 + lane; j < j1; j += 32) {
    const float x = s32[4 * (j / 2) + (j & 1)], y = s32[4 * (j / 2) + 2 + (j & 1)];
    finite = finite && isfinite(x) && isfinite(y);
    x0 = fminf(x0, x);
    x1 = fmaxf(x1, x);
    y0 = fminf(y0, y);
    y1 = fmaxf(y1, y);
    amax = fmaxf(amax, fmaxf(fabsf(x), fabsf(y)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    x0 = fminf(x0, __shfl_xor_sync(0xFFFFFFFFu, x0, o));
    x1 = fmaxf(x1, __shfl_xor_sync(0xFFFFFFFFu, x1, o));
    y0 = fminf(y0, __shfl_xor_sync(0xFFFFFFFFu, y0, o));
    y1 = fmaxf(y1, __shfl_xor_sync(0xFFFFFFFFu, y1, o));
    amax = fmaxf(amax, __shfl_xor_sync(0xFFFFFFFFu, amax, o));
  }
  finite = __all_sync(0xFFFFFFFFu, finite);
  const float cx = 0.5f * x0 + 0.5f * x1, cy = 0.5f * y0 + 0.5f * y1;  // any center serves
  float d2 = 0.0f;
  for (uint32_t j = j0 + lane; j < j1; j += 32) {
    const float dx = s32[4 * (j / 2) + (j & 1)] - cx, dy = s32[4 * (j / 2) + 2 + (j & 1)] - cy;
    d2 = fmaxf(d2, fmaf(dx, dx, dy * dy));
  }
  for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xFFFFFFFFu, d2, o));
  if (lane == 0) {
    // six roundings at most, each within 2^-24 relative; 1e-30 covers underflow
    const float r32 = finite ? __fmaf_ru(sqrtf(d2), 1.0f + 0x1p-20f, 1e-30f) : inf;
    T.disk32[disk] = make_float4(cx, cy, r32, 0.0f);
    Disk64 D;
    D.cr = cx;
    D.ci = cy;
    D.rho = finite ? ((double)r32 + (double)amax * 0x1p-23) * (1.0 + 0x1p-40)
                   : __longlong_as_double(0x7FF0000000000000ll);
    D.pad = 0.0;
    T.disk64[disk] = D;
  }
}

// Operator norms of prefix slot `slot`'s pole-form matrix (the FP64 norm from
// the FP32 one where that is finite and nonzero, since the FP32 entries are
// the FP64 ones rounded).
__device__ __forceinline__ void cull_norm(const Tables& T, uint32_t slot) {
  const Pre32 k = T.pre32[slot];
  const float n32 = opnorm32(k.c1, k.c2, k.c3, k.c4);
  T.nrm32[slot] = n32;
  if (isfinite(n32) && n32 > 0.0f) {
    T.nrm64[slot] = (double)n32 * (1.0 + 0x1p-20);
  } else {
    const Pre64 c = T.pre64[slot];
    T.nrm64[slot] = opnorm64(c.c1, c.c2, c.c3, c.c4);
  }
}

// The same for a small block, by one thread.
__device__ __forceinline__ void cull_disk_thread(const Plan& L, const Tables& T, uint32_t disk) {
  uint32_t l = 0;
  while (l + 1 < L.clev && L.cdisk[l + 1] <= disk) ++l;
  const uint32_t rem = disk - L.cdisk[l];
  const uint32_t u = rem / L.cnb[l], j0 = (rem % L.cnb[l]) * L.csz[l], j1 = j0 + L.csz[l];
  const float* s32 = reinterpret_cast<const float*>(T.suf32p + (size_t)u * L.npairs);
  const float inf = __int_as_float(0x7F800000);
  float x0 = inf, y0 = inf, x1 = -inf, y1 = -inf, amax = 0.0f;
  bool finite = true;
  for (uint32_t j = j0; j < j1; ++j) {
    const float x = s32[4 * (j / 2) + (j & 1)], y = s32[4 * (j / 2) + 2 + (j & 1)];
    finite = finite && isfinite(x) && isfinite(y);
    x0 = fminf(x0, x);
    x1 = fmaxf(x1, x);
    y0 = fminf(y0, y);
    y1 = fmaxf(y1, y);
    amax = fmaxf(amax, fmaxf(fabsf(x), fabsf(y)));
  }
  const float cx = 0.5f * x0 + 0.5f * x1, cy = 0.5f * y0 + 0.5f * y1;
  float d2 = 0.0f;
  for (uint32_t j = j0; j < j1; ++j) {
    const float dx = s32[4 * (j / 2) + (j & 1)] - cx, dy = s32[4 * (j / 2) + 2 + (j & 1)] - cy;
    d2 = fmaxf(d2, fmaf(dx, dx, dy * dy));
  }
  const float r32 = finite ? __fmaf_ru(sqrtf(d2), 1.0f + 0x1p-20f, 1e-30f) : inf;
  T.disk32[disk] = make_float4(cx, cy, r32, 0.0f);
  Disk64 D;
  D.cr = cx;
  D.ci = cy;
  D.rho = finite ? ((double)r32 + (double)amax * 0x1p-23) * (1.0 + 0x1p-40)
                 : __longlong_as_double(0x7FF0000000000000ll);
  D.pad = 0.0;
  T.disk64[disk] = D;
}

// Work units of a plan's disk-and-norm pass, in warps: the disks of blocks of
// up to kThreadDiskPoints points one per thread (the smallest levels come
// first in the disk table), then one warp per larger disk, then one thread
// per prefix norm.
constexpr uint32_t kThreadDiskPoints = 81;

__device__ __host__ __forceinline__ uint32_t cull_small_disks(const Plan& L) {
  uint32_t l = 0;
  while (l < L.clev && L.csz[l] <= kThreadDiskPoints) ++l;
  return l < L.clev ? L.cdisk[l] : L.ndisks;
}
__device__ __host__ __forceinline__ uint32_t cull_disk_units(const Plan& L) {
  const uint32_t small = cull_small_disks(L);
  return (small + 31) / 32 + (L.ndisks - small) + (4u * L.np + 31) / 32;
}
// One warp's share (all lanes call): unit w of cull_disk_units(L).
__device__ __forceinline__ void cull_disk_unit(const Plan& L, const Tables& T, uint32_t w,
                                               uint32_t lane) {
  const uint32_t small = cull_small_disks(L), ws = (small + 31) / 32;
  if (w < ws) {
    const uint32_t disk = w * 32 + lane;
    if (disk < small) cull_disk_thread(L, T, disk);
  } else if (w < ws + (L.ndisks - small)) {
    cull_disk(L, T, small + (w - ws), lane);
  } else {
    const uint32_t slot = (w - ws - (L.ndisks - small)) * 32 + lane;
    if (slot < 4u * L.np) cull_norm(T, slot);
  }
}

// Culling levels of one plan in shared memory (the kernels index them by a
// run-time level).
struct CullLevels {
  uint32_t sz[kMaxCullLevels], nb[kMaxCullLevels], disk[kMaxCullLevels];
};

// Stack entry: prefix slot (bits 0-31), suffix letter (32-33), level (34-36),
// FP64 flag (37: a mixed render's fallback prefix), block (38-63).
__device__ __forceinline__ unsigned long long cull_entry(uint32_t slot, uint32_t u, uint32_t l,
                                                         bool f64, uint32_t b) {
  return (unsigned long long)slot | ((unsigned long long)u << 32) |
         ((unsigned long long)l << 34) | ((unsigned long long)f64 << 37) |
         ((unsigned long long)b << 38);
}

// The culling of one warp, over one group at a time: the warp's test stack
// and leaf queue (shared memory), its tally and counts.  Every lane of the
// warp calls every method; the group's plan, view, tables and image are
// passed in.  In a mixed render the fallback prefixes (near-parabolic,
// direct-form and far) take FP64 tests and FP64 words, as in the per-word
// render.
template <bool MIXED>
struct CullWarp {
  unsigned long long* stack;
  unsigned long long* leafq;
  const CullLevels* C;
  uint32_t len = 0, lq = 0, lane;
  unsigned lt;
  Tally t;
  uint32_t words = 0, fp64_words = 0;

  __device__ __forceinline__ CullWarp(unsigned long long* s, unsigned long long* q,
                                      const CullLevels* c)
      : stack(s), leafq(q), C(c), lane(threadIdx.x & 31), lt((1u << (threadIdx.x & 31)) - 1u) {}

  // all words of block b (level l) of letter u under slot, one by one
  __device__ __forceinline__ void block_words(const Plan& L, const View& V, const Tables& T,
                                              uint32_t* __restrict__ img, uint32_t slot,
                                              uint32_t u, uint32_t l, bool f64, uint32_t b) {
    const uint32_t j0 = b * C->sz[l];
    if (MIXED && !f64) {
      mixed_block_words(slot, (int)u, j0, C->sz[l], L, V, T, t, words, img);
    } else {
      words64(T.pre64[slot], T.flags[slot] & kDirect, T.suf64 + (size_t)u * L.ns, j0,
              j0 + C->sz[l], V, t, img);
      words += C->sz[l];
      if (MIXED) fp64_words += C->sz[l];
    }
  }
  // leaf queue entries [0, n), one per lane
  __device__ __forceinline__ void drain_leaves(const Plan& L, const View& V, const Tables& T,
                                               uint32_t* __restrict__ img, uint32_t n) {
    if (lane < n) {
      const unsigned long long e = leafq[lane];
      block_words(L, V, T, img, (uint32_t)e, (uint32_t)(e >> 32) & 3u, 0u, (e >> 37) & 1ull,
                  (uint32_t)(e >> 38));
    }
    __syncwarp();
  }
  // certified pixel of (slot, u, l, b), or kUncertified
  __device__ __forceinline__ int test(const View& V, const Tables& T, uint32_t slot, uint32_t u,
                                      uint32_t l, bool f64, uint32_t b) {
    const uint32_t di = C->disk[l] + u * C->nb[l] + b;
    if (MIXED && !f64) return block_pixel32(T.pre32[slot], T.nrm32[slot], T.disk32[di], V);
    if (T.flags[slot] & kDirect) return kUncertified;
    return block_pixel64(T.pre64[slot], T.nrm64[slot], T.disk64[di], V);
  }
  // the outcome of one test per lane (act: this lane tested an entry)
  __device__ __forceinline__ void settle(const Plan& L, const View& V, const Tables& T,
                                         uint32_t* __restrict__ img, bool act, uint32_t slot,
                                         uint32_t u, uint32_t l, bool f64, uint32_t b, int pix) {
    if (act && pix != kUncertified) {
      t.add_n(pix, C->sz[l], img);
      words += C->sz[l];
      if (MIXED && f64) fp64_words += C->sz[l];
    }
    const bool miss = act && pix == kUncertified;
    const bool direct = miss && f64 && (T.flags[slot] & kDirect);
    const bool kids = miss && l > 0 && !direct;
    const bool leaf = miss && l == 0 && !direct;
    // children onto the stack while there is room; a block that finds none
    // (never with the stack's size) and a direct-form prefix (no pole form to
    // test) are evaluated word by word at once
    const unsigned bk = __ballot_sync(0xFFFFFFFFu, kids);
    const uint32_t room = (uint32_t)(kCullStack - len) / 3u, rank = __popc(bk & lt);
    const bool pushed = kids && rank < room;
    if (pushed)
      for (uint32_t i = 0; i < 3; ++i)
        stack[len + 3 * rank + i] = cull_entry(slot, u, l - 1, f64, 3 * b + 2 - i);
    len += 3u * min((uint32_t)__popc(bk), room);
    if ((kids && !pushed) || direct) block_words(L, V, T, img, slot, u, l, f64, b);
    const unsigned bl = __ballot_sync(0xFFFFFFFFu, leaf);
    if (leaf) leafq[lq + __popc(bl & lt)] = cull_entry(slot, u, 0, f64, b);
    lq += __popc(bl);
    __syncwarp();
    if (lq >= 32) {
      drain_leaves(L, V, T, img, 32);
      lq -= 32;
      if (lane < lq) leafq[lane] = leafq[32 + lane];
      __syncwarp();
    }
  }
  // one round: the top n (<= 32) stack entries, one per lane
  __device__ __forceinline__ void round(const Plan& L, const View& V, const Tables& T,
                                        uint32_t* __restrict__ img, uint32_t n) {
    unsigned long long e = 0;
    if (lane < n) e = stack[len - n + lane];
    __syncwarp();
    len -= n;
    const bool act = lane < n;
    const uint32_t slot = (uint32_t)e, u = (uint32_t)(e >> 32) & 3u;
    const uint32_t l = (uint32_t)(e >> 34) & 7u, b = (uint32_t)(e >> 38);
    const bool f64 = (e >> 37) & 1ull;
    settle(L, V, T, img, act, slot, u, l, f64, b, act ? test(V, T, slot, u, l, f64, b)
                                                      : kUncertified);
  }
  // top-level blocks [b0, b1) of letter u under this lane's prefix slot
  // (live: the lane has one), with the rounds their children call for
  __device__ __forceinline__ void item(const Plan& L, const View& V, const Tables& T,
                                       uint32_t* __restrict__ img, bool live, uint32_t slot,
                                       uint32_t u, bool f64, uint32_t b0, uint32_t b1) {
    const uint32_t top = L.clev - 1;
    for (uint32_t b = b0; b < b1; ++b) {
      settle(L, V, T, img, live, slot, u, top, f64, b,
             live ? test(V, T, slot, u, top, f64, b) : kUncertified);
      while (len >= 32) round(L, V, T, img, 32);
    }
  }
  // everything still on the stack or in the leaf queue
  __device__ __forceinline__ void finish(const Plan& L, const View& V, const Tables& T,
                                         uint32_t* __restrict__ img) {
    while (len > 0) round(L, V, T, img, min(len, 32u));
    drain_leaves(L, V, T, img, lq);
    lq = 0;
  }
};

// The lanes of one culling item: prefix slot of this lane and whether it is
// live, and (mixed) whether it takes the FP64 path.  Items are 32 prefixes x
// a chunk of top-level blocks of one suffix letter.
template <bool MIXED>
__device__ __forceinline__ void cull_item(CullWarp<MIXED>& w, uint32_t item, const Work& Wk,
                                          const Plan& L, const View& V, const Tables& T,
                                          uint32_t* __restrict__ img, uint32_t top_blocks) {
  int x, u;
  uint32_t pb, c;
  item_of(item, Wk, x, u, pb, c);
  const uint32_t k = pb * 32 + w.lane;
  const uint32_t slot = (uint32_t)x * L.np + L.r0 + k;
  const bool live = k < L.nr;
  const bool f64 = !MIXED || (live && (T.flags[slot] & kFallback));
  const uint32_t b0 = c * Wk.chunk, b1 = min(top_blocks, b0 + Wk.chunk);
  w.item(L, V, T, img, live, slot, (uint32_t)u, f64, b0, b1);
}

// ---------------------------------------------------------------------------
// host helpers

// Launch `k` as a programmatic dependent of the previous kernel in stream s
// (it must call pdl_wait before reading that kernel's output).
template <typename... Params, typename... Args>
int launch_dependent(void (*k)(Params...), dim3 grid, dim3 block, cudaStream_t s,
                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k, static_cast<Args&&>(args)...) != cudaSuccess) return KL_ECUDA;
  return KL_OK;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

inline uint32_t pow3u(int e) {
  uint32_t v = 1;
  while (e-- > 0) v *= 3u;
  return v;
}

inline bool valid_view(const kl_params* p) {
  if (p->width < 1 || p->height < 1 || p->width > KL_MAX_IMAGE_SIDE ||
      p->height > KL_MAX_IMAGE_SIDE)
    return false;
  if ((uint64_t)p->width * p->height > (1ull << 31) - 1) return false;
  if (!(p->x0 < p->x1) || !(p->y0 < p->y1)) return false;
  const double v[4] = {p->x0, p->x1, p->y0, p->y1};
  for (double t : v)
    if (!isfinite(t)) return false;
  for (int k = 0; k < 32; ++k)
    if (!isfinite(p->gens[k])) return false;
  for (int k = 0; k < 8; ++k)
    if (!isfinite(p->seeds[k])) return false;
  if (p->block_threads != 0 && p->block_threads != 64 && p->block_threads != 128 &&
      p->block_threads != 256)
    return false;
  return true;
}

// Prefix/suffix split.  Single renders: up to 9 prefix letters while the
// words are few (enough threads), then suffixes of up to 8 letters (9 beyond
// depth 20), the rest prefix.  Batched renders draw their parallelism from
// many groups and use suffixes of up to 8 letters with at least 7 prefix
// letters (729 prefix slots per letter fill whole thread blocks).
inline int make_plan(const kl_params* p, Plan* L, bool batched) {
  const int d = (int)p->depth;
  if (d < 1 || d > kMaxRenderDepth) return KL_ERANGE;
  int pl, sl;
  if (d == 1) {
    pl = 1;
    sl = 0;
  } else if (p->prefix_len) {
    pl = (int)p->prefix_len;
    sl = d - pl;
    if (pl < 1 || sl < 1 || pl > kMaxPrefix || sl > kMaxSuffix) return KL_EINVAL;
  } else if (p->cull) {
    // culled renders: long suffix tables (large blocks, and a prefix table
    // whose FP64 products are the bulk of the table cost kept small): all but
    // one letter up to 9, then about half the word plus one, at most 12
    if (d - 1 <= kMaxPlainSuffix) {
      sl = d - 1;
    } else {
      sl = d / 2 + 1;
      if (sl < kMaxPlainSuffix) sl = kMaxPlainSuffix;
      if (sl > kMaxSuffix) sl = kMaxSuffix;
    }
    pl = d - sl;
    if (pl > kMaxPrefix) return KL_ERANGE;
  } else if (batched) {
    sl = d - 7;
    if (sl > 8) sl = 8;
    if (sl < 1) sl = 1;
    pl = d - sl;
    if (pl > kMaxPrefix) return KL_ERANGE;
  } else if (d <= 10) {
    pl = d - 1;
    sl = 1;
  } else {
    sl = d - 9;
    const int smax = d > 20 ? 9 : 8;
    if (sl > smax) sl = smax;
    pl = d - sl;
    if (pl > kMaxPrefix) return KL_ERANGE;
  }
  L->d = d;
  L->p = pl;
  L->s = sl;
  L->np = pow3u(pl - 1);
  L->ns = sl > 0 ? pow3u(sl - 1) : 0;
  L->npairs = (L->ns + 1) / 2;
  // shard k of n: prefix slots [floor(k np / n), floor((k+1) np / n)) per letter
  if (p->shard_count > 1) {
    if (batched || p->shard_index >= p->shard_count) return KL_EINVAL;
    const uint64_t n = p->shard_count, k = p->shard_index;
    L->r0 = (uint32_t)(k * L->np / n);
    L->nr = (uint32_t)((k + 1) * L->np / n) - L->r0;
  } else {
    L->r0 = 0;
    L->nr = L->np;
  }
  L->q = (pl + 1) / 2;
  L->so = sl / 2;
  L->si = sl - L->so;
  L->p3_q1 = pow3u(L->q - 1);
  L->p3_pq = pow3u(pl - L->q);
  L->p3_so1 = L->so > 0 ? pow3u(L->so - 1) : 1;
  L->p3_si = pow3u(L->si);
  L->p3_si1 = L->si > 0 ? pow3u(L->si - 1) : 1;
  // culling levels: blocks of 9 .. 729 points (fewer levels for short suffixes)
  {
    const int top = sl > 0 ? (sl - 1 < 6 ? sl - 1 : 6) : 0;
    const int j0 = top < 2 ? top : 2;
    L->cj0 = (uint32_t)j0;
    L->clev = sl > 0 ? (uint32_t)(top - j0 + 1) : 0;
    L->ndisks = 0;
    for (uint32_t l = 0; l < (uint32_t)kMaxCullLevels; ++l) {
      const bool on = l < L->clev;
      L->csz[l] = on ? pow3u(j0 + (int)l) : 0;
      L->cnb[l] = on ? L->ns / L->csz[l] : 0;
      L->cdisk[l] = L->ndisks;
      L->ndisks += 4u * L->cnb[l];
    }
  }
  const size_t nP = 4ull * L->np, nS = 4ull * L->ns;
  size_t off = 0;
  L->off_pre64 = off; off = align256(off + nP * sizeof(Pre64));
  L->off_pre32 = off; off = align256(off + nP * sizeof(Pre32));
  L->off_flags = off; off = align256(off + nP * sizeof(uint32_t));
  L->off_suf64 = off; off = align256(off + nS * sizeof(double2));
  L->off_suf32 = off; off = align256(off + 4ull * L->npairs * sizeof(float4));
  L->off_fb = off; off = align256(off + nP * sizeof(unsigned long long));
  L->off_fbcount = off; off = align256(off + 2 * sizeof(uint32_t));  // fallback count, queue
  L->off_L = off; off = align256(off + 4ull * L->p3_q1 * sizeof(PartM));
  L->off_H = off; off = align256(off + 4ull * L->p3_pq * sizeof(M2));
  L->off_So = off; off = align256(off + 4ull * L->p3_so1 * sizeof(PartM));
  L->off_Si = off; off = align256(off + 4ull * L->p3_si1 * sizeof(double2));
  // disks and prefix norms exist in culled plans only
  const size_t nD = p->cull ? L->ndisks : 0, nN = p->cull ? nP : 0;
  L->off_disk32 = off; off = align256(off + nD * sizeof(float4));
  L->off_disk64 = off; off = align256(off + nD * sizeof(Disk64));
  L->off_nrm32 = off; off = align256(off + nN * sizeof(float));
  L->off_nrm64 = off; off = align256(off + nN * sizeof(double));
  // double-float constants and suffix pairs exist in KL_DF64 plans only
  const bool df = p->precision == KL_DF64;
  L->off_predf = off; off = align256(off + (df ? nP : 0) * sizeof(PreDF));
  L->off_sufdf = off; off = align256(off + (df ? 8ull * L->npairs : 0) * sizeof(float4));
  L->total = off;
  return KL_OK;
}

inline View make_view(const kl_params* p) {
  View V;
  V.x0 = p->x0;
  V.y1 = p->y1;
  V.sx = (double)p->width / (p->x1 - p->x0);
  V.sy = (double)p->height / (p->y1 - p->y0);
  V.W = p->width;
  V.H = p->height;
  const double w = (double)p->width, h = (double)p->height;
  uint64_t bw, bh;
  memcpy(&bw, &w, sizeof bw);
  memcpy(&bh, &h, sizeof bh);
  V.hiW = (uint32_t)(bw >> 32);
  V.hiH = (uint32_t)(bh >> 32);
  return V;
}

inline Group make_group(const kl_params* p) {
  Group G;
  for (int k = 0; k < 32; ++k) G.g[k] = p->gens[k];
  for (int k = 0; k < 8; ++k) G.seed[k] = p->seeds[k];
  return G;
}

inline Tables carve(const Plan& L, void* ws) {
  char* b = (char*)ws;
  return {(Pre64*)(b + L.off_pre64),          (Pre32*)(b + L.off_pre32),
          (uint32_t*)(b + L.off_flags),        (double2*)(b + L.off_suf64),
          (float4*)(b + L.off_suf32),          (unsigned long long*)(b + L.off_fb),
          (uint32_t*)(b + L.off_fbcount),      (PartM*)(b + L.off_L),
          (M2*)(b + L.off_H),                  (PartM*)(b + L.off_So),
          (double2*)(b + L.off_Si),            (float4*)(b + L.off_disk32),
          (Disk64*)(b + L.off_disk64),         (float*)(b + L.off_nrm32),
          (double*)(b + L.off_nrm64),          (PreDF*)(b + L.off_predf),
          (float4*)(b + L.off_sufdf)};
}

inline int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

inline int check_launch() { return cudaGetLastError() == cudaSuccess ? KL_OK : KL_ECUDA; }

// SM count and resident blocks per SM of a kernel with BT threads.
inline int device_slots(const void* kernel, int bt, int* sms, int* occ) {
  *sms = sm_count();
  if (*sms <= 0) return KL_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kernel, bt, 0) != cudaSuccess ||
      *occ < 1)
    return KL_ECUDA;
  return KL_OK;
}

// Items of about equal cost.  chunk_units = 0: about 12 items per resident
// block, so that the queue drains within a small fraction of one item, but no
// chunk below 16 units; else chunks of that many units (suffix points or
// point pairs).
inline Work make_work(const Plan& L, int bt, uint32_t units, int slots, uint32_t chunk_units) {
  Work W;
  W.n_pb = (L.nr + bt - 1) / bt;
  if (W.n_pb == 0) {  // an empty shard
    W.n_chunks = 1;
    W.chunk = units > 0 ? units : 1;
    W.n_items = 0;
    return W;
  }
  const uint64_t base = 12ull * W.n_pb;
  if (chunk_units == 0) {
    const uint64_t target = 12ull * (uint64_t)slots;
    uint64_t n_chunks = (target + base - 1) / base;
    const uint64_t most = units / 16 > 0 ? units / 16 : 1;
    if (n_chunks > most) n_chunks = most;
    if (n_chunks < 1) n_chunks = 1;
    W.chunk = (uint32_t)((units + n_chunks - 1) / n_chunks);
  } else {
    W.chunk = chunk_units < units ? chunk_units : units;
  }
  if (W.chunk < 1) W.chunk = 1;
  W.n_chunks = (units + W.chunk - 1) / W.chunk;
  W.n_items = (uint32_t)(base * W.n_chunks);
  return W;
}

}  // namespace
