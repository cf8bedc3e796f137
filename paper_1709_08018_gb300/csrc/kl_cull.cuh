// The culled renders (kl_params.cull): certified blocks of suffix points
// placed at once, shared by the single, batched and level-of-detail renders.
// Included at the end of kl_common.cuh.
#pragma once

#include "kl_common.cuh"

namespace {

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

}  // namespace
