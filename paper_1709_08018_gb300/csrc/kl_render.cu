// Single render, decode and evaluation entry points of the C ABI (sm_103a).
// The arithmetic, tables and per-item bodies are in kl_common.cuh.
#include <mutex>

#include "kl_common.cuh"

namespace {

// ---------------------------------------------------------------------------
// table passes

constexpr uint32_t kPartLanes = 8;

// The first launch of a render.  Blocks [0, part_blocks) build the parts
// tables (and block 0 resets the fallback count, the work queue and the
// counters); the blocks after them clear the image.  The parts work is a few
// thousand short FP64 chains, far from filling the GPU, so the clearing runs
// beside it and a render needs no separate memset.
__global__ void parts_kernel(Group G, Plan L, int renorm, Tables T, Clear C,
                             uint32_t part_blocks) {
  pdl_trigger();
  if (blockIdx.x < part_blocks) {
    if (blockIdx.x == 0) {
      if (threadIdx.x < 2) T.fbcount[threadIdx.x] = 0u;
      if (C.counters && threadIdx.x < KL_N_COUNTERS) C.counters[threadIdx.x] = 0ull;
    }
    // kPartLanes entries per block: each entry is one long chain of dependent
    // FP64 operations, so spreading the entries over more SMs shortens the
    // launch more than filling warps does
    const uint32_t total = parts_count(L);
    if (threadIdx.x < kPartLanes)
      for (uint32_t idx = blockIdx.x * kPartLanes + threadIdx.x; idx < total;
           idx += part_blocks * kPartLanes)
        part_entry(G, L, renorm, idx, T);
    return;
  }
  clear_words(C.img, C.words, (size_t)(blockIdx.x - part_blocks) * blockDim.x + threadIdx.x,
              (size_t)(gridDim.x - part_blocks) * blockDim.x);
}

__global__ void combine_kernel(View V, Plan L, double ptol, int mixed, Tables T) {
  pdl_trigger();
  pdl_wait();
  const uint32_t total = combine_count(L);
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += gridDim.x * blockDim.x)
    combine_entry(V, L, ptol, mixed, idx, T, 0u, T.fb, T.fbcount);
}

// ---------------------------------------------------------------------------
// render kernels: persistent blocks drain a device work queue (one atomic per
// item) of items of equal cost.

// FP64: per item each thread evaluates its prefix on `chunk` consecutive
// suffix points, read with a warp-uniform address (a broadcast from L1).
template <int BT>
__global__ void __launch_bounds__(BT) render64_kernel(Tables T, Plan L, View V, Work Wk,
                                                      uint32_t* __restrict__ img,
                                                      unsigned long long* counters) {
  pdl_wait();
  Tally t;
  uint32_t words = 0;
  for (;;) {
    const uint32_t item = next_item(T.fbcount + 1);
    if (item >= Wk.n_items) break;
    fp64_item<BT>(item, Wk, L, V, T, t, words, img);
  }
  publish_counts(t.in_window, words, 0, t.atomics, counters);
}

// Mixed: the queue holds first the FP64 fallback items (32 units each: the
// near-parabolic, direct-form and far prefixes), then the FP32 items (32
// prefixes x one suffix chunk).  Each warp draws its own items, so warps never
// wait for one another; warps that draw fallback items keep the FP64 pipe busy
// while the others run FP32 work, so the fallback words overlap the FP32 words.
template <int BT>
__global__ void __launch_bounds__(BT, 1536 / BT) render_mixed_kernel(
    Tables T, Plan L, View V, Work Wk, uint32_t* __restrict__ img,
    unsigned long long* counters) {
  pdl_wait();
  const uint32_t chunks = (L.ns + kFbChunk - 1) / kFbChunk;
  const uint32_t fb_units = 3u * chunks * (*T.fbcount);
  const uint32_t n64 = (fb_units + 31) / 32;
  const uint32_t total = n64 + Wk.n_items;
  const uint32_t lane = threadIdx.x & 31;
  Tally t;
  uint32_t words = 0, fp64_words = 0;
  for (;;) {
    const uint32_t item = next_item_warp(T.fbcount + 1);
    if (item >= total) break;
    if (item < n64) {
      const uint32_t unit = item * 32 + lane;
      if (unit < fb_units) {
        const uint32_t e = unit / (3u * chunks), rem = unit % (3u * chunks);
        const uint32_t slot = (uint32_t)(T.fb[e] & 0xFFFFFFFFull);
        const UnitTally r = fallback_unit(T.pre64, T.flags, T.suf64, slot, rem / chunks,
                                          rem % chunks, L.np, L.ns, V, img);
        words += r.words;
        fp64_words += r.words;
        t.in_window += r.in_window;
        t.atomics += r.atomics;
      }
      continue;
    }
    mixed_item<32>(item - n64, Wk, L, V, T, t, words, img);
  }
  publish_counts(t.in_window, words, fp64_words, t.atomics, counters);
}

// ---------------------------------------------------------------------------
// culled renders (kl_params.cull)
//
// The suffix points of one first letter come in aligned blocks of 3^j
// consecutive points: the points of one subtree, which share all but their
// last j letters and so lie close together.  Blocks of 9 .. 729 points form a
// tree (a block's children are the three blocks of a third its size inside
// it), and disk_kernel bounds every block by a disk.  A prefix in pole form,
// (u, v) = M (w_re, w_im) / |w|^2 + (ax, ay) with w = v + gamma, sends a disk
// D(c, rho) with |c + gamma| > rho onto a set inside the disk of center
// M (c + gamma) / q + (ax, ay) and radius |M| rho / q, q = |c + gamma|^2 - rho^2
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

// Disks of all culling blocks, one warp per block, from the FP32 points that
// the mixed per-word path reads: center = middle of their bounding box,
// radius = largest distance from it, with a relative allowance for the FP32
// rounding of that distance.  The FP64 disk has the same center and a radius
// larger by 2^-23 of the largest coordinate, which covers the distance from
// an FP64 point to its FP32 rounding.  A block with a non-finite point gets
// an infinite radius, which no test certifies.  The warps after those compute
// the operator norm of every prefix's pole-form matrix (one thread per slot;
// the FP64 norm from the FP32 one where that is finite and nonzero, since the
// FP32 entries are the FP64 ones rounded).
__global__ void __launch_bounds__(128) disk_kernel(Plan L, Tables T) {
  pdl_trigger();
  pdl_wait();
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= L.ndisks) {
    const uint32_t slot = (warp - L.ndisks) * 32u + lane;
    if (slot < 4u * L.np) {
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
    return;
  }
  uint32_t l = 0;
  while (l + 1 < L.clev && L.cdisk[l + 1] <= warp) ++l;
  const uint32_t rem = warp - L.cdisk[l];
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
    T.disk32[warp] = make_float4(cx, cy, r32, 0.0f);
    Disk64 D;
    D.cr = cx;
    D.ci = cy;
    D.rho = finite ? ((double)r32 + (double)amax * 0x1p-23) * (1.0 + 0x1p-40)
                   : __longlong_as_double(0x7FF0000000000000ll);
    D.pad = 0.0;
    T.disk64[warp] = D;
  }
}

// Culling levels of a plan in shared memory (the kernels index them by a
// run-time level).
struct CullLevels {
  uint32_t sz[kMaxCullLevels], nb[kMaxCullLevels], disk[kMaxCullLevels];
};

__device__ __forceinline__ void load_levels(const Plan& L, CullLevels* C) {
  if (threadIdx.x < (unsigned)kMaxCullLevels) {
    C->sz[threadIdx.x] = L.csz[threadIdx.x];
    C->nb[threadIdx.x] = L.cnb[threadIdx.x];
    C->disk[threadIdx.x] = L.cdisk[threadIdx.x];
  }
  __syncthreads();
}

// Stack entry: prefix slot (bits 0-31), suffix letter (32-33), level (34-36),
// FP64 flag (37: a mixed render's fallback prefix), block (38-63).
__device__ __forceinline__ unsigned long long cull_entry(uint32_t slot, uint32_t u, uint32_t l,
                                                         bool f64, uint32_t b) {
  return (unsigned long long)slot | ((unsigned long long)u << 32) |
         ((unsigned long long)l << 34) | ((unsigned long long)f64 << 37) |
         ((unsigned long long)b << 38);
}

// Culled render, both precisions.  Items of 32 prefixes x a chunk of top
// blocks, one prefix per lane, each block tested and its failing children
// pushed; whenever the warp's stack holds 32 entries they are tested, one per
// lane.  In a mixed render the fallback prefixes (near-parabolic, direct-form
// and far) take the FP64 tests and FP64 words, as in the per-word render.
template <int BT, bool MIXED>
__global__ void __launch_bounds__(BT, 1024 / BT) cull_kernel(
    Tables T, Plan L, View V, Work Wk, uint32_t* __restrict__ img,
    unsigned long long* counters) {
  __shared__ unsigned long long s_stack[BT / 32][kCullStack];
  __shared__ unsigned long long s_leaf[BT / 32][kLeafQueue];
  __shared__ CullLevels C;
  load_levels(L, &C);
  pdl_wait();
  const uint32_t top = L.clev - 1;
  const uint32_t lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long* stack = s_stack[threadIdx.x >> 5];
  unsigned long long* leafq = s_leaf[threadIdx.x >> 5];
  uint32_t len = 0, lq = 0;
  Tally t;
  uint32_t words = 0, fp64_words = 0;

  // all words of block b (level l) of letter u under slot, one by one
  auto block_words = [&](uint32_t slot, uint32_t u, uint32_t l, bool f64, uint32_t b) {
    const uint32_t j0 = b * C.sz[l];
    if (MIXED && !f64) {
      mixed_block_words(slot, (int)u, j0, C.sz[l], L, V, T, t, words, img);
    } else {
      words64(T.pre64[slot], T.flags[slot] & kDirect, T.suf64 + (size_t)u * L.ns, j0,
              j0 + C.sz[l], V, t, img);
      words += C.sz[l];
      if (MIXED) fp64_words += C.sz[l];
    }
  };
  auto drain_leaves = [&](uint32_t n) {  // leaf queue entries [0, n), one per lane
    if (lane < n) {
      const unsigned long long e = leafq[lane];
      block_words((uint32_t)e, (uint32_t)(e >> 32) & 3u, 0u, (e >> 37) & 1ull,
                  (uint32_t)(e >> 38));
    }
    __syncwarp();
  };
  // certified pixel of (slot, u, l, b), or kUncertified
  auto test = [&](uint32_t slot, uint32_t u, uint32_t l, bool f64, uint32_t b) -> int {
    const uint32_t di = C.disk[l] + u * C.nb[l] + b;
    if (MIXED && !f64) return block_pixel32(T.pre32[slot], T.nrm32[slot], T.disk32[di], V);
    if (T.flags[slot] & kDirect) return kUncertified;
    return block_pixel64(T.pre64[slot], T.nrm64[slot], T.disk64[di], V);
  };
  // the outcome of one test per lane (act: this lane tested an entry)
  auto settle = [&](bool act, uint32_t slot, uint32_t u, uint32_t l, bool f64, uint32_t b,
                    int pix) {
    if (act && pix != kUncertified) {
      t.add_n(pix, C.sz[l], img);
      words += C.sz[l];
      if (MIXED && f64) fp64_words += C.sz[l];
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
    if ((kids && !pushed) || direct) block_words(slot, u, l, f64, b);
    const unsigned bl = __ballot_sync(0xFFFFFFFFu, leaf);
    if (leaf) leafq[lq + __popc(bl & lt)] = cull_entry(slot, u, 0, f64, b);
    lq += __popc(bl);
    __syncwarp();
    if (lq >= 32) {
      drain_leaves(32);
      lq -= 32;
      if (lane < lq) leafq[lane] = leafq[32 + lane];
      __syncwarp();
    }
  };
  // one round: the top n (<= 32) stack entries, one per lane
  auto round = [&](uint32_t n) {
    unsigned long long e = 0;
    if (lane < n) e = stack[len - n + lane];
    __syncwarp();
    len -= n;
    const bool act = lane < n;
    const uint32_t slot = (uint32_t)e, u = (uint32_t)(e >> 32) & 3u;
    const uint32_t l = (uint32_t)(e >> 34) & 7u, b = (uint32_t)(e >> 38);
    const bool f64 = (e >> 37) & 1ull;
    settle(act, slot, u, l, f64, b, act ? test(slot, u, l, f64, b) : kUncertified);
  };

  for (;;) {
    const uint32_t item = next_item_warp(T.fbcount + 1);
    if (item >= Wk.n_items) break;
    int x, u;
    uint32_t pb, c;
    item_of(item, Wk, x, u, pb, c);
    const uint32_t r = pb * 32 + lane;
    const uint32_t slot = (uint32_t)x * L.np + r;
    const bool live = r < L.np;
    const bool f64 = !MIXED || (live && (T.flags[slot] & kFallback));
    const uint32_t b0 = c * Wk.chunk, b1 = min(C.nb[top], b0 + Wk.chunk);
    for (uint32_t b = b0; b < b1; ++b) {
      settle(live, slot, (uint32_t)u, top, f64, b,
             live ? test(slot, (uint32_t)u, top, f64, b) : kUncertified);
      while (len >= 32) round(32);
    }
  }
  while (len > 0) round(min(len, 32u));
  drain_leaves(lq);
  t.flush(img);
  publish_counts(t.in_window, words, fp64_words, t.atomics, counters);
}

// ---------------------------------------------------------------------------
// decode, sequential words (d = 1) and evaluation

__global__ void decode_kernel(const uint64_t* __restrict__ idx, uint64_t n, int d, uint64_t N,
                              uint8_t* __restrict__ out) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = idx[t];
    uint8_t* o = out + t * (uint64_t)d;
    if (i >= N) {
      for (int k = 0; k < d; ++k) o[k] = 0xFF;
      continue;
    }
    int w[KL_MAX_DEPTH];
    decode_word(i, d, w);
    for (int k = 0; k < d; ++k) o[k] = (uint8_t)w[k];
  }
}

// Words of length 1: the map of the letter applied to its own seed.
__global__ void render_single_letter_kernel(Group G, View V, uint32_t* img,
                                            unsigned long long* counters) {
  const int x = threadIdx.x;
  if (x >= 4) return;
  dc z = mobius(load_gen(G, x), {G.seed[2 * x], G.seed[2 * x + 1]});
  const int pix = pixel64((z.re - V.x0) * V.sx, (V.y1 - z.im) * V.sy, V);
  if (pix >= 0) atomicAdd(img + pix, 1u);
  if (counters) {
    atomicAdd(counters + (pix >= 0 ? KL_CNT_IN_WINDOW : KL_CNT_DROPPED), 1ull);
    if (pix >= 0) atomicAdd(counters + KL_CNT_ATOMICS, 1ull);
  }
}

// Tiling mode, the short lengths 1..k0: one thread per node, its word
// decoded from the node's index within its length and evaluated point by
// point from the inside out (the seed of w_k, then the maps of w_k, ..., w_1),
// in FP64 with a refined reciprocal instead of division.  These lengths hold
// few words (2 (3^k0 - 1)), so one launch for all of them replaces a render
// per length, whose launches would cost more than its words.
constexpr uint32_t kShortTiling = 9;

__global__ void tiling_short_kernel(Group G, View V, uint32_t k0, int mixed,
                                    uint32_t* __restrict__ img, unsigned long long* counters) {
  uint64_t total = 0, nk = 4;
  for (uint32_t k = 1; k <= k0; ++k, nk *= 3) total += nk;
  uint32_t in_window = 0, words = 0, atomics = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t r = i, n = 4;
    uint32_t k = 1;
    while (r >= n) {
      r -= n;
      n *= 3;
      ++k;
    }
    int w[kShortTiling];
    decode_word(r, (int)k, w);
    dc z = {G.seed[2 * w[k - 1]], G.seed[2 * w[k - 1] + 1]};
    for (int j = (int)k - 1; j >= 0; --j) {
      const double* M = G.g + 8 * w[j];
      const dc num = {M[0] * z.re - M[1] * z.im + M[2], M[0] * z.im + M[1] * z.re + M[3]};
      const dc den = {M[4] * z.re - M[5] * z.im + M[6], M[4] * z.im + M[5] * z.re + M[7]};
      const double rc = rcp64(den.re * den.re + den.im * den.im);
      z = {(num.re * den.re + num.im * den.im) * rc, (num.im * den.re - num.re * den.im) * rc};
    }
    const int pix = pixel64((z.re - V.x0) * V.sx, (V.y1 - z.im) * V.sy, V);
    ++words;
    if (pix >= 0) {
      atomicAdd(img + pix, 1u);
      ++in_window;
      ++atomics;
    }
  }
  publish_counts(in_window, words, mixed ? words : 0u, atomics, counters);
}

__global__ void eval_kernel(const uint64_t* __restrict__ idx, uint64_t n, uint64_t N, Group G,
                            Plan L, View V, int mixed, Tables T, double* __restrict__ out) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = idx[t];
    double uu = __longlong_as_double(0x7FF8000000000000ll), vv = uu;
    if (i < N) {
      int w[kMaxRenderDepth];
      decode_word(i, L.d, w);
      if (L.d == 1) {
        const int x = w[0];
        dc z = mobius(load_gen(G, x), {G.seed[2 * x], G.seed[2 * x + 1]});
        uu = (z.re - V.x0) * V.sx;
        vv = (V.y1 - z.im) * V.sy;
      } else {
        uint32_t r = 0;
        for (int k = L.p - 2; k >= 0; --k) {
          const int ban = (w[k + 1] + 2) & 3;
          r = 3u * r + (uint32_t)(w[k] - (w[k] > ban ? 1 : 0));
        }
        const uint32_t slot = (uint32_t)w[L.p - 1] * L.np + r;
        const uint32_t jj = (uint32_t)(i % (uint64_t)L.ns);
        const uint32_t sslot = (uint32_t)w[L.p] * L.ns + jj;
        const uint32_t fl = T.flags[slot];
        if (mixed && !(fl & kFallback)) {
          const Pre32 c = T.pre32[slot];
          const float4 e = T.suf32p[(uint64_t)w[L.p] * L.npairs + jj / 2u];
          float uf, vf;
          uv_pole32(c, (jj & 1u) ? e.y : e.x, (jj & 1u) ? e.w : e.z, uf, vf);
          uu = (double)c.axi + (double)uf;
          vv = (double)c.ayi + (double)vf;
        } else if (fl & kDirect) {
          const double2 s = T.suf64[sslot];
          uv_direct64(T.pre64[slot], s.x, s.y, V, uu, vv);
        } else {
          const double2 s = T.suf64[sslot];
          uv_pole64(T.pre64[slot], s.x, s.y, uu, vv);
        }
      }
      if (!isfinite(uu) || !isfinite(vv)) {
        uu = __longlong_as_double(0x7FF8000000000000ll);
        vv = uu;
      }
    }
    out[2 * t] = uu;
    out[2 * t + 1] = vv;
  }
}

// ---------------------------------------------------------------------------
// host side

// caller events recorded around the main per-word kernel (kl_set_profile_events)
cudaEvent_t g_prof_start = nullptr, g_prof_stop = nullptr;

int prof_mark(cudaEvent_t e, cudaStream_t s) {
  if (!e) return KL_OK;
  return cudaEventRecord(e, s) == cudaSuccess ? KL_OK : KL_ECUDA;
}

// Tables of a render: parts (with the image clearing of C riding along),
// then combine, launched as a programmatic dependent of parts.
int build_tables(const kl_params* p, const Plan& L, const View& V, const Group& G,
                 const Tables& T, cudaStream_t st, const Clear& C = Clear{}) {
  const int mixed = p->precision == KL_MIXED;
  const uint32_t nParts = parts_count(L);
  const uint32_t part_blocks = (nParts + kPartLanes - 1) / kPartLanes;
  uint32_t clear_blocks = 0;
  if (C.words) {
    const int sms = sm_count();
    if (sms <= 0) return KL_ECUDA;
    const size_t need = (C.words / 4 + 31) / 32;  // 16-byte stores, 32-thread blocks
    clear_blocks = (uint32_t)(need < (size_t)sms * 8 ? (need > 0 ? need : 1) : (size_t)sms * 8);
  }
  parts_kernel<<<part_blocks + clear_blocks, 32, 0, st>>>(G, L, (int)p->renorm_every, T, C,
                                                          part_blocks);
  if (check_launch() != KL_OK) return KL_ECUDA;
  const uint32_t n = combine_count(L);
  return launch_dependent(combine_kernel, dim3((n + 127) / 128), dim3(128), st, V, L,
                          p->parabolic_tol, mixed, T);
}

// Length k of a tiling render of *p: a limit-set render of the words of
// length k; the caller's prefix length applies to length d only.
kl_params length_params(const kl_params* p, uint32_t k) {
  kl_params q = *p;
  q.depth = k;
  q.mode = KL_LIMIT_SET;
  if (k != p->depth) q.prefix_len = 0;
  return q;
}

// Workspace bytes of *p (tiling: the largest over its lengths), or 0.
size_t plan_bytes(const kl_params* p) {
  if (!p || !valid_view(p)) return 0;
  if (p->mode != KL_LIMIT_SET && p->mode != KL_TILING) return 0;
  Plan L;
  if (make_plan(p, &L, false) != KL_OK) return 0;
  size_t most = L.total;
  if (p->mode == KL_TILING) {
    for (uint32_t k = 1; k < p->depth; ++k) {
      const kl_params q = length_params(p, k);
      if (make_plan(&q, &L, false) != KL_OK) return 0;
      most = L.total > most ? L.total : most;
    }
  }
  return most;
}

int validate(const kl_params* p, size_t ws_bytes, void* ws, Plan* L) {
  if (!p || !valid_view(p)) return KL_EINVAL;
  if (p->precision != KL_FP64 && p->precision != KL_MIXED) return KL_EINVAL;
  if (p->mode != KL_LIMIT_SET && p->mode != KL_TILING) return KL_EINVAL;
  if (p->cull > 1) return KL_EINVAL;
  if (!(p->parabolic_tol >= 0.0)) return KL_EINVAL;
  const int st = make_plan(p, L, false);
  if (st != KL_OK) return st;
  if (L->d > 1) {
    if (!ws) return KL_EINVAL;
    if (((uintptr_t)ws & 255u) != 0) return KL_EINVAL;
    const size_t need = plan_bytes(p);
    if (need == 0) return KL_EINVAL;
    if (ws_bytes < need) return KL_ENOSPACE;
  }
  return KL_OK;
}

template <int BT>
int launch_render(const kl_params* p, const Plan& L, const View& V, const Tables& T,
                  uint32_t* img, unsigned long long* cnt, cudaStream_t s, bool profile) {
  const cudaEvent_t ev0 = profile ? g_prof_start : nullptr, ev1 = profile ? g_prof_stop : nullptr;
  int sms = 0, occ = 0;
  if (p->cull) {
    // block disks (a programmatic dependent of combine), then the culled render
    const uint32_t warps = L.ndisks + (4u * L.np + 31u) / 32u;
    if (launch_dependent(disk_kernel, dim3((warps + 3u) / 4u), dim3(128), s, L, T) != KL_OK)
      return KL_ECUDA;
    const bool mixed = p->precision == KL_MIXED;
    const void* k = mixed ? (const void*)cull_kernel<BT, true> : (const void*)cull_kernel<BT, false>;
    if (device_slots(k, BT, &sms, &occ) != KL_OK) return KL_ECUDA;
    // warp-sized items: 32 prefixes x a chunk of top-level blocks (one by default)
    const Work Wk = make_work(L, 32, L.cnb[L.clev - 1], sms * occ * (BT / 32),
                              p->chunk_pairs ? p->chunk_pairs : 1u);
    if (prof_mark(ev0, s) != KL_OK) return KL_ECUDA;
    const int st = mixed ? launch_dependent(cull_kernel<BT, true>, dim3(sms * occ), dim3(BT), s,
                                            T, L, V, Wk, img, cnt)
                         : launch_dependent(cull_kernel<BT, false>, dim3(sms * occ), dim3(BT),
                                            s, T, L, V, Wk, img, cnt);
    if (st != KL_OK) return KL_ECUDA;
    return prof_mark(ev1, s);
  }
  if (p->precision == KL_FP64) {
    if (device_slots((const void*)render64_kernel<BT>, BT, &sms, &occ) != KL_OK) return KL_ECUDA;
    const Work Wk = make_work(L, BT, L.ns, sms * occ, 2u * p->chunk_pairs);
    if (prof_mark(ev0, s) != KL_OK) return KL_ECUDA;
    if (launch_dependent(render64_kernel<BT>, dim3(sms * occ), dim3(BT), s, T, L, V, Wk, img,
                         cnt) != KL_OK)
      return KL_ECUDA;
    return prof_mark(ev1, s);
  }
  if (device_slots((const void*)render_mixed_kernel<BT>, BT, &sms, &occ) != KL_OK)
    return KL_ECUDA;
  // warp-sized items (32 prefixes), about 12 per resident warp
  const Work Wk = make_work(L, 32, L.npairs, sms * occ * (BT / 32), p->chunk_pairs);
  if (prof_mark(ev0, s) != KL_OK) return KL_ECUDA;
  if (launch_dependent(render_mixed_kernel<BT>, dim3(sms * occ), dim3(BT), s, T, L, V, Wk, img,
                       cnt) != KL_OK)
    return KL_ECUDA;
  return prof_mark(ev1, s);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI

extern "C" size_t kl_workspace_bytes(const kl_params* p) { return plan_bytes(p); }

extern "C" int kl_decode_words(uint32_t depth, const uint64_t* d_index, uint64_t n,
                               uint8_t* d_letters, void* stream) {
  if (depth < 1 || depth > KL_MAX_DEPTH) return KL_EINVAL;
  if (n == 0) return KL_OK;
  if (!d_index || !d_letters) return KL_EINVAL;
  const int sms = sm_count();
  if (sms <= 0) return KL_ECUDA;
  const uint64_t blocks = (n + 127) / 128;
  const unsigned g = (unsigned)(blocks < (uint64_t)sms * 16 ? blocks : (uint64_t)sms * 16);
  decode_kernel<<<g, 128, 0, (cudaStream_t)stream>>>(d_index, n, (int)depth,
                                                     kl_word_count(depth), d_letters);
  return check_launch();
}

extern "C" int kl_eval_words(const kl_params* p, const uint64_t* d_index, uint64_t n,
                             double* d_uv, void* d_workspace, size_t workspace_bytes,
                             void* stream) {
  Plan L;
  int st = validate(p, workspace_bytes, d_workspace, &L);
  if (st != KL_OK) return st;
  if (n == 0) return KL_OK;
  if (!d_index || !d_uv) return KL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const View V = make_view(p);
  const Group G = make_group(p);
  Tables T{};
  if (L.d > 1) {
    T = carve(L, d_workspace);
    st = build_tables(p, L, V, G, T, s);
    if (st != KL_OK) return st;
  }
  const int sms = sm_count();
  if (sms <= 0) return KL_ECUDA;
  const uint64_t blocks = (n + 127) / 128;
  const unsigned g = (unsigned)(blocks < (uint64_t)sms * 16 ? blocks : (uint64_t)sms * 16);
  eval_kernel<<<g, 128, 0, s>>>(d_index, n, kl_word_count(p->depth), G, L, V,
                                p->precision == KL_MIXED, T, d_uv);
  return check_launch();
}

namespace {

// One limit-set render of *p (already validated).
int render_length(const kl_params* p, uint32_t* d_image, unsigned long long* cnt,
                  void* d_workspace, cudaStream_t s, bool profile) {
  Plan L;
  int st = make_plan(p, &L, false);
  if (st != KL_OK) return st;
  const View V = make_view(p);
  const Group G = make_group(p);
  if (L.d == 1) {
    if (!p->accumulate) {
      if (cudaMemsetAsync(d_image, 0, (size_t)p->width * p->height * sizeof(uint32_t), s) !=
          cudaSuccess)
        return KL_ECUDA;
      if (cnt && cudaMemsetAsync(cnt, 0, KL_N_COUNTERS * sizeof(uint64_t), s) != cudaSuccess)
        return KL_ECUDA;
    }
    render_single_letter_kernel<<<1, 32, 0, s>>>(G, V, d_image, cnt);
    return check_launch();
  }
  const Tables T = carve(L, d_workspace);
  Clear C{};
  if (!p->accumulate) C = {d_image, (size_t)p->width * p->height, cnt};
  st = build_tables(p, L, V, G, T, s, C);
  if (st != KL_OK) return st;
  switch (p->block_threads) {
    case 64: return launch_render<64>(p, L, V, T, d_image, cnt, s, profile);
    case 256: return launch_render<256>(p, L, V, T, d_image, cnt, s, profile);
    default: return launch_render<128>(p, L, V, T, d_image, cnt, s, profile);
  }
}

}  // namespace

extern "C" int kl_render(const kl_params* p, uint32_t* d_image, uint64_t* d_counters,
                         void* d_workspace, size_t workspace_bytes, void* stream) {
  Plan L;
  int st = validate(p, workspace_bytes, d_workspace, &L);
  if (st != KL_OK) return st;
  if (!d_image) return KL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* cnt = (unsigned long long*)d_counters;
  if (p->mode == KL_TILING) {
    // the lengths above kShortTiling as renders of their own, the longest
    // first (it clears the image unless accumulating), each next one added
    // in; then all the short lengths in one launch
    const uint32_t k0 = p->depth < kShortTiling ? p->depth : kShortTiling;
    for (uint32_t k = p->depth; k > k0; --k) {
      kl_params q = length_params(p, k);
      q.accumulate = k == p->depth ? p->accumulate : 1u;
      st = render_length(&q, d_image, cnt, d_workspace, s, k == p->depth);
      if (st != KL_OK) return st;
    }
    if (p->depth <= k0 && !p->accumulate) {
      if (cudaMemsetAsync(d_image, 0, (size_t)p->width * p->height * sizeof(uint32_t), s) !=
          cudaSuccess)
        return KL_ECUDA;
      if (cnt && cudaMemsetAsync(cnt, 0, KL_N_COUNTERS * sizeof(uint64_t), s) != cudaSuccess)
        return KL_ECUDA;
    }
    const int sms = sm_count();
    if (sms <= 0) return KL_ECUDA;
    tiling_short_kernel<<<sms * 4, 256, 0, s>>>(make_group(p), make_view(p), k0,
                                                p->precision == KL_MIXED, d_image, cnt);
    return check_launch();
  }
  return render_length(p, d_image, cnt, d_workspace, s, true);
}

extern "C" int kl_set_profile_events(void* ev_start, void* ev_stop) {
  if ((ev_start == nullptr) != (ev_stop == nullptr)) return KL_EINVAL;
  g_prof_start = (cudaEvent_t)ev_start;
  g_prof_stop = (cudaEvent_t)ev_stop;
  return KL_OK;
}

// ---------------------------------------------------------------------------
// kl_render without allocation: the workspace is a static device array of this
// file.  In host code the symbol g_noalloc_scratch is only a host-side stand-in,
// so its device address is looked up once per device (with that device
// current) and cached.

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[KL_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KL_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return KL_ERANGE;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return KL_ECUDA;
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return KL_OK;
}

}  // namespace

extern "C" int kl_render_noalloc(const kl_params* p, uint32_t* d_image, uint64_t* d_counters,
                                 void* stream) {
  if (!p) return KL_EINVAL;
  if (kl_workspace_bytes(p) > KL_STATIC_SCRATCH_BYTES) return KL_ENOSPACE;
  void* scratch = nullptr;
  const int st = noalloc_scratch(&scratch);
  if (st != KL_OK) return st;
  return kl_render(p, d_image, d_counters, scratch, KL_STATIC_SCRATCH_BYTES, stream);
}
