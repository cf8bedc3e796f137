// Single render, decode and evaluation entry points of the C ABI (sm_103a).
// The arithmetic, tables and per-item bodies are in kl_common.cuh and the
// headers it includes (kl_df.cuh, kl_cull.cuh, kl_plan.cuh).
#include <cmath>
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
// Entries [first, parts_count) of the parts tables; first > 0 (the prefix
// parts skipped) when the prefix tables are already in place, whose fallback
// count is then kept.
__global__ void parts_kernel(Group G, Plan L, int renorm, Tables T, Clear C,
                             uint32_t part_blocks, uint32_t first) {
  pdl_trigger();
  if (blockIdx.x < part_blocks) {
    if (blockIdx.x == 0) {
      if (threadIdx.x == 0 && first == 0) T.fbcount[0] = 0u;  // fallback prefixes
      if (threadIdx.x == 1) T.fbcount[1] = 0u;                // the work queue
      if (C.counters && threadIdx.x < KL_N_COUNTERS) C.counters[threadIdx.x] = 0ull;
    }
    // kPartLanes entries per block: each entry is one long chain of dependent
    // FP64 operations, so spreading the entries over more SMs shortens the
    // launch more than filling warps does
    const uint32_t total = parts_count(L);
    if (threadIdx.x < kPartLanes)
      for (uint32_t idx = first + blockIdx.x * kPartLanes + threadIdx.x; idx < total;
           idx += part_blocks * kPartLanes)
        part_entry(G, L, renorm, idx, T);
    return;
  }
  clear_words(C.img, C.words, (size_t)(blockIdx.x - part_blocks) * blockDim.x + threadIdx.x,
              (size_t)(gridDim.x - part_blocks) * blockDim.x);
}

// Entries [first, combine_count): first = 4 nr (the prefixes skipped) when
// the prefix tables are already in place.
__global__ void combine_kernel(View V, Plan L, double ptol, int prec, Tables T, uint32_t first) {
  pdl_trigger();
  pdl_wait();
  const uint32_t total = combine_count(L);
  for (uint32_t idx = first + blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += gridDim.x * blockDim.x)
    combine_entry(V, L, ptol, prec, idx, T, 0u, T.fb, T.fbcount);
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
// 48 registers (10 blocks of 128 threads per SM): at 40 the loop and the
// fallback call spill; 48 measured 1-2% faster than 40 and than 64.
template <int BT>
__global__ void __launch_bounds__(BT, 1280 / BT) render_mixed_kernel(
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

// Double-float (KL_DF64): the queue holds first the FP64 fallback items (the
// direct-form, far and out-of-float-range prefixes), then the double-float
// items (32 prefixes x one chunk of suffix pairs), drawn per warp like the
// mixed render's.  The per-word map is 117 FP32 operations in dependent
// double-float chains, so the FMA pipe and the chains' latency, not issue,
// bound the loop.  72 registers (7 blocks of 128 threads per SM): 2% faster
// than at 82 registers (5 blocks) and than at 64 (8 blocks, spilling in the
// loop); at 72 a few values are spilled per work item, not per word (local
// loads are 0.01% of the instructions).
template <int BT>
__global__ void __launch_bounds__(BT, 896 / BT) render_df64_kernel(
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
    df64_item<32>(item - n64, Wk, L, V, T, t, words, img);
  }
  publish_counts(t.in_window, words, fp64_words, t.atomics, counters);
}

// ---------------------------------------------------------------------------
// culled renders (kl_params.cull; the culling itself is in kl_cull.cuh)

// Disks of all culling blocks, then the prefix norms (cull_disk_unit).
__global__ void __launch_bounds__(128) disk_kernel(Plan L, Tables T) {
  pdl_trigger();
  pdl_wait();
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp < cull_disk_units(L)) cull_disk_unit(L, T, warp, threadIdx.x & 31);
}

// Culled render of one group: persistent warps take items of 32 prefixes x
// one top-level block from the work queue.
template <int BT, bool MIXED>
__global__ void __launch_bounds__(BT, 1024 / BT) cull_kernel(
    Tables T, Plan L, View V, Work Wk, uint32_t* __restrict__ img,
    unsigned long long* counters) {
  __shared__ unsigned long long s_stack[BT / 32][kCullStack];
  __shared__ unsigned long long s_leaf[BT / 32][kLeafQueue];
  __shared__ CullLevels C;
  if (threadIdx.x < (unsigned)kMaxCullLevels) {
    C.sz[threadIdx.x] = L.csz[threadIdx.x];
    C.nb[threadIdx.x] = L.cnb[threadIdx.x];
    C.disk[threadIdx.x] = L.cdisk[threadIdx.x];
  }
  __syncthreads();
  pdl_wait();
  CullWarp<MIXED> w(s_stack[threadIdx.x >> 5], s_leaf[threadIdx.x >> 5], &C);
  const uint32_t top_blocks = L.cnb[L.clev - 1];
  for (;;) {
    const uint32_t item = next_item_warp(T.fbcount + 1);
    if (item >= Wk.n_items) break;
    cull_item(w, item, Wk, L, V, T, img, top_blocks);
  }
  w.finish(L, V, T, img);
  w.t.flush(img);
  publish_counts(w.t.in_window, w.words, w.fp64_words, w.t.atomics, counters);
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

__global__ void tiling_short_kernel(Group G, View V, uint32_t k0, int fp64_count,
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
  publish_counts(in_window, words, fp64_count ? words : 0u, atomics, counters);
}

__global__ void eval_kernel(const uint64_t* __restrict__ idx, uint64_t n, uint64_t N, Group G,
                            Plan L, View V, int prec, Tables T, double* __restrict__ out) {
  const bool mixed = prec == KL_MIXED, df = prec == KL_DF64;
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
        } else if (df && !(fl & kFallback)) {
          // the render's pair arithmetic, with this word in both halves
          const DfConst K = df_const(T.predf[slot]);
          const float4* q = T.sufdf + 2ull * ((uint64_t)w[L.p] * L.npairs + jj / 2u);
          const float4 a = q[0], b = q[1];
          const bool odd = jj & 1u;
          const float rh = odd ? a.y : a.x, rl = odd ? a.w : a.z;
          const float ih = odd ? b.y : b.x, il = odd ? b.w : b.z;
          const DD vr = {pk(rh, rh), pk(rl, rl)}, vi = {pk(ih, ih), pk(il, il)};
          DD U, Vv;
          uv_df2(K, vr, vi, U, Vv);
          uu = (double)__uint_as_float((uint32_t)U.hi) + (double)__uint_as_float((uint32_t)U.lo);
          vv = (double)__uint_as_float((uint32_t)Vv.hi) +
               (double)__uint_as_float((uint32_t)Vv.lo);
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

// caller events recorded around the main per-word kernel (kl_set_profile_events),
// one setting per host thread
thread_local cudaEvent_t g_prof_start = nullptr, g_prof_stop = nullptr;

int prof_mark(cudaEvent_t e, cudaStream_t s) {
  if (!e) return KL_OK;
  return cudaEventRecord(e, s) == cudaSuccess ? KL_OK : KL_ECUDA;
}

// Tables of a render: parts (with the image clearing of C riding along),
// then combine, launched as a programmatic dependent of parts.
// The tables of plan L; with prefix_ready the prefix tables (and the list of
// fallback prefixes) are taken as they are and only the suffix side is built.
int build_tables(const kl_params* p, const Plan& L, const View& V, const Group& G,
                 const Tables& T, cudaStream_t st, const Clear& C = Clear{},
                 bool prefix_ready = false) {
  const int prec = (int)p->precision;
  const uint32_t first_part = prefix_ready ? 4u * L.p3_q1 + (L.p > L.q ? 4u * L.p3_pq : 0u) : 0u;
  const uint32_t first_comb = prefix_ready ? 4u * L.nr : 0u;
  const uint32_t nParts = parts_count(L) - first_part;
  const uint32_t part_blocks = nParts > 0 ? (nParts + kPartLanes - 1) / kPartLanes : 1u;
  uint32_t clear_blocks = 0;
  if (C.words) {
    const int sms = sm_count();
    if (sms <= 0) return KL_ECUDA;
    const size_t need = (C.words / 4 + 31) / 32;  // 16-byte stores, 32-thread blocks
    clear_blocks = (uint32_t)(need < (size_t)sms * 8 ? (need > 0 ? need : 1) : (size_t)sms * 8);
  }
  parts_kernel<<<part_blocks + clear_blocks, 32, 0, st>>>(G, L, (int)p->renorm_every, T, C,
                                                          part_blocks, first_part);
  if (check_launch() != KL_OK) return KL_ECUDA;
  const uint32_t n = combine_count(L) - first_comb;
  return launch_dependent(combine_kernel, dim3(n > 0 ? (n + 127) / 128 : 1u), dim3(128), st, V,
                          L, p->parabolic_tol, prec, T, first_comb);
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
  if (p->precision != KL_FP64 && p->precision != KL_MIXED && p->precision != KL_DF64)
    return KL_EINVAL;
  if (p->mode != KL_LIMIT_SET && p->mode != KL_TILING) return KL_EINVAL;
  if (p->cull > 1 || (p->cull && p->precision == KL_DF64)) return KL_EINVAL;
  if (p->shard_count > 1 && (p->mode != KL_LIMIT_SET || p->shard_index >= p->shard_count))
    return KL_EINVAL;
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
    const uint32_t warps = cull_disk_units(L);
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
  if (p->precision == KL_DF64) {
    if (device_slots((const void*)render_df64_kernel<BT>, BT, &sms, &occ) != KL_OK)
      return KL_ECUDA;
    const Work Wk = make_work(L, 32, L.npairs, sms * occ * (BT / 32), p->chunk_pairs);
    if (prof_mark(ev0, s) != KL_OK) return KL_ECUDA;
    if (launch_dependent(render_df64_kernel<BT>, dim3(sms * occ), dim3(BT), s, T, L, V, Wk,
                         img, cnt) != KL_OK)
      return KL_ECUDA;
    return prof_mark(ev1, s);
  }
  if (p->precision == KL_FP64) {
    if (device_slots((const void*)render64_kernel<BT>, BT, &sms, &occ) != KL_OK) return KL_ECUDA;
    // items of 64 suffix points by default: an FP64 item is slow (a 128-prefix block on
    // 2,187 points takes milliseconds), so many small items keep the end of the queue
    // even (0.7% faster than about 12 items per block at length 20)
    const Work Wk = make_work(L, BT, L.ns, sms * occ, 2u * (p->chunk_pairs ? p->chunk_pairs : 32u));
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

extern "C" int kl_eval_words(const kl_params* p_in, const uint64_t* d_index, uint64_t n,
                             double* d_uv, void* d_workspace, size_t workspace_bytes,
                             void* stream) {
  if (!p_in) return KL_EINVAL;
  // every word can be asked for: the tables cover all prefix slots
  kl_params q = *p_in;
  q.shard_index = 0;
  q.shard_count = 0;
  const kl_params* p = &q;
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
                                (int)p->precision, T, d_uv);
  return check_launch();
}

namespace {

// One limit-set render of *p (already validated).  prev (if not null) is the
// plan of the render that last built tables in d_workspace, whose prefix
// tables are reused when they serve this plan too (the lengths of a tiling
// render).  *used: this render's plan.
int render_length(const kl_params* p, uint32_t* d_image, unsigned long long* cnt,
                  void* d_workspace, cudaStream_t s, bool profile, const Plan* prev = nullptr,
                  Plan* used = nullptr) {
  Plan L;
  int st = make_plan(p, &L, false);
  if (st != KL_OK) return st;
  if (used) *used = L;
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
    if (L.nr == 0) return KL_OK;  // a shard without the one prefix slot
    render_single_letter_kernel<<<1, 32, 0, s>>>(G, V, d_image, cnt);
    return check_launch();
  }
  const Tables T = carve(L, d_workspace);
  Clear C{};
  if (!p->accumulate) C = {d_image, (size_t)p->width * p->height, cnt};
  st = build_tables(p, L, V, G, T, s, C, prev && prefix_tables_shared(*prev, L, p));
  if (st != KL_OK) return st;
  switch (p->block_threads) {
    case 64: return launch_render<64>(p, L, V, T, d_image, cnt, s, profile);
    case 256: return launch_render<256>(p, L, V, T, d_image, cnt, s, profile);
    default: return launch_render<128>(p, L, V, T, d_image, cnt, s, profile);
  }
}

}  // namespace

namespace {

// A tiling render of *p (already validated): the lengths above kShortTiling
// as renders of their own, the longest first (it clears the image unless
// accumulating), each next one added in; then all the short lengths in one
// launch.  Consecutive lengths with the same prefix length share its prefix
// tables, built once.
int render_tiling(const kl_params* p, uint32_t* d_image, unsigned long long* cnt,
                  void* d_workspace, cudaStream_t s) {
  const uint32_t k0 = p->depth < kShortTiling ? p->depth : kShortTiling;
  Plan prev;
  bool have_prev = false;
  for (uint32_t k = p->depth; k > k0; --k) {
    kl_params q = length_params(p, k);
    q.accumulate = k == p->depth ? p->accumulate : 1u;
    Plan used;
    const int st = render_length(&q, d_image, cnt, d_workspace, s, k == p->depth,
                                 have_prev ? &prev : nullptr, &used);
    if (st != KL_OK) return st;
    prev = used;
    have_prev = used.d > 1;
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
                                              p->precision != KL_FP64, d_image, cnt);
  return check_launch();
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
  if (p->mode == KL_TILING) return render_tiling(p, d_image, cnt, d_workspace, s);
  return render_length(p, d_image, cnt, d_workspace, s, true);
}

extern "C" int kl_render_multiseed(const kl_params* p, const double* points, uint32_t n_points,
                                   uint32_t* d_image, uint64_t* d_counters, void* d_workspace,
                                   size_t workspace_bytes, void* stream) {
  Plan L;
  int st = validate(p, workspace_bytes, d_workspace, &L);
  if (st != KL_OK) return st;
  if (!d_image || !points || n_points == 0) return KL_EINVAL;
  for (uint32_t i = 0; i < 2 * n_points; ++i)
    if (!std::isfinite(points[i])) return KL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* cnt = (unsigned long long*)d_counters;
  Plan prev;
  bool have_prev = false;
  for (uint32_t i = 0; i < n_points; ++i) {
    kl_params q = *p;
    for (int x = 0; x < 4; ++x) {
      q.seeds[2 * x] = points[2 * i];
      q.seeds[2 * x + 1] = points[2 * i + 1];
    }
    q.accumulate = i == 0 ? p->accumulate : 1u;
    if (p->mode == KL_TILING) {
      st = render_tiling(&q, d_image, cnt, d_workspace, s);
    } else {
      // the points' renders differ only in their suffix tables
      Plan used;
      st = render_length(&q, d_image, cnt, d_workspace, s, i == 0, have_prev ? &prev : nullptr,
                         &used);
      prev = used;
      have_prev = used.d > 1;
    }
    if (st != KL_OK) return st;
  }
  return KL_OK;
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
// so its device address is looked up with the calling device current.  The
// lookup (cudaGetSymbolAddress, which allocates nothing) runs on every call
// whose stream is not capturing, so the address always belongs to the context
// current now (a device reset or a different context on the same device gets
// its own address).  A call on a capturing stream cannot look it up and takes
// the address the last uncaptured call on that device found.

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[KL_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

int noalloc_scratch(cudaStream_t stream, void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KL_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return KL_ERANGE;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return KL_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (cap == cudaStreamCaptureStatusNone) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return KL_ECUDA;
    g_noalloc_ptr[dev] = ptr;
  } else if (!g_noalloc_ptr[dev]) {
    return KL_EINVAL;  // no uncaptured call has run on this device yet
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
  const int st = noalloc_scratch((cudaStream_t)stream, &scratch);
  if (st != KL_OK) return st;
  return kl_render(p, d_image, d_counters, scratch, KL_STATIC_SCRATCH_BYTES, stream);
}
