// Host helpers of the render entry points: plans (the prefix/suffix split
// and a shard's prefix slots), workspace carving, work queues and launches.
// Included at the end of kl_common.cuh.
#pragma once

#include "kl_common.cuh"

namespace {

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
  // The prefix side first: its offsets depend only on the prefix (its length,
  // the shard, the precision and culling), so two plans with the same prefix
  // find each other's prefix tables in the same place (prefix_tables_shared).
  const size_t nP = 4ull * L->np, nS = 4ull * L->ns;
  const bool df = p->precision == KL_DF64;
  // disks and prefix norms exist in culled plans only
  const size_t nD = p->cull ? L->ndisks : 0, nN = p->cull ? nP : 0;
  size_t off = 0;
  L->off_pre64 = off; off = align256(off + nP * sizeof(Pre64));
  L->off_pre32 = off; off = align256(off + nP * sizeof(Pre32));
  L->off_flags = off; off = align256(off + nP * sizeof(uint32_t));
  L->off_fb = off; off = align256(off + nP * sizeof(unsigned long long));
  L->off_fbcount = off; off = align256(off + 2 * sizeof(uint32_t));  // fallback count, queue
  L->off_L = off; off = align256(off + 4ull * L->p3_q1 * sizeof(PartM));
  L->off_H = off; off = align256(off + 4ull * L->p3_pq * sizeof(M2));
  L->off_nrm32 = off; off = align256(off + nN * sizeof(float));
  L->off_nrm64 = off; off = align256(off + nN * sizeof(double));
  // double-float constants and suffix pairs exist in KL_DF64 plans only
  L->off_predf = off; off = align256(off + (df ? nP : 0) * sizeof(PreDF));
  // the suffix side
  L->off_suf64 = off; off = align256(off + nS * sizeof(double2));
  L->off_suf32 = off; off = align256(off + 4ull * L->npairs * sizeof(float4));
  L->off_So = off; off = align256(off + 4ull * L->p3_so1 * sizeof(PartM));
  L->off_Si = off; off = align256(off + 4ull * L->p3_si1 * sizeof(double2));
  L->off_disk32 = off; off = align256(off + nD * sizeof(float4));
  L->off_disk64 = off; off = align256(off + nD * sizeof(Disk64));
  L->off_sufdf = off; off = align256(off + (df ? 8ull * L->npairs : 0) * sizeof(float4));
  L->total = off;
  return KL_OK;
}

// Whether a plan B built after plan A (same parameters apart from the word
// length) can use A's prefix tables as they are: the same prefix length and
// shard, and neither culled (culled plans also hold per-prefix norms computed
// with their own suffix blocks).
inline bool prefix_tables_shared(const Plan& A, const Plan& B, const kl_params* p) {
  return !p->cull && A.p == B.p && A.q == B.q && A.np == B.np && A.r0 == B.r0 &&
         A.nr == B.nr && B.off_suf64 == A.off_suf64;
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
