// Batched render (a sweep over many groups of uneven depth) in one persistent
// launch, optionally captured in a CUDA graph.  Every group's words are
// rendered with the same arithmetic as kl_render (kl_common.cuh); what this
// file adds is the flattening of all groups' table entries and work items
// into single index spaces, so that one launch per pass covers the batch and
// one device queue balances groups of very different size (a depth-12 and a
// depth-18 group differ 729-fold in words).
#include <new>
#include <vector>

#include "kl_common.cuh"

namespace {

// Per-group descriptor in device memory.
struct GroupDesc {
  Group G;
  View V;
  Plan L;
  Work Wk;
  Tables T;
  uint32_t* img;
  unsigned long long* cnt;
  double ptol;
  int renorm;
  int pad;
};

// Largest g with bases[g] <= idx (bases ascending, bases[0] = 0).
__device__ __forceinline__ uint32_t find_group(const uint32_t* __restrict__ bases, uint32_t n,
                                               uint32_t idx) {
  uint32_t lo = 0, hi = n;  // bases[lo] <= idx < bases[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(bases + mid) <= idx)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

__global__ void batch_parts_kernel(const GroupDesc* __restrict__ D,
                                   const uint32_t* __restrict__ bases, uint32_t n,
                                   uint32_t total) {
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += gridDim.x * blockDim.x) {
    const uint32_t g = find_group(bases, n, idx);
    const Plan L = D[g].L;
    const Tables T = D[g].T;
    part_entry(D[g].G, L, D[g].renorm, idx - bases[g], T);
  }
}

__global__ void batch_combine_kernel(const GroupDesc* __restrict__ D,
                                     const uint32_t* __restrict__ bases, uint32_t n,
                                     uint32_t total, int mixed, unsigned long long* fb,
                                     uint32_t* fb_count) {
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += gridDim.x * blockDim.x) {
    const uint32_t g = find_group(bases, n, idx);
    const Plan L = D[g].L;
    const View V = D[g].V;
    const Tables T = D[g].T;
    combine_entry(V, L, D[g].ptol, mixed, idx - bases[g], T, g, fb, fb_count);
  }
}

// One persistent launch for the whole batch.  Queue order: all groups' FP64
// fallback units (32 per item; mixed mode only), then every group's items in
// group order.  Counters are published per group whenever a warp moves to
// another group (the item, hence the group, is uniform over the warp, and
// over the block for FP64 items).
// Registers are capped at 48 (10 blocks of 128 threads per SM): the group
// lookup and descriptor spill at the single render's 40, and the batch ran
// 3% faster at 48.
template <int BT, bool MIXED>
__global__ void __launch_bounds__(BT, 1280 / BT) batch_render_kernel(
    const GroupDesc* __restrict__ D, const uint32_t* __restrict__ item_bases, uint32_t n,
    uint32_t n_items, const unsigned long long* __restrict__ fb,
    const uint32_t* __restrict__ fb_count, uint32_t cmax, uint32_t* queue) {
  // mixed items are drawn per warp (32 prefixes each, no block barrier), FP64
  // items per block (BT prefixes)
  constexpr uint32_t IT = MIXED ? 32u : (uint32_t)BT;
  const uint32_t fb_units = MIXED ? 3u * cmax * (*fb_count) : 0u;
  const uint32_t n64 = (fb_units + IT - 1) / IT;
  const uint32_t total = n64 + n_items;
  Tally t;
  uint32_t words = 0;
  int gcur = -1;
  // the current group's items are [glo, ghi): consecutive items of a warp
  // (or block) usually stay in one group, which then needs no search
  uint32_t glo = 0u, ghi = 0u;  // empty: the first item searches
  for (;;) {
    const uint32_t item = MIXED ? next_item_warp(queue) : next_item(queue);
    if (item >= total) break;
    if (MIXED && item < n64) {
      const uint32_t unit = item * IT + (threadIdx.x & 31u);
      if (unit < fb_units) {
        const unsigned long long ent = fb[unit / (3u * cmax)];
        const uint32_t rem = unit % (3u * cmax);
        const uint32_t g = (uint32_t)(ent >> 32), slot = (uint32_t)(ent & 0xFFFFFFFFull);
        const Tables T = D[g].T;
        const UnitTally r = fallback_unit(T.pre64, T.flags, T.suf64, slot, rem / cmax,
                                          rem % cmax, D[g].L.np, D[g].L.ns, D[g].V, D[g].img);
        if (r.words) {
          unsigned long long* c = D[g].cnt;
          atomicAdd(c + KL_CNT_IN_WINDOW, (unsigned long long)r.in_window);
          atomicAdd(c + KL_CNT_DROPPED, (unsigned long long)(r.words - r.in_window));
          atomicAdd(c + KL_CNT_FP64_WORDS, (unsigned long long)r.words);
          atomicAdd(c + KL_CNT_ATOMICS, (unsigned long long)r.atomics);
        }
      }
      continue;
    }
    const uint32_t local = item - n64;
    if (local - glo >= ghi - glo) {  // outside [glo, ghi): another group
      const int g = (int)find_group(item_bases, n, local);
      if (gcur >= 0) publish_counts(t.in_window, words, 0, t.atomics, D[gcur].cnt);
      t = Tally();
      words = 0;
      gcur = g;
      glo = item_bases[g];
      ghi = item_bases[g + 1];
    }
    const int g = gcur;
    const Plan L = D[g].L;
    const View V = D[g].V;
    const Tables T = D[g].T;
    const Work Wk = D[g].Wk;
    if (MIXED)
      mixed_item<32>(local - glo, Wk, L, V, T, t, words, D[g].img);
    else
      fp64_item<BT>(local - glo, Wk, L, V, T, t, words, D[g].img);
  }
  if (gcur >= 0) publish_counts(t.in_window, words, 0, t.atomics, D[gcur].cnt);
}

// Culling disks and prefix norms of every group (culled batches): unit =
// one warp, bases over the groups' units (cull_disk_units each).
__global__ void __launch_bounds__(128) batch_disk_kernel(const GroupDesc* __restrict__ D,
                                                         const uint32_t* __restrict__ bases,
                                                         uint32_t n, uint32_t total) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nw = gridDim.x * (blockDim.x / 32);
  for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
    const uint32_t g = find_group(bases, n, w);
    cull_disk_unit(D[g].L, D[g].T, w - bases[g], lane);
  }
}

// Culled batch in one persistent launch: warps take items (32 prefixes x one
// top-level block of one group) in group order.  A warp that moves to another
// group first finishes the culling of the one it leaves and publishes that
// group's counts, so its stack never mixes groups.
template <int BT, bool MIXED>
__global__ void __launch_bounds__(BT, 1024 / BT) batch_cull_kernel(
    const GroupDesc* __restrict__ D, const uint32_t* __restrict__ item_bases, uint32_t n,
    uint32_t n_items, uint32_t* queue) {
  __shared__ unsigned long long s_stack[BT / 32][kCullStack];
  __shared__ unsigned long long s_leaf[BT / 32][kLeafQueue];
  __shared__ CullLevels s_lev[BT / 32];
  const uint32_t wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  CullWarp<MIXED> w(s_stack[wi], s_leaf[wi], &s_lev[wi]);
  int gcur = -1;
  auto leave = [&]() {  // finish and publish the current group
    const GroupDesc& d = D[gcur];
    w.finish(d.L, d.V, d.T, d.img);
    w.t.flush(d.img);
    publish_counts(w.t.in_window, w.words, w.fp64_words, w.t.atomics, d.cnt);
    w.t = Tally();
    w.words = 0;
    w.fp64_words = 0;
  };
  for (;;) {
    const uint32_t item = next_item_warp(queue);
    if (item >= n_items) break;
    const int g = (int)find_group(item_bases, n, item);
    if (g != gcur) {
      if (gcur >= 0) leave();
      if (lane < (uint32_t)kMaxCullLevels) {
        s_lev[wi].sz[lane] = D[g].L.csz[lane];
        s_lev[wi].nb[lane] = D[g].L.cnb[lane];
        s_lev[wi].disk[lane] = D[g].L.cdisk[lane];
      }
      __syncwarp();
      gcur = g;
    }
    const GroupDesc& d = D[g];
    cull_item(w, item - item_bases[g], d.Wk, d.L, d.V, d.T, d.img, d.L.cnb[d.L.clev - 1]);
  }
  if (gcur >= 0) leave();
}

}  // namespace

// Host handle.
struct kl_batch {
  uint32_t n = 0;
  int mixed = 0;
  int cull = 0;
  int bt = kDefaultThreads;
  uint32_t W = 0, H = 0;
  std::vector<kl_params> params;
  std::vector<Plan> plans;
  std::vector<Work> works;
  std::vector<size_t> table_off;
  std::vector<uint32_t> bases;  // parts [n+1], combine [n+1], items [n+1], disk units [n+1]
  std::vector<GroupDesc> desc;
  size_t off_desc = 0, off_bases = 0, off_fb = 0, off_cnt = 0, total = 0;
  uint32_t n_parts = 0, n_comb = 0, n_items = 0, n_disk = 0, cmax = 1;
  int sms = 0, occ = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

const void* render_fn(int bt, bool mixed, bool cull) {
  if (cull) {
    switch (bt) {
      case 64: return mixed ? (const void*)batch_cull_kernel<64, true>
                            : (const void*)batch_cull_kernel<64, false>;
      case 256: return mixed ? (const void*)batch_cull_kernel<256, true>
                             : (const void*)batch_cull_kernel<256, false>;
      default: return mixed ? (const void*)batch_cull_kernel<128, true>
                            : (const void*)batch_cull_kernel<128, false>;
    }
  }
  if (mixed) {
    switch (bt) {
      case 64: return (const void*)batch_render_kernel<64, true>;
      case 256: return (const void*)batch_render_kernel<256, true>;
      default: return (const void*)batch_render_kernel<128, true>;
    }
  }
  switch (bt) {
    case 64: return (const void*)batch_render_kernel<64, false>;
    case 256: return (const void*)batch_render_kernel<256, false>;
    default: return (const void*)batch_render_kernel<128, false>;
  }
}

template <int BT>
void launch_batch(int grid, cudaStream_t s, bool mixed, bool cull, const GroupDesc* D,
                  const uint32_t* item_bases, uint32_t n, uint32_t n_items,
                  const unsigned long long* fb, uint32_t* cnt2, uint32_t cmax) {
  if (cull && mixed)
    batch_cull_kernel<BT, true><<<grid, BT, 0, s>>>(D, item_bases, n, n_items, cnt2 + 1);
  else if (cull)
    batch_cull_kernel<BT, false><<<grid, BT, 0, s>>>(D, item_bases, n, n_items, cnt2 + 1);
  else if (mixed)
    batch_render_kernel<BT, true><<<grid, BT, 0, s>>>(D, item_bases, n, n_items, fb, cnt2, cmax,
                                                      cnt2 + 1);
  else
    batch_render_kernel<BT, false><<<grid, BT, 0, s>>>(D, item_bases, n, n_items, fb, cnt2, cmax,
                                                       cnt2 + 1);
}

bool same_frame(const kl_params& a, const kl_params& b) {
  return a.precision == b.precision && a.cull == b.cull && a.width == b.width &&
         a.height == b.height &&
         a.x0 == b.x0 && a.x1 == b.x1 && a.y0 == b.y0 && a.y1 == b.y1 &&
         a.renorm_every == b.renorm_every && a.parabolic_tol == b.parabolic_tol;
}

// Device descriptors for the given buffers (host copy in b->desc).
void fill_desc(kl_batch* b, uint32_t* images, uint64_t* counters, void* ws) {
  char* base = (char*)ws;
  for (uint32_t g = 0; g < b->n; ++g) {
    GroupDesc& d = b->desc[g];
    d.G = make_group(&b->params[g]);
    d.V = make_view(&b->params[g]);
    d.L = b->plans[g];
    d.Wk = b->works[g];
    d.T = carve(b->plans[g], base + b->table_off[g]);
    d.img = images + (size_t)g * b->W * b->H;
    d.cnt = (unsigned long long*)counters + (size_t)g * KL_N_COUNTERS;
    d.ptol = b->params[g].parabolic_tol;
    d.renorm = (int)b->params[g].renorm_every;
    d.pad = 0;
  }
}

int check_buffers(const kl_batch* b, uint32_t* images, uint64_t* counters, void* ws,
                  size_t bytes) {
  if (!b || !images || !counters || !ws) return KL_EINVAL;
  if (((uintptr_t)ws & 255u) != 0) return KL_EINVAL;
  if (bytes < b->total) return KL_ENOSPACE;
  return KL_OK;
}

int upload(kl_batch* b, void* ws, cudaStream_t s) {
  char* base = (char*)ws;
  if (cudaMemcpyAsync(base + b->off_desc, b->desc.data(), b->desc.size() * sizeof(GroupDesc),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return KL_ECUDA;
  if (cudaMemcpyAsync(base + b->off_bases, b->bases.data(), b->bases.size() * sizeof(uint32_t),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return KL_ECUDA;
  return KL_OK;
}

// Zeroing, the two table passes and the render launch.
int enqueue(kl_batch* b, uint32_t* images, uint64_t* counters, void* ws, cudaStream_t s) {
  char* base = (char*)ws;
  const GroupDesc* D = (const GroupDesc*)(base + b->off_desc);
  const uint32_t* bases = (const uint32_t*)(base + b->off_bases);
  unsigned long long* fb = (unsigned long long*)(base + b->off_fb);
  uint32_t* cnt2 = (uint32_t*)(base + b->off_cnt);  // [0] fallback entries, [1] queue
  const size_t img_bytes = (size_t)b->n * b->W * b->H * sizeof(uint32_t);
  if (cudaMemsetAsync(images, 0, img_bytes, s) != cudaSuccess) return KL_ECUDA;
  if (cudaMemsetAsync(counters, 0, (size_t)b->n * KL_N_COUNTERS * sizeof(uint64_t), s) !=
      cudaSuccess)
    return KL_ECUDA;
  if (cudaMemsetAsync(cnt2, 0, 2 * sizeof(uint32_t), s) != cudaSuccess) return KL_ECUDA;
  const uint32_t n = b->n;
  const uint32_t gp = (b->n_parts + 63) / 64;
  batch_parts_kernel<<<gp < 65535u ? gp : 65535u, 64, 0, s>>>(D, bases, n, b->n_parts);
  if (check_launch() != KL_OK) return KL_ECUDA;
  const uint32_t gc = (b->n_comb + 127) / 128;
  batch_combine_kernel<<<gc < 1048576u ? gc : 1048576u, 128, 0, s>>>(
      D, bases + (n + 1), n, b->n_comb, b->mixed, fb, cnt2);
  if (check_launch() != KL_OK) return KL_ECUDA;
  if (b->cull) {
    const uint32_t gd = (b->n_disk + 3) / 4;  // four warps per block
    batch_disk_kernel<<<gd < 65535u ? gd : 65535u, 128, 0, s>>>(D, bases + 3 * (n + 1), n,
                                                                b->n_disk);
    if (check_launch() != KL_OK) return KL_ECUDA;
  }
  const uint32_t* item_bases = bases + 2 * (n + 1);
  const int grid = b->sms * b->occ;
  const bool cull = b->cull != 0;
  switch (b->bt) {
    case 64:
      launch_batch<64>(grid, s, b->mixed, cull, D, item_bases, n, b->n_items, fb, cnt2, b->cmax);
      break;
    case 256:
      launch_batch<256>(grid, s, b->mixed, cull, D, item_bases, n, b->n_items, fb, cnt2,
                        b->cmax);
      break;
    default:
      launch_batch<128>(grid, s, b->mixed, cull, D, item_bases, n, b->n_items, fb, cnt2,
                        b->cmax);
  }
  return check_launch();
}

void drop_graph(kl_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

}  // namespace

extern "C" int kl_batch_create(const kl_params* params, uint32_t n_groups, kl_batch** out) {
  if (!params || !out || n_groups == 0) return KL_EINVAL;
  *out = nullptr;
  const kl_params& p0 = params[0];
  for (uint32_t g = 0; g < n_groups; ++g) {
    if (!valid_view(&params[g]) || !same_frame(p0, params[g])) return KL_EINVAL;
    if (params[g].precision != KL_FP64 && params[g].precision != KL_MIXED) return KL_EINVAL;
    if (params[g].mode != KL_LIMIT_SET || params[g].cull > 1) return KL_EINVAL;
    if (params[g].shard_count > 1) return KL_EINVAL;  // a batch is not sharded
    if (!(params[g].parabolic_tol >= 0.0)) return KL_EINVAL;
    if (params[g].depth < 2) return KL_EINVAL;
  }
  kl_batch* b = new (std::nothrow) kl_batch();
  if (!b) return KL_ERANGE;
  b->n = n_groups;
  b->mixed = p0.precision == KL_MIXED;
  b->cull = p0.cull ? 1 : 0;
  b->bt = p0.block_threads ? (int)p0.block_threads : kDefaultThreads;
  b->W = p0.width;
  b->H = p0.height;
  b->params.assign(params, params + n_groups);
  b->plans.resize(n_groups);
  b->works.resize(n_groups);
  b->table_off.resize(n_groups);
  b->desc.resize(n_groups);
  b->bases.assign(4 * (n_groups + 1), 0u);
  if (device_slots(render_fn(b->bt, b->mixed, b->cull), b->bt, &b->sms, &b->occ) != KL_OK) {
    delete b;
    return KL_ECUDA;
  }
  const uint32_t chunk = p0.chunk_pairs ? p0.chunk_pairs : 64u;
  uint64_t parts = 0, comb = 0, items = 0, fb = 0, disk = 0;
  size_t off = 0;
  b->off_desc = off; off = align256(off + n_groups * sizeof(GroupDesc));
  b->off_bases = off; off = align256(off + b->bases.size() * sizeof(uint32_t));
  for (uint32_t g = 0; g < n_groups; ++g) {
    Plan& L = b->plans[g];
    const int st = make_plan(&params[g], &L, true);
    if (st != KL_OK) {
      delete b;
      return st;
    }
    // culled: warp items of 32 prefixes x one top-level block
    b->works[g] = b->cull    ? make_work(L, 32, L.cnb[L.clev - 1], 1, 1u)
                  : b->mixed ? make_work(L, 32, L.npairs, 1, chunk)
                             : make_work(L, b->bt, L.ns, 1, 2u * chunk);
    b->bases[g] = (uint32_t)parts;
    b->bases[(n_groups + 1) + g] = (uint32_t)comb;
    b->bases[2 * (n_groups + 1) + g] = (uint32_t)items;
    b->bases[3 * (n_groups + 1) + g] = (uint32_t)disk;
    parts += parts_count(L);
    comb += combine_count(L);
    items += b->works[g].n_items;
    if (b->cull) disk += cull_disk_units(L);
    fb += 4ull * L.np;
    const uint32_t cg = (L.ns + kFbChunk - 1) / kFbChunk;
    if (cg > b->cmax) b->cmax = cg;
  }
  if (parts >= (1ull << 32) || comb >= (1ull << 32) || items >= (1ull << 31) ||
      disk >= (1ull << 31) || 3ull * b->cmax * fb >= (1ull << 32)) {
    delete b;
    return KL_ERANGE;
  }
  b->bases[n_groups] = (uint32_t)parts;
  b->bases[(n_groups + 1) + n_groups] = (uint32_t)comb;
  b->bases[2 * (n_groups + 1) + n_groups] = (uint32_t)items;
  b->bases[3 * (n_groups + 1) + n_groups] = (uint32_t)disk;
  b->n_disk = (uint32_t)disk;
  b->n_parts = (uint32_t)parts;
  b->n_comb = (uint32_t)comb;
  b->n_items = (uint32_t)items;
  b->off_fb = off; off = align256(off + fb * sizeof(unsigned long long));
  b->off_cnt = off; off = align256(off + 2 * sizeof(uint32_t));
  for (uint32_t g = 0; g < n_groups; ++g) {
    b->table_off[g] = off;
    off = align256(off + b->plans[g].total);
  }
  b->total = off;
  *out = b;
  return KL_OK;
}

extern "C" size_t kl_batch_workspace_bytes(const kl_batch* b) { return b ? b->total : 0; }

extern "C" int kl_batch_render(kl_batch* b, uint32_t* d_images, uint64_t* d_counters,
                               void* d_workspace, size_t workspace_bytes, void* stream) {
  int st = check_buffers(b, d_images, d_counters, d_workspace, workspace_bytes);
  if (st != KL_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  fill_desc(b, d_images, d_counters, d_workspace);
  st = upload(b, d_workspace, s);
  if (st != KL_OK) return st;
  return enqueue(b, d_images, d_counters, d_workspace, s);
}

extern "C" int kl_batch_capture(kl_batch* b, uint32_t* d_images, uint64_t* d_counters,
                                void* d_workspace, size_t workspace_bytes, void* stream) {
  int st = check_buffers(b, d_images, d_counters, d_workspace, workspace_bytes);
  if (st != KL_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  fill_desc(b, d_images, d_counters, d_workspace);
  st = upload(b, d_workspace, s);
  if (st != KL_OK) return st;
  if (cudaStreamSynchronize(s) != cudaSuccess) return KL_ECUDA;
  drop_graph(b);
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return KL_ECUDA;
  st = enqueue(b, d_images, d_counters, d_workspace, s);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &g);
  if (st != KL_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    return st != KL_OK ? st : KL_ECUDA;
  }
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    b->exec = nullptr;
    return KL_ECUDA;
  }
  b->graph = g;
  return KL_OK;
}

extern "C" int kl_batch_replay(kl_batch* b, void* stream) {
  if (!b || !b->exec) return KL_EINVAL;
  return cudaGraphLaunch(b->exec, (cudaStream_t)stream) == cudaSuccess ? KL_OK : KL_ECUDA;
}

extern "C" void kl_batch_destroy(kl_batch* b) {
  if (!b) return;
  drop_graph(b);
  delete b;
}
