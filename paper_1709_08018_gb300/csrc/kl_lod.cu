// Level of detail: training labels for the network and the network-pruned
// render.
//
// Tree levels.  A node at level k is a reduced prefix w_1 .. w_k, numbered by
// its prefix slot (x = w_k, base-3 ranks of w_{k-1} .. w_1, most significant
// first): slot = x 3^(k-1) + r, N_k = 4 3^(k-1) nodes.  The children of
// (x, r) are (y, rank(x | y) 3^(k-1) + r) for the three letters y != inv(x),
// rank(x | y) being the rank of x among the letters other than inv(y).  A
// node's subtree is the set of its 3^(D-k) words of length D.
//
// Labels.  The exact render with prefix length hi also records, per level-hi
// node, the box of all its words (pixel coordinates in 1/256-pixel fixed
// point).  A node is resolved when its image falls under one pixel (box
// width and height below `extent` pixels, 1 by default) or misses the
// window entirely.  label = 0 for a resolved node, else 1 + max(label of its
// children); at level hi, unresolved nodes get 1 ("needs the exact
// enumeration").
//
// Pruned render.  From level lo down, the network predicts each active
// node's label from the 8 features of its prefix matrix (a product of det-1
// generators), on the tensor cores in tiles of 128 nodes.  A
// node predicted resolved (y + margin < 1/2) is pruned when its first, middle
// and last words in index order (the two ends and the middle of its piece of
// the limit set) fall into one pixel, each at least `edge` pixels away from
// that pixel's sides (or all three at least `edge` outside the window): it
// adds its 3^(D-k) words to that pixel (or counts them dropped).  A resolved
// node's words all lie within `extent` of one another, so with edge = extent
// a right prediction never moves a word across a pixel edge; a node too near
// an edge is expanded instead, and its smaller children are tried in turn.
// The others expand to their children; nodes still active at level hi are
// rendered exactly (all their words) by the culling engine of kl_cull.cuh,
// with the image of the per-word mixed render of those nodes.  Every word is
// counted once.
#include "kl_mlp_tc.cuh"

namespace {

constexpr int kLodThreads = 128;

struct LodPlan {
  int D, lo, hi;
  uint32_t p3[kMaxPrefix + 1];       // p3[k] = 3^(k-1): nodes per letter at level k
  uint64_t base[kMaxPrefix + 2];     // first node of level k in the level-concatenated arrays
  uint64_t total;
};

__host__ __device__ __forceinline__ uint32_t level_nodes(const LodPlan& P, int k) {
  return 4u * P.p3[k];
}

// An active node: its prefix matrix p, q, r, s (re, im) as double-floats
// (hi + lo float pairs, about 48 bits: the FP64 pipe, the scarce one on this
// GPU, is left out of the tree levels) and its slot.
struct __align__(16) Active {
  float hi[8], lo[8];
  uint32_t slot;
  uint32_t pad[3];
};

__device__ __forceinline__ M1 m1_load(const Active& a) {
  M1 P;
  D1* e = &P.p.re;
#pragma unroll
  for (int i = 0; i < 8; ++i) e[i] = {a.hi[i], a.lo[i]};
  return P;
}
__device__ __forceinline__ void m1_store(const M1& P, Active& a) {
  const D1* e = &P.p.re;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    a.hi[i] = e[i].hi;
    a.lo[i] = e[i].lo;
  }
}

// Prefix matrix of node `slot` at level k (nk = 3^(k-1)): letters right to left.
__device__ M2 node_matrix(const Group& G, int k, uint32_t slot, uint32_t nk) {
  const int x = (int)(slot / nk);
  const uint32_t r = slot % nk;
  M2 P = load_gen(G, x);
  int right = x;
  uint32_t place = nk / 3u;
  for (int j = 0; j < k - 1; ++j) {
    const int digit = (int)((r / place) % 3u);
    place /= 3u;
    const int w = allowed_letter(digit, (right + 2) & 3);
    P = mmul(load_gen(G, w), P);
    right = w;
  }
  return P;
}

// The 8 features: P / sqrt(det P) (principal root), negated if needed so that
// Re tr > 0 (a zero trace takes the sign of the first nonzero entry), then
// sign(v) log(1 + |v|) for each real part and imaginary part.
__device__ void node_features(const M2& P, float* f) {
  // A node matrix is a product of generators of determinant one, so its own
  // determinant is one up to rounding (relative 1e-15 at these depths) and
  // dividing by its square root would change no feature at FP32 (let alone
  // at the network's BF16): the features are taken from P as it is, and the
  // FP64 pipe, the scarce one on this GPU, is spared that division.
  double lead = P.p.re + P.s.re;
  const double v[8] = {P.p.re, P.p.im, P.q.re, P.q.im, P.r.re, P.r.im, P.s.re, P.s.im};
  for (int i = 0; i < 8 && lead == 0.0; ++i) lead = v[i];
  const bool neg = lead < 0.0;
  for (int i = 0; i < 8; ++i) {
    const float a = neg ? -(float)v[i] : (float)v[i];
    f[i] = copysignf(log1pf(fabsf(a)), a);
  }
}

// The same features from a double-float node matrix: the high parts are the
// FP32 roundings of the entries (what node_features converts), and the sign
// of the trace is taken from its double-float sum.
__device__ void node_features_df(const M1& P, float* f) {
  const D1* e = &P.p.re;
  float lead = d1_add(P.p.re, P.s.re).hi;
  for (int i = 0; i < 8 && lead == 0.0f; ++i) lead = e[i].hi;
  const bool neg = lead < 0.0f;
  for (int i = 0; i < 8; ++i) {
    const float a = neg ? -e[i].hi : e[i].hi;
    f[i] = copysignf(log1pf(fabsf(a)), a);
  }
}

// Resolved: no word inside the window, or the box (1/256-pixel fixed point)
// narrower and lower than `ext` (= 256 extent).
__device__ __forceinline__ bool resolved(int4 b, int W, int H, int ext) {
  if (b.x > b.y) return true;  // no finite word: nothing drawn
  const bool outside = b.y < 0 || b.x >= 256 * W || b.w < 0 || b.z >= 256 * H;
  const bool small = b.y - b.x < ext && b.w - b.z < ext;
  return outside || small;
}

// ---------------------------------------------------------------------------
// labels

// The exact mixed (or FP64) render with per-slot pixel boxes; one persistent
// launch like render_mixed_kernel / render64_kernel.
template <int BT, bool MIXED>
__global__ void __launch_bounds__(BT, 1536 / BT) lod_exact_kernel(
    Tables T, Plan L, View V, Work Wk, BoxRef B, uint32_t* __restrict__ img,
    unsigned long long* counters) {
  const uint32_t chunks = (L.ns + kFbChunk - 1) / kFbChunk;
  const uint32_t fb_units = MIXED ? 3u * chunks * (*T.fbcount) : 0u;
  const uint32_t n64 = (fb_units + BT - 1) / BT;
  const uint32_t total = n64 + Wk.n_items;
  Tally t;
  uint32_t words = 0, fp64_words = 0;
  for (;;) {
    const uint32_t item = next_item(T.fbcount + 1);
    if (item >= total) break;
    if (MIXED && item < n64) {
      const uint32_t unit = item * BT + threadIdx.x;
      if (MIXED && unit < fb_units) {
        const uint32_t e = unit / (3u * chunks), rem = unit % (3u * chunks);
        const uint32_t slot = (uint32_t)(T.fb[e] & 0xFFFFFFFFull);
        const UnitTally r = fallback_unit<true>(T.pre64, T.flags, T.suf64, slot, rem / chunks,
                                                rem % chunks, L.np, L.ns, V, img, B);
        words += r.words;
        fp64_words += r.words;
        t.in_window += r.in_window;
        t.atomics += r.atomics;
      }
      continue;
    }
    const uint32_t it = item - n64;
    if (MIXED) {
      mixed_item<BT, true>(it, Wk, L, V, T, t, words, img, &B);
    } else {
      int x, u;
      uint32_t pb, c;
      item_of(it, Wk, x, u, pb, c);
      const uint32_t r = pb * BT + threadIdx.x;
      if (r < L.np) {
        const uint32_t slot = (uint32_t)x * L.np + r;
        const uint32_t j0 = c * Wk.chunk, j1 = min(L.ns, j0 + Wk.chunk);
        words64<true>(T.pre64[slot], T.flags[slot] & kDirect, T.suf64 + (size_t)u * L.ns, j0,
                      j1, V, t, img, &B, slot);
        words += j1 - j0;
      }
    }
  }
  publish_counts(t.in_window, words, fp64_words, t.atomics, counters);
}

__global__ void box_init_kernel(BoxRef B, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    B.cmin[i] = 0x7FFFFFFF;
    B.rmin[i] = 0x7FFFFFFF;
    B.cmax[i] = -0x7FFFFFFF;
    B.rmax[i] = -0x7FFFFFFF;
  }
}

// Level hi: labels from the boxes.
__global__ void leaf_labels_kernel(BoxRef B, uint32_t n, int W, int H, int ext, int4* box,
                                   uint8_t* label) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int4 b = make_int4(B.cmin[i], B.cmax[i], B.rmin[i], B.rmax[i]);
    box[i] = b;
    label[i] = resolved(b, W, H, ext) ? 0 : 1;
  }
}

// Level k < hi: union of the children's boxes, label from the children's.
__global__ void reduce_labels_kernel(uint32_t nk, const int4* __restrict__ cbox,
                                     const uint8_t* __restrict__ clabel, int W, int H, int ext,
                                     int4* box, uint8_t* label) {
  for (uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x; slot < 4u * nk;
       slot += gridDim.x * blockDim.x) {
    const int x = (int)(slot / nk);
    const uint32_t r = slot % nk;
    int4 b = make_int4(0x7FFFFFFF, -0x7FFFFFFF, 0x7FFFFFFF, -0x7FFFFFFF);
    int worst = 0;
    for (int k = 0; k < 3; ++k) {
      const int y = allowed_letter(k, (x + 2) & 3);
      const int rk = x - (x > ((y + 2) & 3) ? 1 : 0);
      const uint32_t child = (uint32_t)y * 3u * nk + (uint32_t)rk * nk + r;
      const int4 c = cbox[child];
      if (c.x <= c.y) {
        b.x = min(b.x, c.x); b.y = max(b.y, c.y); b.z = min(b.z, c.z); b.w = max(b.w, c.w);
      }
      worst = max(worst, (int)clabel[child]);
    }
    box[slot] = b;
    label[slot] = resolved(b, W, H, ext) ? 0 : (uint8_t)min(255, 1 + worst);
  }
}

// Features of the level-k nodes.  As for the render's prefixes, each node
// matrix is one product P = H L of a tail (the q innermost letters) and a head
// (the other k - q) from two small tables built first by part_entry, instead
// of k - 1 products per node.
__global__ void feature_parts_kernel(Group G, Plan Lk, int renorm, Tables T) {
  const uint32_t n = 4u * Lk.p3_q1 + (Lk.p > Lk.q ? 4u * Lk.p3_pq : 0u);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    part_entry(G, Lk, renorm, i, T);
}

__global__ void features_kernel(Plan Lk, Tables T, float* __restrict__ out) {
  const uint32_t n = 4u * Lk.np;
  for (uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x; slot < n;
       slot += gridDim.x * blockDim.x) {
    const uint32_t x = slot / Lk.np, r = slot % Lk.np;
    const PartM& TL = T.Lt[x * Lk.p3_q1 + r / Lk.p3_pq];
    const M2 P =
        Lk.p > Lk.q ? mmul(T.Ht[(uint32_t)TL.edge * Lk.p3_pq + r % Lk.p3_pq], TL.m) : TL.m;
    float f[8];
    node_features(P, f);
    for (int j = 0; j < 8; ++j) out[(size_t)slot * 8 + j] = f[j];
  }
}

// ---------------------------------------------------------------------------
// pruned render

// vstar[(e * 4 + x) * (hi + 1) + k]: the suffix point of the first (e = 0),
// middle (e = 1) and last (e = 2) word, in index order, of the subtree of any
// level-k node ending in letter x: the suffix of D - k letters that takes the
// allowed letter of rank e at every step.
constexpr int kReps = 3;
constexpr int kNearEdge = -2;

// Pixel id of pixel coordinates (u, v) if the point lies at least `edge`
// inside that pixel; -1 if it lies at least `edge` outside the window (or is
// not finite); kNearEdge otherwise.
// Coordinates u, v are double-floats; u = cu + ru with cu an integer (exact
// as a float near the window) and ru in [0, 1) from the exact fraction of
// u.hi plus u.lo.
__device__ __forceinline__ void split_unit(D1 u, float& c, float& r) {
  c = floorf(u.hi);
  r = __fadd_rn(__fsub_rn(u.hi, c), u.lo);
  if (r < 0.0f) {
    r = __fadd_rn(r, 1.0f);
    c -= 1.0f;
  } else if (r >= 1.0f) {
    r = __fsub_rn(r, 1.0f);
    c += 1.0f;
  }
}
__device__ __forceinline__ int guarded_pixel_df(D1 u, D1 v, const View& V, float edge) {
  const float W = (float)V.W, H = (float)V.H;
  // far outside (or not finite): no finer test needed
  if (!(u.hi > -2.0f - edge && u.hi < W + 2.0f + edge && v.hi > -2.0f - edge &&
        v.hi < H + 2.0f + edge))
    return -1;
  float cu, ru, cv, rv;
  split_unit(u, cu, ru);
  split_unit(v, cv, rv);
  // at least `edge` outside the window
  const bool out_u = cu <= -2.0f || (cu == -1.0f && ru < 1.0f - edge) || cu >= W + 1.0f ||
                     (cu == W && ru >= edge);
  const bool out_v = cv <= -2.0f || (cv == -1.0f && rv < 1.0f - edge) || cv >= H + 1.0f ||
                     (cv == H && rv >= edge);
  if (out_u || out_v) return -1;
  if (cu < 0.0f || cv < 0.0f || cu >= W || cv >= H) return kNearEdge;
  if (ru < edge || 1.0f - ru <= edge || rv < edge || 1.0f - rv <= edge) return kNearEdge;
  return (int)cv * (int)V.W + (int)cu;
}

__global__ void vstar_kernel(Group G, int D, int lo, int hi, double2* vstar) {
  const int x = threadIdx.x & 3, e = (threadIdx.x >> 2) % kReps;
  const int k = lo + (threadIdx.x >> 2) / kReps;
  if (k > hi) return;
  const int m = D - k;
  int w[KL_MAX_DEPTH];
  int prev = x;
  for (int j = 0; j < m; ++j) {
    w[j] = allowed_letter(e, (prev + 2) & 3);
    prev = w[j];
  }
  dc z = {G.seed[2 * w[m - 1]], G.seed[2 * w[m - 1] + 1]};
  for (int j = m - 1; j >= 0; --j) z = mobius(load_gen(G, w[j]), z);
  vstar[(e * 4 + x) * (hi + 1) + k] = make_double2(z.re, z.im);
}

__global__ void init_active_kernel(Group G, int k, uint32_t nk, Active* out, uint32_t* count) {
  const uint32_t n = 4u * nk;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    Active a;
    m1_store(m1_of(node_matrix(G, k, s, nk)), a);
    a.slot = s;
    a.pad[0] = a.pad[1] = a.pad[2] = 0;
    out[s] = a;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = n;
}

// One level: each CTA takes tiles of 128 active nodes (thread t: node t of
// the tile), scores them with the network on the tensor cores (the tcgen05
// forward pass of kl_mlp_tc.cuh) or takes their true labels, then prunes,
// expands or defers each node.  stats: [0] nodes visited, [1] pruned, [2]
// deferred to the exact render.  If a tensor-core wait runs out, the CTA's
// later scores are NaN, which prunes nothing: those nodes are still drawn
// exactly.
static_assert(kLodThreads == kTile, "one tile row per thread");
__global__ void __launch_bounds__(kLodThreads) expand_kernel(
    const float* __restrict__ mlp, const uint8_t* __restrict__ labels, Group G, View V, int D,
    int k, int hi, uint32_t nk,
    float margin, double edge, const double2* __restrict__ vstar, const Active* __restrict__ in,
    const uint32_t* __restrict__ in_count, Active* __restrict__ out, uint32_t* out_count,
    uint32_t* __restrict__ deferred, uint32_t* deferred_count, uint32_t* __restrict__ img,
    unsigned long long* counters, unsigned long long* stats) {
  extern __shared__ __align__(1024) unsigned char sm[];  // kFwdSmem bytes when mlp
  // the generators, this level's representative suffix points and the view
  // as double-floats (split once per block)
  __shared__ M1 gen[4];
  __shared__ C1 reps[kReps * 4];
  __shared__ D1 vx0, vy1, vsx, vsy;
  Fwd F{};
  if (mlp) F = fwd_begin(sm, mlp);  // uniform: mlp is the same for every thread
  if (threadIdx.x < 4) gen[threadIdx.x] = m1_of(load_gen(G, (int)threadIdx.x));
  if (threadIdx.x < kReps * 4) {
    const double2 v = vstar[threadIdx.x * (hi + 1) + k];
    reps[threadIdx.x] = {d1_of(v.x), d1_of(v.y)};
  }
  if (threadIdx.x == 0) {
    vx0 = d1_neg(d1_of(V.x0));
    vy1 = d1_of(V.y1);
    vsx = d1_of(V.sx);
    vsy = d1_of(V.sy);
  }
  __syncthreads();
  const float edge_f = (float)edge;
  const int lane = threadIdx.x & 31;
  const uint32_t n = *in_count;
  unsigned long long words_sub = 1;
  for (int j = k; j < D; ++j) words_sub *= 3ull;
  unsigned long long visited = 0, pruned = 0, defer = 0, inw = 0, drop = 0;
  // the tile loop is uniform over the CTA (the forward pass synchronises it)
  for (uint64_t tile = blockIdx.x; tile * kLodThreads < n; tile += gridDim.x) {
    const uint64_t e = tile * kLodThreads + threadIdx.x;
    const bool valid = e < n;
    Active a;
    if (valid) a = in[e];
    float y;
    if (mlp) {
      float f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (valid) node_features_df(m1_load(a), f);
      y = fwd_tile(F, f);
    } else {
      y = valid ? (float)labels[a.slot] : 0.0f;  // the level's true labels
    }
    int action = 0;  // 1: expand to the three children, 2: defer to the exact render
    if (valid) {
      ++visited;
      const M1 P = m1_load(a);
      const int x = (int)(a.slot / nk);
      // prune when the score says resolved and the subtree's first, middle and
      // last words agree on one pixel (or all miss the window); the words'
      // values in double-float arithmetic
      bool prune = y + margin < 0.5f;
      int pix = -1;
      if (prune) {
        for (int e = 0; e < kReps; ++e) {
          const C1 z = m1_apply(P, reps[e * 4 + x]);
          const D1 u = d1_mul(d1_add(z.re, vx0), vsx);
          const D1 v = d1_mul(d1_add(vy1, d1_neg(z.im)), vsy);
          const int pe = guarded_pixel_df(u, v, V, edge_f);
          if (e == 0) pix = pe;
          if (pe == kNearEdge || pe != pix) prune = false;
        }
      }
      if (prune) {
        ++pruned;
        if (pix >= 0) {
          atomicAdd(img + pix, (uint32_t)words_sub);  // counts wrap modulo 2^32
          inw += words_sub;
        } else {
          drop += words_sub;
        }
      } else if (k < hi) {
        action = 1;
      } else {
        ++defer;
        action = 2;
      }
    }
    // output slots, one atomic per warp and list (all lanes take part: the
    // tile loop is uniform over the CTA)
    const unsigned be = __ballot_sync(0xFFFFFFFFu, action == 1);
    const unsigned bd = __ballot_sync(0xFFFFFFFFu, action == 2);
    uint32_t base_e = 0, base_d = 0;
    if (lane == 0) {
      if (be) base_e = atomicAdd(out_count, 3u * (uint32_t)__popc(be));
      if (bd) base_d = atomicAdd(deferred_count, (uint32_t)__popc(bd));
    }
    base_e = __shfl_sync(0xFFFFFFFFu, base_e, 0);
    base_d = __shfl_sync(0xFFFFFFFFu, base_d, 0);
    const unsigned lt = (1u << lane) - 1u;
    if (action == 1) {
      const M1 P = m1_load(a);
      const int x = (int)(a.slot / nk);
      const uint32_t base = base_e + 3u * (uint32_t)__popc(be & lt);
      const uint32_t r = a.slot % nk;
      for (int q = 0; q < 3; ++q) {
        const int yl = allowed_letter(q, (x + 2) & 3);
        const int rk = x - (x > ((yl + 2) & 3) ? 1 : 0);
        Active b;
        m1_store(m1_mul(P, gen[yl]), b);
        b.slot = (uint32_t)yl * 3u * nk + (uint32_t)rk * nk + r;
        b.pad[0] = b.pad[1] = b.pad[2] = 0;
        out[base + q] = b;
      }
    } else if (action == 2) {
      deferred[base_d + (uint32_t)__popc(bd & lt)] = a.slot;
    }
    __syncwarp();
  }
  for (int o = 16; o > 0; o >>= 1) {
    visited += __shfl_down_sync(0xFFFFFFFFu, visited, o);
    pruned += __shfl_down_sync(0xFFFFFFFFu, pruned, o);
    defer += __shfl_down_sync(0xFFFFFFFFu, defer, o);
    inw += __shfl_down_sync(0xFFFFFFFFu, inw, o);
    drop += __shfl_down_sync(0xFFFFFFFFu, drop, o);
  }
  if (lane == 0) {
    if (visited) atomicAdd(stats + 0, visited);
    if (pruned) atomicAdd(stats + 1, pruned);
    if (defer) atomicAdd(stats + 2, defer);
    if (inw) atomicAdd(counters + KL_CNT_IN_WINDOW, inw);
    if (drop) atomicAdd(counters + KL_CNT_DROPPED, drop);
  }
  if (mlp) fwd_end(F);
}

// Culled exact render of the deferred level-hi nodes (the culling of
// kl_params.cull, kl_cull.cuh): the same image as the per-word render of
// those nodes on this split, with whole blocks of a node's words placed at
// once where certified.
// lod_disk_kernel first bounds the suffix blocks (warps [0, ndisks)) and
// computes the operator norms of the listed nodes' prefixes (the other
// threads, striding over the list).
__global__ void __launch_bounds__(128) lod_disk_kernel(Plan L, Tables T,
                                                       const uint32_t* __restrict__ slots,
                                                       const uint32_t* n_slots) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t small = cull_small_disks(L), ws = (small + 31) / 32;
  const uint32_t nd = ws + (L.ndisks - small);  // disk warps (cull_disk_unit)
  if (warp < nd) {
    cull_disk_unit(L, T, warp, lane);
    return;
  }
  const uint32_t n = *n_slots;
  const uint32_t stride = gridDim.x * blockDim.x - 32u * nd;
  for (uint32_t e = (warp - nd) * 32u + lane; e < n; e += stride) cull_norm(T, slots[e]);
}

// Items: (block of 32 listed nodes, one of the three compatible suffix
// letters, one top-level block); each lane's letter follows its node's last
// letter.
template <int BT, bool MIXED>
__global__ void __launch_bounds__(BT, 1024 / BT) lod_cull_kernel(
    Tables T, Plan L, View V, const uint32_t* __restrict__ deferred,
    const uint32_t* deferred_count, uint32_t* __restrict__ img, unsigned long long* counters) {
  __shared__ unsigned long long s_stack[BT / 32][kCullStack];
  __shared__ unsigned long long s_leaf[BT / 32][kLeafQueue];
  __shared__ CullLevels C;
  if (threadIdx.x < (unsigned)kMaxCullLevels) {
    C.sz[threadIdx.x] = L.csz[threadIdx.x];
    C.nb[threadIdx.x] = L.cnb[threadIdx.x];
    C.disk[threadIdx.x] = L.cdisk[threadIdx.x];
  }
  __syncthreads();
  CullWarp<MIXED> w(s_stack[threadIdx.x >> 5], s_leaf[threadIdx.x >> 5], &C);
  const uint32_t n = *deferred_count, nbt = L.cnb[L.clev - 1];
  const uint32_t n_items = ((n + 31) / 32) * 3u * nbt;
  for (;;) {
    const uint32_t item = next_item_warp(T.fbcount + 1);
    if (item >= n_items) break;
    const uint32_t bt = item % nbt, rest = item / nbt;
    const uint32_t kq = rest % 3u, e = (rest / 3u) * 32u + w.lane;
    const bool live = e < n;
    const uint32_t slot = live ? deferred[e] : 0u;
    const int u = allowed_letter((int)kq, ((int)(slot / L.np) + 2) & 3);
    const bool f64 = !MIXED || (live && (T.flags[slot] & kFallback));
    w.item(L, V, T, img, live, slot, (uint32_t)u, f64, bt, bt + 1);
  }
  w.finish(L, V, T, img);
  w.t.flush(img);
  publish_counts(w.t.in_window, w.words, w.fp64_words, w.t.atomics, counters);
}

// ---------------------------------------------------------------------------
// host side

int lod_plan(const kl_params* p, uint32_t lo, uint32_t hi, LodPlan* P, Plan* L) {
  if (!p || !valid_view(p)) return KL_EINVAL;
  if (p->precision != KL_FP64 && p->precision != KL_MIXED) return KL_EINVAL;
  if (p->mode != KL_LIMIT_SET || p->cull != 0 || p->shard_count > 1) return KL_EINVAL;
  const int D = (int)p->depth;
  if (lo < 1 || lo > hi || (int)hi >= D || hi > (uint32_t)kMaxPrefix ||
      D - (int)hi > kMaxPlainSuffix)
    return KL_ERANGE;
  kl_params q = *p;
  q.prefix_len = hi;
  const int st = make_plan(&q, L, false);
  if (st != KL_OK) return st;
  P->D = D;
  P->lo = (int)lo;
  P->hi = (int)hi;
  for (int k = 0; k <= kMaxPrefix; ++k) P->p3[k] = k >= 1 ? pow3u(k - 1) : 0;
  uint64_t acc = 0;
  for (int k = 0; k <= kMaxPrefix + 1; ++k) P->base[k] = 0;
  for (int k = (int)lo; k <= (int)hi; ++k) {
    P->base[k] = acc;
    acc += 4ull * P->p3[k];
  }
  P->base[hi + 1] = acc;
  P->total = acc;
  return KL_OK;
}

// The pruned render's plan: the same split, with the culling disks and the
// prefix norms that its exact render of the deferred nodes uses.
int lod_render_plan(const kl_params* p, uint32_t lo, uint32_t hi, LodPlan* P, Plan* L) {
  const int st = lod_plan(p, lo, hi, P, L);
  if (st != KL_OK) return st;
  kl_params q = *p;
  q.prefix_len = hi;
  q.cull = 1;
  return make_plan(&q, L, false);
}

// Workspace of kl_lod_labels: render tables | boxes of level hi | per-level int4 boxes
struct LabelLayout {
  size_t tables, box4, lvl_box, total;
};

LabelLayout label_layout(const LodPlan& P, const Plan& L) {
  LabelLayout Y;
  size_t off = 0;
  Y.tables = off; off = align256(off + L.total);
  Y.box4 = off; off = align256(off + 4ull * level_nodes(P, P.hi) * sizeof(int));
  Y.lvl_box = off; off = align256(off + P.total * sizeof(int4));
  Y.total = off;
  return Y;
}

// Workspace of kl_render_lod: render tables | vstar | two active lists | deferred | counts | stats
struct RenderLayout {
  size_t tables, vstar, act0, act1, deferred, counts, total;
};

RenderLayout render_layout(const LodPlan& P, const Plan& L) {
  RenderLayout Y;
  size_t off = 0;
  const size_t cap = level_nodes(P, P.hi);
  Y.tables = off; off = align256(off + L.total);
  Y.vstar = off; off = align256(off + 4ull * kReps * (P.hi + 1) * sizeof(double2));
  Y.act0 = off; off = align256(off + cap * sizeof(Active));
  Y.act1 = off; off = align256(off + cap * sizeof(Active));
  Y.deferred = off; off = align256(off + cap * sizeof(uint32_t));
  Y.counts = off; off = align256(off + 64 * sizeof(uint32_t));
  Y.total = off;
  return Y;
}

int build_tables_forced(const kl_params* p, const Plan& L, const View& V, const Group& G,
                        const Tables& T, cudaStream_t st, const uint32_t* slots,
                        const uint32_t* n_slots);

unsigned grid_for(uint64_t n, int threads, int cap_per_sm) {
  const int sms = sm_count();
  const uint64_t b = (n + threads - 1) / threads;
  const uint64_t cap = (uint64_t)(sms > 0 ? sms : 1) * cap_per_sm;
  return (unsigned)(b < 1 ? 1 : (b < cap ? b : cap));
}

__global__ void lod_parts_kernel(Group G, Plan L, int renorm, Tables T) {
  const uint32_t total = parts_count(L);
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += gridDim.x * blockDim.x)
    part_entry(G, L, renorm, idx, T);
}

__global__ void lod_combine_kernel(View V, Plan L, double ptol, int mixed, Tables T) {
  const uint32_t total = combine_count(L);
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += gridDim.x * blockDim.x)
    combine_entry(V, L, ptol, mixed, idx, T, 0u, T.fb, T.fbcount);
}

// The pruned render needs the prefix constants of the deferred level-hi
// nodes only: the entries of the `n` slots listed in `slots`, then every
// suffix point.
__global__ void lod_combine_listed_kernel(View V, Plan L, double ptol, int mixed, Tables T,
                                          const uint32_t* __restrict__ slots,
                                          const uint32_t* __restrict__ n_slots) {
  const uint32_t n = *n_slots, total = n + 4u * L.ns;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += gridDim.x * blockDim.x) {
    const uint32_t idx = e < n ? slots[e] : 4u * L.np + (e - n);
    combine_entry(V, L, ptol, mixed, idx, T, 0u, T.fb, T.fbcount);
  }
}

// Tables of *p for the split (prefix hi, suffix D - hi): every prefix slot,
// or, with `slots`, only the listed ones.
int build_tables_forced(const kl_params* p, const Plan& L, const View& V, const Group& G,
                        const Tables& T, cudaStream_t st, const uint32_t* slots,
                        const uint32_t* n_slots) {
  if (cudaMemsetAsync(T.fbcount, 0, 2 * sizeof(uint32_t), st) != cudaSuccess) return KL_ECUDA;
  const uint32_t nParts = parts_count(L);
  lod_parts_kernel<<<(nParts + 31) / 32, 32, 0, st>>>(G, L, (int)p->renorm_every, T);
  if (check_launch() != KL_OK) return KL_ECUDA;
  if (slots) {
    lod_combine_listed_kernel<<<grid_for(combine_count(L), 128, 8), 128, 0, st>>>(
        V, L, p->parabolic_tol, p->precision == KL_MIXED, T, slots, n_slots);
    return check_launch();
  }
  const uint32_t n = combine_count(L);
  lod_combine_kernel<<<(n + 127) / 128, 128, 0, st>>>(V, L, p->parabolic_tol,
                                                       p->precision == KL_MIXED, T);
  return check_launch();
}

}  // namespace

extern "C" uint64_t kl_lod_node_count(uint32_t lo, uint32_t hi) {
  if (lo < 1 || lo > hi || hi > (uint32_t)kMaxPrefix) return 0;
  uint64_t n = 0;
  for (uint32_t k = lo; k <= hi; ++k) n += 4ull * pow3u((int)k - 1);
  return n;
}

extern "C" size_t kl_lod_label_bytes(const kl_params* p, uint32_t lo, uint32_t hi) {
  LodPlan P;
  Plan L;
  if (lod_plan(p, lo, hi, &P, &L) != KL_OK) return 0;
  return label_layout(P, L).total;
}

extern "C" int kl_lod_labels(const kl_params* p, uint32_t lo, uint32_t hi, float extent,
                             uint32_t* d_image, uint64_t* d_counters, float* d_features,
                             uint8_t* d_labels, void* d_workspace, size_t workspace_bytes,
                             void* stream) {
  if (!(extent > 0.0f && extent <= 65536.0f)) return KL_EINVAL;
  const int ext = (int)ceilf(256.0f * extent);
  LodPlan P;
  Plan L;
  int st = lod_plan(p, lo, hi, &P, &L);
  if (st != KL_OK) return st;
  if (!d_image || !d_counters || !d_features || !d_labels || !d_workspace) return KL_EINVAL;
  if (((uintptr_t)d_workspace & 255u) != 0) return KL_EINVAL;
  const LabelLayout Y = label_layout(P, L);
  if (workspace_bytes < Y.total) return KL_ENOSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)d_workspace;
  const View V = make_view(p);
  const Group G = make_group(p);
  kl_params q = *p;
  q.prefix_len = hi;
  const Tables T = carve(L, ws + Y.tables);
  const uint32_t nh = level_nodes(P, (int)hi);
  int* b4 = (int*)(ws + Y.box4);
  const BoxRef B = {b4, b4 + nh, b4 + 2 * nh, b4 + 3 * nh};
  int4* lvl_box = (int4*)(ws + Y.lvl_box);
  unsigned long long* cnt = (unsigned long long*)d_counters;
  if (cudaMemsetAsync(d_image, 0, (size_t)p->width * p->height * sizeof(uint32_t), s) !=
          cudaSuccess ||
      cudaMemsetAsync(cnt, 0, KL_N_COUNTERS * sizeof(uint64_t), s) != cudaSuccess)
    return KL_ECUDA;
  box_init_kernel<<<grid_for(nh, 256, 8), 256, 0, s>>>(B, nh);
  if (check_launch() != KL_OK) return KL_ECUDA;
  st = build_tables_forced(&q, L, V, G, T, s, nullptr, nullptr);
  if (st != KL_OK) return st;
  int sms = 0, occ = 0;
  const bool mixed = p->precision == KL_MIXED;
  const void* fn = mixed ? (const void*)lod_exact_kernel<128, true>
                         : (const void*)lod_exact_kernel<128, false>;
  if (device_slots(fn, 128, &sms, &occ) != KL_OK) return KL_ECUDA;
  const Work Wk = make_work(L, 128, mixed ? L.npairs : L.ns, sms * occ, 0);
  if (mixed)
    lod_exact_kernel<128, true><<<sms * occ, 128, 0, s>>>(T, L, V, Wk, B, d_image, cnt);
  else
    lod_exact_kernel<128, false><<<sms * occ, 128, 0, s>>>(T, L, V, Wk, B, d_image, cnt);
  if (check_launch() != KL_OK) return KL_ECUDA;
  const int W = (int)p->width, H = (int)p->height;
  leaf_labels_kernel<<<grid_for(nh, 256, 8), 256, 0, s>>>(B, nh, W, H, ext,
                                                          lvl_box + P.base[hi],
                                                          d_labels + P.base[hi]);
  if (check_launch() != KL_OK) return KL_ECUDA;
  for (int k = (int)hi - 1; k >= (int)lo; --k) {
    const uint32_t nk = P.p3[k];
    reduce_labels_kernel<<<grid_for(4ull * nk, 256, 8), 256, 0, s>>>(
        nk, lvl_box + P.base[k + 1], d_labels + P.base[k + 1], W, H, ext,
        lvl_box + P.base[k], d_labels + P.base[k]);
    if (check_launch() != KL_OK) return KL_ECUDA;
  }
  // the render tables are no longer needed: their tail and head arrays hold
  // each level's (smaller) feature tables in turn
  for (int k = (int)lo; k <= (int)hi; ++k) {
    Plan Lk = L;
    Lk.p = k;
    Lk.q = (k + 1) / 2;
    Lk.np = pow3u(k - 1);
    Lk.p3_q1 = pow3u(Lk.q - 1);
    Lk.p3_pq = pow3u(k - Lk.q);
    const uint32_t nparts = 4u * Lk.p3_q1 + (k > Lk.q ? 4u * Lk.p3_pq : 0u);
    feature_parts_kernel<<<(nparts + 63) / 64, 64, 0, s>>>(G, Lk, (int)p->renorm_every, T);
    if (check_launch() != KL_OK) return KL_ECUDA;
    features_kernel<<<grid_for(4ull * Lk.np, 128, 16), 128, 0, s>>>(Lk, T,
                                                                    d_features + P.base[k] * 8);
    if (check_launch() != KL_OK) return KL_ECUDA;
  }
  return KL_OK;
}

extern "C" size_t kl_lod_render_bytes(const kl_params* p, uint32_t lo, uint32_t hi) {
  LodPlan P;
  Plan L;
  if (lod_render_plan(p, lo, hi, &P, &L) != KL_OK) return 0;
  return render_layout(P, L).total;
}

namespace {

int render_lod_impl(const kl_params* p, uint32_t lo, uint32_t hi, const float* d_mlp,
                    const uint8_t* d_labels, float margin, float edge, uint32_t* d_image,
                    uint64_t* d_counters, uint64_t* d_stats, void* d_workspace,
                    size_t workspace_bytes, void* stream) {
  LodPlan P;
  Plan L;
  int st = lod_render_plan(p, lo, hi, &P, &L);
  if (st != KL_OK) return st;
  if (p->precision != KL_MIXED) return KL_EINVAL;
  if (!(edge >= 0.0f && edge < 0.5f)) return KL_EINVAL;
  if ((!d_mlp && !d_labels) || !d_image || !d_counters || !d_stats || !d_workspace)
    return KL_EINVAL;
  if (((uintptr_t)d_workspace & 255u) != 0) return KL_EINVAL;
  const RenderLayout Y = render_layout(P, L);
  if (workspace_bytes < Y.total) return KL_ENOSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)d_workspace;
  const View V = make_view(p);
  const Group G = make_group(p);
  kl_params q = *p;
  q.prefix_len = hi;
  const Tables T = carve(L, ws + Y.tables);
  double2* vstar = (double2*)(ws + Y.vstar);
  Active* act[2] = {(Active*)(ws + Y.act0), (Active*)(ws + Y.act1)};
  uint32_t* deferred = (uint32_t*)(ws + Y.deferred);
  uint32_t* counts = (uint32_t*)(ws + Y.counts);  // [k]: active count of level k, [32]: deferred
  unsigned long long* cnt = (unsigned long long*)d_counters;
  unsigned long long* stats = (unsigned long long*)d_stats;
  if (cudaMemsetAsync(d_image, 0, (size_t)p->width * p->height * sizeof(uint32_t), s) !=
          cudaSuccess ||
      cudaMemsetAsync(cnt, 0, KL_N_COUNTERS * sizeof(uint64_t), s) != cudaSuccess ||
      cudaMemsetAsync(stats, 0, 4 * sizeof(uint64_t), s) != cudaSuccess ||
      cudaMemsetAsync(counts, 0, 64 * sizeof(uint32_t), s) != cudaSuccess)
    return KL_ECUDA;
  vstar_kernel<<<1, 4 * kReps * (kMaxPrefix + 1), 0, s>>>(G, P.D, P.lo, P.hi, vstar);
  if (check_launch() != KL_OK) return KL_ECUDA;
  init_active_kernel<<<grid_for(4ull * P.p3[lo], 128, 8), 128, 0, s>>>(G, (int)lo, P.p3[lo],
                                                                        act[0], counts + lo);
  if (check_launch() != KL_OK) return KL_ECUDA;
  if (d_mlp && cudaFuncSetAttribute(expand_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kFwdSmem) != cudaSuccess)
    return KL_ECUDA;
  for (int k = (int)lo; k <= (int)hi; ++k) {
    const int cur = (k - (int)lo) & 1;
    expand_kernel<<<grid_for(4ull * P.p3[k], kLodThreads, 4), kLodThreads,
                    d_mlp ? kFwdSmem : 0u, s>>>(
        d_mlp, d_labels ? d_labels + P.base[k] : nullptr, G, V, P.D, k, (int)hi, P.p3[k],
        d_mlp ? margin : 0.0f, (double)edge, vstar, act[cur], counts + k, act[cur ^ 1],
        counts + k + 1, deferred, counts + 32, d_image, cnt, stats);
    if (check_launch() != KL_OK) return KL_ECUDA;
  }
  st = build_tables_forced(&q, L, V, G, T, s, deferred, counts + 32);
  if (st != KL_OK) return st;
  int sms = 0, occ = 0;
  if (device_slots((const void*)lod_cull_kernel<128, true>, 128, &sms, &occ) != KL_OK)
    return KL_ECUDA;
  // block disks (four warps per block), then the deferred prefixes' norms
  const uint32_t small = cull_small_disks(L);
  const uint32_t disk_warps = (small + 31) / 32 + (L.ndisks - small);
  lod_disk_kernel<<<(disk_warps + 3) / 4 + 2u * (uint32_t)sms, 128, 0, s>>>(L, T, deferred,
                                                                              counts + 32);
  if (check_launch() != KL_OK) return KL_ECUDA;
  lod_cull_kernel<128, true><<<sms * occ, 128, 0, s>>>(T, L, V, deferred, counts + 32, d_image,
                                                       cnt);
  return check_launch();
}

}  // namespace

extern "C" int kl_render_lod(const kl_params* p, uint32_t lo, uint32_t hi, const float* d_mlp,
                             float margin, float edge, uint32_t* d_image, uint64_t* d_counters,
                             uint64_t* d_stats, void* d_workspace, size_t workspace_bytes,
                             void* stream) {
  if (!d_mlp) return KL_EINVAL;
  return render_lod_impl(p, lo, hi, d_mlp, nullptr, margin, edge, d_image, d_counters, d_stats,
                         d_workspace, workspace_bytes, stream);
}

extern "C" int kl_render_lod_labels(const kl_params* p, uint32_t lo, uint32_t hi,
                                    const uint8_t* d_labels, float edge, uint32_t* d_image,
                                    uint64_t* d_counters, uint64_t* d_stats, void* d_workspace,
                                    size_t workspace_bytes, void* stream) {
  if (!d_labels) return KL_EINVAL;
  return render_lod_impl(p, lo, hi, nullptr, d_labels, 0.0f, edge, d_image, d_counters,
                         d_stats, d_workspace, workspace_bytes, stream);
}
