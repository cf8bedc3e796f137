// General presentations: the paper's own enumeration (Sec. "Implementation")
// for any group given by an indexed Cayley table (Sec. "Cayley Multiplication
// Tables").  Every index n of the unpruned m-ary tree of depth d is written as
// d base-m digits plus one (symbols 1..m, w_1 most significant); the string
// is kept when the table run over it, read right to left from state 0, never
// reaches the crash state 0; a kept string is drawn at its word value (the
// seed of w_d, then the maps of w_d, ..., w_1).
//
// GPU layout.  Each warp takes items of 32 x kPerLane consecutive indices;
// lane l scans its own kPerLane indices with an odometer (the digits packed 4
// bits each, the last digit, i.e. the first-applied letter, in the lowest
// nibble), so no index is divided by m more than once per item.  The kept
// strings are sparse (4 3^(d-1) of 4^d for the once-punctured torus), so the
// warp compacts them: each round every lane tests one string, the kept ones
// are appended to a per-warp queue in shared memory (ballot + prefix count),
// and whenever the queue holds 32 words all lanes evaluate one each, with
// every lane busy.  Word values are FP64; the splat is the run-length tally
// of the other renders.
#include "kl_common.cuh"

namespace {

constexpr int kFsaThreads = 256;
constexpr int kFsaWarps = kFsaThreads / 32;
constexpr uint32_t kPerLane = 64;
constexpr int kFsaMaxDepth = 32;

struct FsaDev {
  uint32_t m, d;
  uint8_t table[(KL_FSA_MAX_LETTERS + 1) * (KL_FSA_MAX_LETTERS + 1)];
  double g[KL_FSA_MAX_LETTERS * 8];
  double seed[KL_FSA_MAX_LETTERS * 2];
};

// Packed digits: nibble k holds the symbol of w_{d-k} (k = 0: the first-
// applied letter).  Two words of 16 nibbles cover d <= 32.
struct Digits {
  unsigned long long lo, hi;
};

__device__ __forceinline__ uint32_t nibble(const Digits& s, int k) {
  return (uint32_t)((k < 16 ? s.lo >> (4 * k) : s.hi >> (4 * (k - 16))) & 15ull);
}

// The string of index n (symbols = base-m digits plus one).
__device__ Digits digits_of(unsigned long long n, uint32_t m, uint32_t d) {
  Digits s{0ull, 0ull};
  for (uint32_t k = 0; k < d; ++k) {
    const unsigned long long sym = n % m + 1;
    n /= m;
    if (k < 16) s.lo |= sym << (4 * k);
    else s.hi |= sym << (4 * (k - 16));
  }
  return s;
}

// n + 1: the lowest symbol steps up, symbols past m wrap to 1 and carry.
__device__ __forceinline__ void step(Digits& s, uint32_t m, uint32_t d) {
  for (uint32_t k = 0; k < d; ++k) {
    const uint32_t v = nibble(s, (int)k);
    const unsigned long long one = 1ull << (4 * (k & 15u));
    unsigned long long& w = k < 16 ? s.lo : s.hi;
    if (v < m) {
      w += one;
      return;
    }
    w -= (unsigned long long)(m - 1) * one;  // m -> 1, carry on
  }
}

// Table run right to left from state 0; true if no crash.
__device__ __forceinline__ bool kept(const Digits& s, const uint8_t* tab, uint32_t m,
                                     uint32_t d) {
  uint32_t state = 0;
  for (uint32_t k = 0; k < d; ++k) {
    state = tab[state * (m + 1) + nibble(s, (int)k)];
    if (state == 0) return false;
  }
  return true;
}

// Word value, FP64: z = seed of w_d, then the maps of w_d, ..., w_1.
__device__ __forceinline__ dc fsa_value(const Digits& s, const double* g, const double* seed,
                                        uint32_t d) {
  const uint32_t x0 = nibble(s, 0) - 1;
  dc z = {seed[2 * x0], seed[2 * x0 + 1]};
  for (uint32_t k = 0; k < d; ++k) {
    const double* M = g + 8 * (nibble(s, (int)k) - 1);
    const dc num = {M[0] * z.re - M[1] * z.im + M[2], M[0] * z.im + M[1] * z.re + M[3]};
    const dc den = {M[4] * z.re - M[5] * z.im + M[6], M[4] * z.im + M[5] * z.re + M[7]};
    const double r = rcp64(den.re * den.re + den.im * den.im);
    z = {(num.re * den.re + num.im * den.im) * r, (num.im * den.re - num.re * den.im) * r};
  }
  return z;
}

__global__ void __launch_bounds__(kFsaThreads) fsa_render_kernel(
    FsaDev F, View V, unsigned long long n_idx, unsigned long long n_items,
    unsigned long long* queue, uint32_t* __restrict__ img, unsigned long long* counters) {
  // (the evaluated words of one thread fit uint32: a thread evaluates at most
  // one word per 32 scanned strings of its warp's items)
  __shared__ uint8_t tab[(KL_FSA_MAX_LETTERS + 1) * (KL_FSA_MAX_LETTERS + 1)];
  __shared__ double g[KL_FSA_MAX_LETTERS * 8];
  __shared__ double seed[KL_FSA_MAX_LETTERS * 2];
  __shared__ Digits wq[kFsaWarps][64];
  for (int i = threadIdx.x; i < (int)((F.m + 1) * (F.m + 1)); i += blockDim.x) tab[i] = F.table[i];
  for (int i = threadIdx.x; i < (int)(8 * F.m); i += blockDim.x) g[i] = F.g[i];
  for (int i = threadIdx.x; i < (int)(2 * F.m); i += blockDim.x) seed[i] = F.seed[i];
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  Digits* q = wq[warp];
  uint32_t qlen = 0;
  Tally t;
  uint32_t evaluated = 0;
  auto drain = [&](uint32_t k) {  // evaluate queue entries [0, k) (k <= 32), one per lane
    if (lane < k) {
      const dc z = fsa_value(q[lane], g, seed, F.d);
      t.add(pixel64((z.re - V.x0) * V.sx, (V.y1 - z.im) * V.sy, V), img);
      ++evaluated;
    }
    __syncwarp();
  };
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(queue, 1ull);
    item = __shfl_sync(0xFFFFFFFFu, item, 0);
    if (item >= n_items) break;
    const unsigned long long first = item * 32ull * kPerLane + (unsigned long long)lane * kPerLane;
    Digits s = digits_of(first < n_idx ? first : 0ull, F.m, F.d);
    for (uint32_t r = 0; r < kPerLane; ++r) {
      const bool ok = first + r < n_idx && kept(s, tab, F.m, F.d);
      const unsigned b = __ballot_sync(0xFFFFFFFFu, ok);
      if (ok) q[qlen + __popc(b & lt)] = s;
      qlen += __popc(b);
      __syncwarp();
      if (qlen >= 32) {
        drain(32);
        qlen -= 32;
        if (lane < qlen) q[lane] = q[32 + lane];
        __syncwarp();
      }
      step(s, F.m, F.d);
    }
  }
  drain(qlen);
  t.flush(img);
  publish_counts(t.in_window, evaluated, evaluated, t.atomics, counters);
}

int fsa_check(const kl_fsa* f, uint32_t d, unsigned long long* n_idx) {
  if (!f || f->m < 1 || f->m > KL_FSA_MAX_LETTERS) return KL_EINVAL;
  if (d < 1 || d > (uint32_t)kFsaMaxDepth) return KL_ERANGE;
  const uint32_t m = f->m;
  for (uint32_t i = 0; i < (m + 1) * (m + 1); ++i)
    if (f->table[(i / (m + 1)) * (KL_FSA_MAX_LETTERS + 1) + i % (m + 1)] > m) return KL_EINVAL;
  for (uint32_t k = 0; k < 8 * m; ++k)
    if (!isfinite(f->gens[k])) return KL_EINVAL;
  for (uint32_t k = 0; k < 2 * m; ++k)
    if (!isfinite(f->seeds[k])) return KL_EINVAL;
  unsigned long long n = 1;
  for (uint32_t k = 0; k < d; ++k) {
    if (n > (1ull << 40) / m) return KL_ERANGE;
    n *= m;
  }
  *n_idx = n;
  return KL_OK;
}

}  // namespace

extern "C" int kl_fsa_count(const kl_fsa* f, uint32_t depth, uint64_t* count) {
  unsigned long long n_idx = 0;
  const int st = fsa_check(f, depth, &n_idx);
  if (st != KL_OK) return st;
  if (!count) return KL_EINVAL;
  // ways[s] = strings of the remaining length that run from state s without a
  // crash; one more symbol in front of the run: ways'(s) = sum over symbols
  // of ways(table[s][symbol]) for non-crash targets.
  const uint32_t m = f->m;
  unsigned long long ways[KL_FSA_MAX_LETTERS + 1], next[KL_FSA_MAX_LETTERS + 1];
  for (uint32_t s = 0; s <= m; ++s) ways[s] = 1;
  for (uint32_t k = 0; k < depth; ++k) {
    for (uint32_t s = 0; s <= m; ++s) {
      unsigned long long acc = 0;
      for (uint32_t sym = 1; sym <= m; ++sym) {
        const uint32_t to = f->table[s * (KL_FSA_MAX_LETTERS + 1) + sym];
        if (to != 0) acc += ways[to];
      }
      next[s] = acc;
    }
    for (uint32_t s = 0; s <= m; ++s) ways[s] = next[s];
  }
  *count = ways[0];
  return KL_OK;
}

extern "C" int kl_render_fsa(const kl_fsa* f, const kl_params* p, uint32_t* d_image,
                             uint64_t* d_counters, void* d_workspace, size_t workspace_bytes,
                             void* stream) {
  if (!p || !d_image || !valid_view(p)) return KL_EINVAL;
  if (p->precision != KL_FP64) return KL_EINVAL;
  unsigned long long n_idx = 0;
  int st = fsa_check(f, p->depth, &n_idx);
  if (st != KL_OK) return st;
  if (!d_workspace || ((uintptr_t)d_workspace & 255u) != 0) return KL_EINVAL;
  if (workspace_bytes < KL_FSA_WORKSPACE_BYTES) return KL_ENOSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* cnt = (unsigned long long*)d_counters;
  if (!p->accumulate) {
    if (cudaMemsetAsync(d_image, 0, (size_t)p->width * p->height * sizeof(uint32_t), s) !=
        cudaSuccess)
      return KL_ECUDA;
    if (cnt && cudaMemsetAsync(cnt, 0, KL_N_COUNTERS * sizeof(uint64_t), s) != cudaSuccess)
      return KL_ECUDA;
  }
  FsaDev F;
  F.m = f->m;
  F.d = p->depth;
  for (uint32_t i = 0; i < (F.m + 1) * (F.m + 1); ++i)
    F.table[i] = f->table[(i / (F.m + 1)) * (KL_FSA_MAX_LETTERS + 1) + i % (F.m + 1)];
  for (uint32_t k = 0; k < 8 * F.m; ++k) F.g[k] = f->gens[k];
  for (uint32_t k = 0; k < 2 * F.m; ++k) F.seed[k] = f->seeds[k];
  int sms = 0, occ = 0;
  if (device_slots((const void*)fsa_render_kernel, kFsaThreads, &sms, &occ) != KL_OK)
    return KL_ECUDA;
  const unsigned long long per_item = 32ull * kPerLane;
  const unsigned long long n_items = (n_idx + per_item - 1) / per_item;
  unsigned long long* queue = (unsigned long long*)d_workspace;  // the item queue head
  if (cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s) != cudaSuccess) return KL_ECUDA;
  fsa_render_kernel<<<sms * occ, kFsaThreads, 0, s>>>(F, make_view(p), n_idx, n_items, queue,
                                                      d_image, cnt);
  return check_launch();
}
