// The level-of-detail network: an MLP 8 -> 64 -> 64 -> 1 with ReLU, BF16
// weights and activations on the fifth-generation tensor cores (tcgen05,
// FP32 accumulators in tensor memory), and its training kernels (forward and
// backward with the weight gradients in one kernel, a fixed-order reduction,
// Adam).
//
// Parameter vector (FP32 master copy, KL_MLP_NPARAMS floats):
//   W1 [8][64] | b1 [64] | W2 [64][64] | b2 [64] | w3 [64] | b3
// (W[in][out]: h_out = sum_in x_in W[in][out] + b_out).  Loss: mean squared
// error over the batch.
//
// A CTA of 128 threads takes tiles of 128 rows; thread t owns row t of the
// tile, which is lane t of every accumulator in tensor memory (M = 128), so
// bias, ReLU, the last layer's dot product and the error are row-local.  The
// layer products run as tcgen05 MMAs on BF16 tiles in shared memory:
//   H1 = X W1 (K = 16: 8 inputs and zero padding), H2 = H1 W2, dH1 = dH2 W2^T.
// The gradients are sums over rows, i.e. products with the rows as the K
// dimension, accumulated in tensor memory over all the CTA's tiles:
//   [H1^T; H2^T] [dH2 | dy]   -> dW2 (rows 0..63, columns 0..63) and
//                                dw3 (rows 64..127, column 64),
//   [dH1^T; dH2^T] [X | 1]    -> dW1^T (rows 0..63, columns 0..7), db1 (rows
//                                0..63, column 8) and db2 (rows 64..127,
//                                column 8).
// The transposed operands are stored MN-major, so that a row-owning thread
// writes 8 of its values with one 16-byte store.  The forward pass (its
// shared-memory layout and per-tile steps) is in kl_mlp_tc.cuh, shared with
// the pruned render's scoring.
#include "kl_mlp_tc.cuh"

namespace {

// Training kernel's shared memory (bytes from a 1024-aligned base).  BF16
// tiles (kl_tc.cuh): K-major where the threads own the rows of the tile (the
// layer inputs) or where the tile is staged once (the weights), MN-major
// where a thread owns one K index (the row of the batch) of the gradient
// products' operands.  LBO = 16 x (rows, or MN extent) in both cases.
constexpr uint32_t kLboA = kTile * 16;        // [H1^T; H2^T], [dH1^T; dH2^T]: M = 128, MN-major
constexpr uint32_t kLboB1 = 80 * 16;          // [dH2 | dy | 0]: N = 80, MN-major
constexpr uint32_t kLboB2 = 16 * 16;          // [X | 1 | 0]: N = 16, MN-major

// training kernel
constexpr uint32_t SM_W1 = 0;                      // B of layer 1: [h][f], f < 16
constexpr uint32_t SM_W2 = SM_W1 + 2 * kLboW;      // B of layer 2: [out][in] (W2^T)
constexpr uint32_t SM_W2T = SM_W2 + 8 * kLboW;     // B of dH1:     [in][out] (W2)
constexpr uint32_t SM_X = SM_W2T + 8 * kLboW;      // A of layer 1: [row][f]
constexpr uint32_t SM_H1 = SM_X + 2 * kLboRow;     // A of layer 2: [row][in]
constexpr uint32_t SM_DH2 = SM_H1 + 8 * kLboRow;   // A of dH1:     [row][out]
constexpr uint32_t SM_A1 = SM_DH2 + 8 * kLboRow;   // [H1^T; H2^T]:  [m][row]
constexpr uint32_t SM_A2 = SM_A1 + 16 * kLboA;     // [dH1^T; dH2^T]: [m][row]
constexpr uint32_t SM_B1 = SM_A2 + 16 * kLboA;     // [n][row], n < 80
constexpr uint32_t SM_B2 = SM_B1 + 16 * kLboB1;    // [n][row], n < 16
constexpr uint32_t SM_PAR = SM_B2 + 16 * kLboB2;   // b1, b2, w3 (FP32)
constexpr uint32_t SM_RED = SM_PAR + 3 * kHid * 4; // per-warp loss and db3
constexpr uint32_t SM_BAR = SM_RED + 32;           // mbarrier, TMEM address
constexpr uint32_t kGradSmem = SM_BAR + 16;

static_assert(kGradSmem <= 227 * 1024, "training shared memory");

// TMEM columns beyond the layer outputs TD1, TD2 (dH1 reuses TD1): the two
// gradient accumulators.
constexpr uint32_t TWA = 128, TWB = 224;

// MN elements m .. m+7 (m a multiple of 8) of K index t of an MN-major tile.
__device__ __forceinline__ void st_mn8(unsigned char* base, uint32_t lbo, int m, int t,
                                       const float* v) {
  *reinterpret_cast<uint4*>(base + tc_off_mn(m, t, lbo)) = pack8(v);
}

// y = network(x) for n rows of 8 features, one 128-row tile per CTA at a time.
__global__ void __launch_bounds__(kTile, 1) mlp_forward_kernel(const float* __restrict__ P,
                                                               const float* __restrict__ x,
                                                               uint64_t n,
                                                               float* __restrict__ y) {
  extern __shared__ __align__(1024) unsigned char sm[];
  Fwd F = fwd_begin(sm, P);
  const uint64_t tiles = (n + kTile - 1) / kTile;
  for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const uint64_t row = tile * kTile + threadIdx.x;
    float xv[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (row < n) {
      const float4 u = *reinterpret_cast<const float4*>(x + row * kIn);
      const float4 w = *reinterpret_cast<const float4*>(x + row * kIn + 4);
      xv[0] = u.x; xv[1] = u.y; xv[2] = u.z; xv[3] = u.w;
      xv[4] = w.x; xv[5] = w.y; xv[6] = w.z; xv[7] = w.w;
    }
    // NaN for the whole CTA's rows once an MMA has not finished
    const float v = fwd_tile(F, xv);
    if (row < n) y[row] = v;
  }
  fwd_end(F);
}

// Gradients are summed in a fixed order, so that a training run repeats
// bit for bit: every block of mlp_grad_kernel writes its partial sums to
// scratch (its tiles are fixed by its index), and mlp_reduce_kernel adds
// them up in a fixed order.  Per-block partials:
//   backward: db1 [64] | db2 [64] | dw3 [64] | db3 | loss;
//   weights:  dW2 [64][64] | dW1 [8][64].
constexpr int kBwdPart = 3 * kHid + 2;
constexpr int kWgPart = kHid * kHid + kIn * kHid;
constexpr int kBwdMaxBlocks = 512, kWgMaxBlocks = 256;

__global__ void __launch_bounds__(kTile, 1) mlp_grad_kernel(
    const float* __restrict__ P, const float* __restrict__ x, const float* __restrict__ tgt,
    uint64_t n, float under, float* __restrict__ bwd_part, float* __restrict__ wg_part) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const float* b1 = reinterpret_cast<const float*>(sm + SM_PAR);
  const float* b2 = b1 + kHid;
  const float* w3 = b2 + kHid;
  float* red = reinterpret_cast<float*>(sm + SM_RED);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + SM_BAR);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + SM_BAR + 8);
  stage_weights(sm, SM_W1, SM_W2, (int)SM_W2T, SM_PAR, P);
  const float b3 = P[OFF_B3];
  // constant parts of the operand tiles: X padding, the zero columns 72..79 of B1
  *reinterpret_cast<uint4*>(sm + SM_X + tc_off(t, 8, kLboRow)) = make_uint4(0u, 0u, 0u, 0u);
  *reinterpret_cast<uint4*>(sm + SM_B1 + tc_off_mn(72, t, kLboB1)) = make_uint4(0u, 0u, 0u, 0u);
  if (t == 0) mbar_init(bar, 1);
  if (warp == 0) tc_alloc(slot, 256);
  sync_for_mma();
  const uint32_t tm = *slot;
  const uint32_t la = tm + ((uint32_t)(warp * 32) << 16);
  const uint32_t id64 = tc_idesc_bf16(128, 64), id80 = tc_idesc_bf16(128, 80, 1, 1),
                 id16 = tc_idesc_bf16(128, 16, 1, 1);
  const uint32_t aX = smem_u32(sm + SM_X), aH1 = smem_u32(sm + SM_H1),
                 aDH2 = smem_u32(sm + SM_DH2), aA1 = smem_u32(sm + SM_A1),
                 aA2 = smem_u32(sm + SM_A2), aB1 = smem_u32(sm + SM_B1),
                 aB2 = smem_u32(sm + SM_B2), aW1 = smem_u32(sm + SM_W1),
                 aW2 = smem_u32(sm + SM_W2), aW2T = smem_u32(sm + SM_W2T);
  const float inv_n = 1.0f / (float)n;
  float lsum = 0.0f, gb3 = 0.0f;
  uint32_t phase = 0;
  bool ok = true, first = true;
  const uint64_t tiles = (n + kTile - 1) / kTile;
  for (uint64_t tile = blockIdx.x; ok && tile < tiles; tile += gridDim.x) {
    const uint64_t row = tile * kTile + t;
    const bool valid = row < n;
    float xv[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    float tg = 0.0f;
    if (valid) {
      const float4 u = *reinterpret_cast<const float4*>(x + row * kIn);
      const float4 w = *reinterpret_cast<const float4*>(x + row * kIn + 4);
      xv[0] = u.x; xv[1] = u.y; xv[2] = u.z; xv[3] = u.w;
      xv[4] = w.x; xv[5] = w.y; xv[6] = w.z; xv[7] = w.w;
      tg = tgt[row];
    }
    *reinterpret_cast<uint4*>(sm + SM_X + tc_off(t, 0, kLboRow)) =
        make_uint4(pack_bf16(xv[0], xv[1]), pack_bf16(xv[2], xv[3]), pack_bf16(xv[4], xv[5]),
                   pack_bf16(xv[6], xv[7]));
    st_mn8(sm + SM_B2, kLboB2, 0, t, xv);
    {
      const float one[8] = {valid ? 1.0f : 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      st_mn8(sm + SM_B2, kLboB2, kIn, t, one);
    }
    // layer 1: H1 = relu(X W1 + b1)
    sync_for_mma();
    if (t == 0) {
      tc_mma(tm + TD1, tc_desc(aX, kLboRow), tc_desc(aW1, kLboW), id64, 0u);
      tc_commit(bar);
    }
    if (!(ok = mma_done(bar, phase))) break;
    tc_fence_after();
    uint64_t m1 = 0;
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
      float v[16];
      tc_ld16(la + TD1 + c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float a = v[j] + b1[c + j];
        m1 |= (uint64_t)(a > 0.0f) << (c + j);
        v[j] = fmaxf(a, 0.0f);
      }
      st_mn8(sm + SM_A1, kLboA, c, t, v);
      st_mn8(sm + SM_A1, kLboA, c + 8, t, v + 8);
      st_row16(sm + SM_H1, t, c, v);
    }
    // layer 2: H2 = relu(H1 W2 + b2), y = H2 . w3 + b3
    sync_for_mma();
    if (t == 0) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        tc_mma(tm + TD2, tc_desc(aH1 + 2 * ks * kLboRow, kLboRow),
               tc_desc(aW2 + 2 * ks * kLboW, kLboW), id64, ks > 0 ? 1u : 0u);
      tc_commit(bar);
    }
    if (!(ok = mma_done(bar, phase))) break;
    tc_fence_after();
    uint64_t m2 = 0;
    float yv = 0.0f;
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
      float v[16];
      tc_ld16(la + TD2 + c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float a = v[j] + b2[c + j];
        m2 |= (uint64_t)(a > 0.0f) << (c + j);
        v[j] = fmaxf(a, 0.0f);
        yv += v[j] * w3[c + j];
      }
      st_mn8(sm + SM_A1, kLboA, kHid + c, t, v);
      st_mn8(sm + SM_A1, kLboA, kHid + c + 8, t, v + 8);
    }
    yv += b3;
    // weighted squared error: weight `under` where the output is below the target
    const float e = yv - tg;
    const float wgt = e < 0.0f ? under : 1.0f;
    const float dy = valid ? 2.0f * wgt * e * inv_n : 0.0f;
    if (valid) lsum += wgt * e * e;
    gb3 += dy;
    // dH2 = dy w3 through the second ReLU
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
      float v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = ((m2 >> (c + j)) & 1ull) ? dy * w3[c + j] : 0.0f;
      st_mn8(sm + SM_B1, kLboB1, c, t, v);
      st_mn8(sm + SM_B1, kLboB1, c + 8, t, v + 8);
      st_mn8(sm + SM_A2, kLboA, kHid + c, t, v);
      st_mn8(sm + SM_A2, kLboA, kHid + c + 8, t, v + 8);
      st_row16(sm + SM_DH2, t, c, v);
    }
    {
      const float dyv[8] = {dy, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      st_mn8(sm + SM_B1, kLboB1, kHid, t, dyv);
    }
    // dH1 = dH2 W2^T through the first ReLU
    sync_for_mma();
    if (t == 0) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        tc_mma(tm + TD1, tc_desc(aDH2 + 2 * ks * kLboRow, kLboRow),
               tc_desc(aW2T + 2 * ks * kLboW, kLboW), id64, ks > 0 ? 1u : 0u);
      tc_commit(bar);
    }
    if (!(ok = mma_done(bar, phase))) break;
    tc_fence_after();
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
      float v[16];
      tc_ld16(la + TD1 + c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = ((m1 >> (c + j)) & 1ull) ? v[j] : 0.0f;
      st_mn8(sm + SM_A2, kLboA, c, t, v);
      st_mn8(sm + SM_A2, kLboA, c + 8, t, v + 8);
    }
    // the sums over this tile's rows, added to the CTA's accumulators
    sync_for_mma();
    if (t == 0) {
#pragma unroll
      for (int ks = 0; ks < kTile / 16; ++ks)
        tc_mma(tm + TWA, tc_desc(aA1 + 2 * ks * kLboA, kLboA),
               tc_desc(aB1 + 2 * ks * kLboB1, kLboB1), id80, (!first || ks > 0) ? 1u : 0u);
#pragma unroll
      for (int ks = 0; ks < kTile / 16; ++ks)
        tc_mma(tm + TWB, tc_desc(aA2 + 2 * ks * kLboA, kLboA),
               tc_desc(aB2 + 2 * ks * kLboB2, kLboB2), id16, (!first || ks > 0) ? 1u : 0u);
      tc_commit(bar);
    }
    if (!(ok = mma_done(bar, phase))) break;
    first = false;
  }
  // this block's partials
  float* bp = bwd_part + (size_t)blockIdx.x * kBwdPart;
  float* wp = wg_part + (size_t)blockIdx.x * kWgPart;
  if (!ok) mbar_wait(bar, phase ^ 1u, kWaitCycles);   // let a late MMA finish first
  tc_fence_after();
  if (ok && !first) {
    // lanes 0..63: dW2 rows, dW1^T rows and db1; lanes 64..127: dw3 and db2
    const int m = t;
    float v[16];
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
      tc_ld16(la + TWA + c, v);
      if (m < kHid)
#pragma unroll
        for (int j = 0; j < 16; ++j) wp[m * kHid + c + j] = v[j];
    }
    tc_ld16(la + TWA + kHid, v);
    if (m >= kHid) bp[2 * kHid + (m - kHid)] = v[0];
    tc_ld16(la + TWB, v);
    if (m < kHid) {
#pragma unroll
      for (int f = 0; f < kIn; ++f) wp[kHid * kHid + f * kHid + m] = v[f];
      bp[m] = v[kIn];
    } else {
      bp[kHid + (m - kHid)] = v[kIn];
    }
  } else {
    for (int i = t; i < kWgPart; i += blockDim.x) wp[i] = 0.0f;
    for (int i = t; i < 3 * kHid; i += blockDim.x) bp[i] = 0.0f;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lsum += __shfl_xor_sync(0xFFFFFFFFu, lsum, o);
    gb3 += __shfl_xor_sync(0xFFFFFFFFu, gb3, o);
  }
  if (lane == 0) {
    red[2 * warp] = lsum;
    red[2 * warp + 1] = gb3;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (t == 0) {
    bp[3 * kHid] = ((red[1] + red[3]) + red[5]) + red[7];
    bp[3 * kHid + 1] =
        ok ? (((red[0] + red[2]) + red[4]) + red[6]) * inv_n : __int_as_float(0x7FC00000);
  }
  if (warp == 0) tc_dealloc(tm, 256);
}

// One Adam step (Kingma and Ba, 2015) for parameter i with gradient g.
struct AdamStep {
  float* p;  // null: no step
  float* m;
  float* v;
  float lr, b1, b2, eps, c1, c2;  // c1, c2: the bias corrections 1 - beta^step
};
__device__ __forceinline__ void adam_one(const AdamStep& A, int i, float g) {
  const float mi = A.b1 * A.m[i] + (1.0f - A.b1) * g;
  const float vi = A.b2 * A.v[i] + (1.0f - A.b2) * g * g;
  A.m[i] = mi;
  A.v[i] = vi;
  A.p[i] -= A.lr * (mi / A.c1) / (sqrtf(vi / A.c2) + A.eps);
}

// grad[i] (and, for i = KL_MLP_NPARAMS, the loss) = the sum of the partials
// of output i: one block per output, thread t takes partials t, t + 128, ...
// in order, then a fixed reduction tree.  With an Adam step, the block then
// applies it to parameter i (grad may then be null).
__global__ void __launch_bounds__(128) mlp_reduce_kernel(const float* __restrict__ bwd, int n_bwd,
                                                         const float* __restrict__ wg, int n_wg,
                                                         float* __restrict__ grad,
                                                         float* __restrict__ loss, AdamStep A) {
  const int i = blockIdx.x;
  const float* src;
  int stride, count;
  if (i == KL_MLP_NPARAMS) {                       // the loss
    src = bwd + 3 * kHid + 1; stride = kBwdPart; count = n_bwd;
  } else if (i < OFF_B1) {                         // W1
    src = wg + kHid * kHid + i; stride = kWgPart; count = n_wg;
  } else if (i < OFF_W2) {                         // b1
    src = bwd + (i - OFF_B1); stride = kBwdPart; count = n_bwd;
  } else if (i < OFF_B2) {                         // W2
    src = wg + (i - OFF_W2); stride = kWgPart; count = n_wg;
  } else if (i < OFF_W3) {                         // b2
    src = bwd + kHid + (i - OFF_B2); stride = kBwdPart; count = n_bwd;
  } else if (i < OFF_B3) {                         // w3
    src = bwd + 2 * kHid + (i - OFF_W3); stride = kBwdPart; count = n_bwd;
  } else {                                         // b3
    src = bwd + 3 * kHid; stride = kBwdPart; count = n_bwd;
  }
  float acc = 0.0f;
  for (int b = threadIdx.x; b < count; b += blockDim.x) acc += src[(size_t)b * stride];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  __shared__ float ws[4];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    const float v = (ws[0] + ws[1]) + (ws[2] + ws[3]);
    if (i == KL_MLP_NPARAMS) {
      *loss = v;
    } else {
      if (grad) grad[i] = v;
      if (A.p) adam_one(A, i, v);
    }
  }
}

__global__ void adam_kernel(float* __restrict__ g, int n, AdamStep A) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    adam_one(A, i, g[i]);
    g[i] = 0.0f;
  }
}

AdamStep adam_args(float* p, float* m, float* v, uint32_t step, float lr, float beta1,
                   float beta2, float eps) {
  return {p, m, v, lr, beta1, beta2, eps, 1.0f - powf(beta1, (float)step),
          1.0f - powf(beta2, (float)step)};
}

}  // namespace

extern "C" int kl_mlp_forward(const float* d_params, const float* d_x, uint64_t n, float* d_y,
                              void* stream) {
  if (n == 0) return KL_OK;
  if (!d_params || !d_x || !d_y) return KL_EINVAL;
  if (((uintptr_t)d_x & 15u) != 0) return KL_EINVAL;
  const int sms = sm_count();
  if (sms <= 0) return KL_ECUDA;
  if (cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kFwdSmem) != cudaSuccess)
    return KL_ECUDA;
  const uint64_t tiles = (n + kTile - 1) / kTile;
  const unsigned grid = (unsigned)(tiles < (uint64_t)sms * 4 ? tiles : (uint64_t)sms * 4);
  mlp_forward_kernel<<<grid, kTile, kFwdSmem, (cudaStream_t)stream>>>(d_params, d_x, n, d_y);
  return check_launch();
}

extern "C" size_t kl_mlp_scratch_bytes(uint64_t n) {
  (void)n;
  return align256((size_t)kBwdMaxBlocks * kBwdPart * sizeof(float)) +
         align256((size_t)kWgMaxBlocks * kWgPart * sizeof(float));
}

namespace {

// Gradient pass, then the fixed-order reduce (with an Adam step when A.p).
int grad_pass(const float* d_params, const float* d_x, const float* d_t, uint64_t n,
              float under_weight, float* d_grad, float* d_loss, void* d_scratch,
              size_t scratch_bytes, cudaStream_t s, const AdamStep& A) {
  if (n == 0 || !d_params || !d_x || !d_t || !d_loss || !d_scratch) return KL_EINVAL;
  if (!(under_weight > 0.0f)) return KL_EINVAL;
  if (scratch_bytes < kl_mlp_scratch_bytes(n)) return KL_ENOSPACE;
  if (((uintptr_t)d_scratch & 255u) != 0 || ((uintptr_t)d_x & 15u) != 0) return KL_EINVAL;
  const int sms = sm_count();
  if (sms <= 0) return KL_ECUDA;
  if (cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kGradSmem) != cudaSuccess)
    return KL_ECUDA;
  float* bwd_part = (float*)d_scratch;
  float* wg_part =
      (float*)((char*)d_scratch + align256((size_t)kBwdMaxBlocks * kBwdPart * sizeof(float)));
  // one CTA per SM (its shared memory allows no second), tiles of 128 rows
  const uint64_t tiles = (n + kTile - 1) / kTile;
  uint64_t grid = tiles < (uint64_t)sms ? tiles : (uint64_t)sms;
  if (grid > (uint64_t)kWgMaxBlocks) grid = kWgMaxBlocks;
  mlp_grad_kernel<<<(unsigned)grid, kTile, kGradSmem, s>>>(d_params, d_x, d_t, n, under_weight,
                                                           bwd_part, wg_part);
  if (check_launch() != KL_OK) return KL_ECUDA;
  mlp_reduce_kernel<<<KL_MLP_NPARAMS + 1, 128, 0, s>>>(bwd_part, (int)grid, wg_part, (int)grid,
                                                       d_grad, d_loss, A);
  return check_launch();
}

}  // namespace

extern "C" int kl_mlp_grad(const float* d_params, const float* d_x, const float* d_t, uint64_t n,
                           float under_weight, float* d_grad, float* d_loss, void* d_scratch,
                           size_t scratch_bytes, void* stream) {
  if (!d_grad) return KL_EINVAL;
  return grad_pass(d_params, d_x, d_t, n, under_weight, d_grad, d_loss, d_scratch, scratch_bytes,
                   (cudaStream_t)stream, AdamStep{});
}

extern "C" int kl_mlp_adam(float* d_params, float* d_m, float* d_v, float* d_grad, uint32_t step,
                           float lr, float beta1, float beta2, float eps, void* stream) {
  if (!d_params || !d_m || !d_v || !d_grad || step == 0) return KL_EINVAL;
  adam_kernel<<<(KL_MLP_NPARAMS + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      d_grad, KL_MLP_NPARAMS, adam_args(d_params, d_m, d_v, step, lr, beta1, beta2, eps));
  return check_launch();
}

namespace {

// One warp: a wait that nothing completes must give up at its bound, and a
// wait on a phase this warp completes must succeed.
__global__ void wait_selftest_kernel(long long limit, uint32_t* out) {
  __shared__ uint64_t bar[2];
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  __syncwarp();
  const long long t0 = clock64();
  const bool done = mbar_wait(&bar[0], 0u, limit);  // no arrival: must give up
  const long long took = clock64() - t0;
  __syncwarp();
  if (threadIdx.x == 0)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar[1])) : "memory");
  __syncwarp();
  const bool done2 = mbar_wait(&bar[1], 0u, limit);
  if (threadIdx.x == 0) {
    out[0] = done ? 0u : 1u;
    out[1] = done2 ? 1u : 0u;
    out[2] = took > 0xFFFFFFFFll ? 0xFFFFFFFFu : (uint32_t)took;
    out[3] = 0u;
  }
}

}  // namespace

extern "C" int kl_wait_selftest(uint64_t limit_cycles, uint32_t* d_result, void* stream) {
  if (!d_result || limit_cycles == 0 || limit_cycles > (1ull << 31)) return KL_EINVAL;
  wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>((long long)limit_cycles, d_result);
  return check_launch();
}

extern "C" int kl_mlp_train_step(float* d_params, float* d_m, float* d_v, const float* d_x,
                                 const float* d_t, uint64_t n, float under_weight, uint32_t step,
                                 float lr, float beta1, float beta2, float eps, float* d_loss,
                                 float* d_grad, void* d_scratch, size_t scratch_bytes,
                                 void* stream) {
  if (!d_params || !d_m || !d_v || step == 0) return KL_EINVAL;
  return grad_pass(d_params, d_x, d_t, n, under_weight, d_grad, d_loss, d_scratch, scratch_bytes,
                   (cudaStream_t)stream,
                   adam_args(d_params, d_m, d_v, step, lr, beta1, beta2, eps));
}
