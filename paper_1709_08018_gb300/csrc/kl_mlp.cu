// The level-of-detail network: an MLP 8 -> 64 -> 64 -> 1 with ReLU, BF16
// weights and activations on the tensor cores with FP32 accumulation, and
// its training kernels (forward, backward, weight gradients, Adam).
//
// Parameter vector (FP32 master copy, KL_MLP_NPARAMS floats):
//   W1 [8][64] | b1 [64] | W2 [64][64] | b2 [64] | w3 [64] | b3
// (W[in][out]: h_out = sum_in x_in W[in][out] + b_out).  Loss: mean squared
// error over the batch.
//
// Tensor-core tiles use mma.sync.m16n8k16 (BF16 in, FP32 accumulate).  A warp
// owns 16 rows; the FP32 accumulator fragment of one layer (rows g, g+8 and
// columns 2c, 2c+1 of each 8-column tile, g = lane/4, c = lane%4) is exactly
// the BF16 A-operand fragment of the next layer's 16-column k-step, so
// activations never leave registers between layers.
#include "kl_mlp_dev.cuh"

namespace {

__global__ void __launch_bounds__(128) mlp_forward_kernel(const float* __restrict__ P,
                                                          const float* __restrict__ x,
                                                          uint64_t n, float* __restrict__ y) {
  __shared__ MlpSmem S;
  load_mlp(S, P);
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t tile = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
       tile * 16 < n; tile += warps) {
    const uint64_t r0 = tile * 16;
    uint32_t xa0, xa1;
    x_fragment(x, n, r0, xa0, xa1);
    Tile T;
    forward_tile(S, xa0, xa1, T);
    if (c == 0) {
      if (r0 + g < n) y[r0 + g] = T.y0;
      if (r0 + g + 8 < n) y[r0 + g + 8] = T.y1;
    }
  }
}

// Gradients are summed in a fixed order, so that a training run repeats
// bit for bit: every block of mlp_backward_kernel and of mlp_wgrad_kernel
// writes its partial sums to scratch, and mlp_reduce_kernel adds them up in a
// fixed order.  Per-block partial of the backward pass:
// db1 [64] | db2 [64] | dw3 [64] | db3 | loss.
constexpr int kBwdPart = 3 * kHid + 2;
constexpr int kWgPart = kHid * kHid + kIn * kHid;  // dW2 [64][64] | dW1 [8][64]
constexpr int kBwdMaxBlocks = 512, kWgMaxBlocks = 256;

// Forward + backward of 16-row tiles.  Per-parameter gradients of the
// biases and w3, and the loss, are accumulated in registers over all tiles
// of the warp and reduced once; the activations the weight gradients need
// (H1, dH2 and dH1, BF16) go to scratch for mlp_wgrad_kernel.
__global__ void __launch_bounds__(128) mlp_backward_kernel(
    const float* __restrict__ P, const float* __restrict__ x, const float* __restrict__ tgt,
    uint64_t n, float under, float* __restrict__ part,
    __nv_bfloat16* __restrict__ h1s, __nv_bfloat16* __restrict__ dh2s,
    __nv_bfloat16* __restrict__ dh1s) {
  __shared__ MlpSmem S;
  load_mlp(S, P);
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  const float inv_n = 1.0f / (float)n;
  float gb1[16], gb2[16], gw3[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) gb1[i] = gb2[i] = gw3[i] = 0.0f;
  float gb3 = 0.0f, lsum = 0.0f;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t tile = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
       tile * 16 < n; tile += warps) {
    const uint64_t r0 = tile * 16, ra = r0 + g, rb = r0 + g + 8;
    uint32_t xa0, xa1;
    x_fragment(x, n, r0, xa0, xa1);
    Tile T;
    forward_tile(S, xa0, xa1, T);
    const bool va = ra < n, vb = rb < n;
    const float ea = va ? T.y0 - tgt[ra] : 0.0f, eb = vb ? T.y1 - tgt[rb] : 0.0f;
    // weighted squared error: weight `under` where the output is below the target
    const float wa = ea < 0.0f ? under : 1.0f, wb = eb < 0.0f ? under : 1.0f;
    if (c == 0) lsum += wa * ea * ea + wb * eb * eb;
    const float dya = 2.0f * wa * ea * inv_n, dyb = 2.0f * wb * eb * inv_n;
    if (c == 0) gb3 += dya + dyb;
    // dH2 = dy w3 (ReLU mask), dw3 += H2^T dy, db2 += dH2
    float dh2[8][4];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int j = 8 * t + 2 * c;
      gw3[2 * t] += T.h2[t][0] * dya + T.h2[t][2] * dyb;
      gw3[2 * t + 1] += T.h2[t][1] * dya + T.h2[t][3] * dyb;
      dh2[t][0] = T.h2[t][0] > 0.0f ? dya * S.w3[j] : 0.0f;
      dh2[t][1] = T.h2[t][1] > 0.0f ? dya * S.w3[j + 1] : 0.0f;
      dh2[t][2] = T.h2[t][2] > 0.0f ? dyb * S.w3[j] : 0.0f;
      dh2[t][3] = T.h2[t][3] > 0.0f ? dyb * S.w3[j + 1] : 0.0f;
      gb2[2 * t] += dh2[t][0] + dh2[t][2];
      gb2[2 * t + 1] += dh2[t][1] + dh2[t][3];
    }
    // dH1 = dH2 W2^T (tensor cores; dH2 fragments reused as A operands), ReLU mask
    uint32_t a[4][4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      a[s][0] = pack_bf16(dh2[2 * s][0], dh2[2 * s][1]);
      a[s][1] = pack_bf16(dh2[2 * s][2], dh2[2 * s][3]);
      a[s][2] = pack_bf16(dh2[2 * s + 1][0], dh2[2 * s + 1][1]);
      a[s][3] = pack_bf16(dh2[2 * s + 1][2], dh2[2 * s + 1][3]);
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&S.w2[8 * t + g][16 * s + 2 * c]);
        const uint32_t b1 =
            *reinterpret_cast<const uint32_t*>(&S.w2[8 * t + g][16 * s + 8 + 2 * c]);
        mma_bf16(d, a[s][0], a[s][1], a[s][2], a[s][3], b0, b1);
      }
      d[0] = T.h1[t][0] > 0.0f ? d[0] : 0.0f;
      d[1] = T.h1[t][1] > 0.0f ? d[1] : 0.0f;
      d[2] = T.h1[t][2] > 0.0f ? d[2] : 0.0f;
      d[3] = T.h1[t][3] > 0.0f ? d[3] : 0.0f;
      gb1[2 * t] += d[0] + d[2];
      gb1[2 * t + 1] += d[1] + d[3];
      const int j = 8 * t + 2 * c;
      if (va) {
        *reinterpret_cast<uint32_t*>(h1s + ra * kHid + j) = pack_bf16(T.h1[t][0], T.h1[t][1]);
        *reinterpret_cast<uint32_t*>(dh2s + ra * kHid + j) = pack_bf16(dh2[t][0], dh2[t][1]);
        *reinterpret_cast<uint32_t*>(dh1s + ra * kHid + j) = pack_bf16(d[0], d[1]);
      }
      if (vb) {
        *reinterpret_cast<uint32_t*>(h1s + rb * kHid + j) = pack_bf16(T.h1[t][2], T.h1[t][3]);
        *reinterpret_cast<uint32_t*>(dh2s + rb * kHid + j) = pack_bf16(dh2[t][2], dh2[t][3]);
        *reinterpret_cast<uint32_t*>(dh1s + rb * kHid + j) = pack_bf16(d[2], d[3]);
      }
    }
  }
  // reduce over the 8 row groups (lanes with the same c), then one atomic per value
#pragma unroll
  for (int i = 0; i < 16; ++i) {
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      gb1[i] += __shfl_xor_sync(0xFFFFFFFFu, gb1[i], o);
      gb2[i] += __shfl_xor_sync(0xFFFFFFFFu, gb2[i], o);
      gw3[i] += __shfl_xor_sync(0xFFFFFFFFu, gw3[i], o);
    }
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    gb3 += __shfl_xor_sync(0xFFFFFFFFu, gb3, o);
    lsum += __shfl_xor_sync(0xFFFFFFFFu, lsum, o);
  }
  // the block's four warp partials, added in warp order: one partial per block
  __shared__ float wp[4][kBwdPart];
  float* out = wp[threadIdx.x >> 5];
  if (g == 0) {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int j = 8 * t + 2 * c;
      out[j] = gb1[2 * t];
      out[j + 1] = gb1[2 * t + 1];
      out[kHid + j] = gb2[2 * t];
      out[kHid + j + 1] = gb2[2 * t + 1];
      out[2 * kHid + j] = gw3[2 * t];
      out[2 * kHid + j + 1] = gw3[2 * t + 1];
    }
  }
  if (lane == 0) {
    out[3 * kHid] = gb3;
    out[3 * kHid + 1] = lsum * inv_n;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kBwdPart; i += blockDim.x)
    part[(size_t)blockIdx.x * kBwdPart + i] = ((wp[0][i] + wp[1][i]) + wp[2][i]) + wp[3][i];
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p, uint64_t stride, uint64_t n,
                                            uint64_t r, int col) {
  const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
  const __nv_bfloat16 lo = r < n ? p[r * stride + col] : z;
  const __nv_bfloat16 hi = r + 1 < n ? p[(r + 1) * stride + col] : z;
  __nv_bfloat162 v;
  v.x = lo;
  v.y = hi;
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Weight gradients, split over the batch: dW2 = H1^T dH2 (64x64) and
// dW1 = X^T dH1 (8x64), K = the batch rows.  Block = 5 warps: warps 0..3 own
// the 16-row m-tiles of dW2, warp 4 the (padded) m-tile of dW1; each block
// takes one row range, accumulates in registers and writes its partial once.
__global__ void __launch_bounds__(160) mlp_wgrad_kernel(
    const float* __restrict__ x, uint64_t n, const __nv_bfloat16* __restrict__ h1s,
    const __nv_bfloat16* __restrict__ dh2s, const __nv_bfloat16* __restrict__ dh1s,
    uint64_t rows_per_block, float* __restrict__ part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  const uint64_t r_begin = blockIdx.x * rows_per_block;
  const uint64_t r_end = min(n, r_begin + rows_per_block);
  float acc[8][4];
#pragma unroll
  for (int t = 0; t < 8; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.0f;
  const __nv_bfloat16* B = warp < 4 ? dh2s : dh1s;
  for (uint64_t r0 = r_begin; r0 < r_end; r0 += 16) {
    uint32_t a0, a1, a2, a3;
    if (warp < 4) {
      const int m = 16 * warp + g;
      a0 = ld_pair(h1s, kHid, r_end, r0 + 2 * c, m);
      a1 = ld_pair(h1s, kHid, r_end, r0 + 2 * c, m + 8);
      a2 = ld_pair(h1s, kHid, r_end, r0 + 2 * c + 8, m);
      a3 = ld_pair(h1s, kHid, r_end, r0 + 2 * c + 8, m + 8);
    } else {
      // X^T rows are features: g < 8 real, g + 8 padding
      const uint64_t ra = r0 + 2 * c, rb = r0 + 2 * c + 8;
      const float xa = ra < r_end ? x[ra * kIn + g] : 0.0f;
      const float xb = ra + 1 < r_end ? x[(ra + 1) * kIn + g] : 0.0f;
      const float xc = rb < r_end ? x[rb * kIn + g] : 0.0f;
      const float xd = rb + 1 < r_end ? x[(rb + 1) * kIn + g] : 0.0f;
      a0 = pack_bf16(xa, xb);
      a1 = 0u;
      a2 = pack_bf16(xc, xd);
      a3 = 0u;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const uint32_t b0 = ld_pair(B, kHid, r_end, r0 + 2 * c, 8 * t + g);
      const uint32_t b1 = ld_pair(B, kHid, r_end, r0 + 2 * c + 8, 8 * t + g);
      mma_bf16(acc[t], a0, a1, a2, a3, b0, b1);
    }
  }
  float* out = part + (size_t)blockIdx.x * kWgPart;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int col = 8 * t + 2 * c;
    if (warp < 4) {
      const int m = 16 * warp + g;
      out[m * kHid + col] = acc[t][0];
      out[m * kHid + col + 1] = acc[t][1];
      out[(m + 8) * kHid + col] = acc[t][2];
      out[(m + 8) * kHid + col + 1] = acc[t][3];
    } else {
      out[kHid * kHid + g * kHid + col] = acc[t][0];
      out[kHid * kHid + g * kHid + col + 1] = acc[t][1];
    }
  }
}

// grad[i] (and, for i = KL_MLP_NPARAMS, the loss) = the sum of the partials
// of output i: one block per output, thread t takes partials t, t + 128, ...
// in order, then a fixed reduction tree.
__global__ void __launch_bounds__(128) mlp_reduce_kernel(const float* __restrict__ bwd, int n_bwd,
                                                         const float* __restrict__ wg, int n_wg,
                                                         float* __restrict__ grad,
                                                         float* __restrict__ loss) {
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
    if (i == KL_MLP_NPARAMS) *loss = v;
    else grad[i] = v;
  }
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            float* __restrict__ g, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    g[i] = 0.0f;
  }
}

}  // namespace

extern "C" int kl_mlp_forward(const float* d_params, const float* d_x, uint64_t n, float* d_y,
                              void* stream) {
  if (n == 0) return KL_OK;
  if (!d_params || !d_x || !d_y) return KL_EINVAL;
  const int sms = sm_count();
  if (sms <= 0) return KL_ECUDA;
  const uint64_t tiles = (n + 15) / 16, blocks = (tiles + 3) / 4;
  const unsigned grid = (unsigned)(blocks < (uint64_t)sms * 8 ? blocks : (uint64_t)sms * 8);
  mlp_forward_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>(d_params, d_x, n, d_y);
  return check_launch();
}

extern "C" size_t kl_mlp_scratch_bytes(uint64_t n) {
  return 3 * align256((size_t)n * kHid * sizeof(__nv_bfloat16)) +
         align256((size_t)kBwdMaxBlocks * kBwdPart * sizeof(float)) +
         align256((size_t)kWgMaxBlocks * kWgPart * sizeof(float));
}

extern "C" int kl_mlp_grad(const float* d_params, const float* d_x, const float* d_t, uint64_t n,
                           float under_weight, float* d_grad, float* d_loss, void* d_scratch,
                           size_t scratch_bytes, void* stream) {
  if (n == 0 || !d_params || !d_x || !d_t || !d_grad || !d_loss || !d_scratch) return KL_EINVAL;
  if (!(under_weight > 0.0f)) return KL_EINVAL;
  if (scratch_bytes < kl_mlp_scratch_bytes(n)) return KL_ENOSPACE;
  if (((uintptr_t)d_scratch & 255u) != 0) return KL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int sms = sm_count();
  if (sms <= 0) return KL_ECUDA;
  const size_t part = align256((size_t)n * kHid * sizeof(__nv_bfloat16));
  char* base = (char*)d_scratch;
  __nv_bfloat16* h1s = (__nv_bfloat16*)base;
  __nv_bfloat16* dh2s = (__nv_bfloat16*)(base + part);
  __nv_bfloat16* dh1s = (__nv_bfloat16*)(base + 2 * part);
  float* bwd_part = (float*)(base + 3 * part);
  float* wg_part =
      (float*)(base + 3 * part + align256((size_t)kBwdMaxBlocks * kBwdPart * sizeof(float)));
  // backward: 4 warps per block, 16-row tiles, at most 4 blocks per SM
  const uint64_t tiles = (n + 15) / 16, blocks = (tiles + 3) / 4;
  uint64_t grid = blocks < (uint64_t)sms * 4 ? blocks : (uint64_t)sms * 4;
  if (grid > (uint64_t)kBwdMaxBlocks) grid = kBwdMaxBlocks;
  mlp_backward_kernel<<<(unsigned)grid, 128, 0, s>>>(d_params, d_x, d_t, n, under_weight,
                                                     bwd_part, h1s, dh2s, dh1s);
  if (check_launch() != KL_OK) return KL_ECUDA;
  // weight gradients: row ranges of at least 64 rows, at most kWgMaxBlocks of them
  uint64_t rows_per_block = (n + kWgMaxBlocks - 1) / kWgMaxBlocks;
  rows_per_block = rows_per_block < 64 ? 64 : (rows_per_block + 15) / 16 * 16;
  const uint64_t wblocks = (n + rows_per_block - 1) / rows_per_block;
  mlp_wgrad_kernel<<<(unsigned)wblocks, 160, 0, s>>>(d_x, n, h1s, dh2s, dh1s, rows_per_block,
                                                     wg_part);
  if (check_launch() != KL_OK) return KL_ECUDA;
  mlp_reduce_kernel<<<KL_MLP_NPARAMS + 1, 128, 0, s>>>(bwd_part, (int)grid, wg_part,
                                                       (int)wblocks, d_grad, d_loss);
  return check_launch();
}

extern "C" int kl_mlp_adam(float* d_params, float* d_m, float* d_v, float* d_grad, uint32_t step,
                           float lr, float beta1, float beta2, float eps, void* stream) {
  if (!d_params || !d_m || !d_v || !d_grad || step == 0) return KL_EINVAL;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  adam_kernel<<<(KL_MLP_NPARAMS + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      d_params, d_m, d_v, d_grad, KL_MLP_NPARAMS, lr, beta1, beta2, eps, c1, c2);
  return check_launch();
}
