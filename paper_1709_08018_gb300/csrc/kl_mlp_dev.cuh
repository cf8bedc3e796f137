// Device pieces of the level-of-detail network shared by its training
// kernels (kl_mlp.cu) and the pruned render (kl_lod.cu).  See kl_mlp.cu.
#pragma once

#include <cuda_bf16.h>

#include "kl_common.cuh"

namespace {

constexpr int kIn = 8, kHid = 64;
constexpr int OFF_W1 = 0, OFF_B1 = 512, OFF_W2 = 576, OFF_B2 = 4672, OFF_W3 = 4736,
              OFF_B3 = 4800;
static_assert(OFF_B3 + 1 == KL_MLP_NPARAMS, "parameter layout");

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Weights staged in shared memory: W1T[n][16] (k = input, padded with zeros),
// W2T[n][k] and W2[k][n] in BF16; biases and w3 in FP32.
struct MlpSmem {
  __nv_bfloat16 w1t[kHid][16];
  __nv_bfloat16 w2t[kHid][kHid];
  __nv_bfloat16 w2[kHid][kHid];
  float b1[kHid], b2[kHid], w3[kHid];
  float b3;
};

__device__ void load_mlp(MlpSmem& S, const float* __restrict__ P) {
  for (int i = threadIdx.x; i < kHid * 16; i += blockDim.x) {
    const int n = i / 16, k = i % 16;
    S.w1t[n][k] = __float2bfloat16_rn(k < kIn ? P[OFF_W1 + k * kHid + n] : 0.0f);
  }
  for (int i = threadIdx.x; i < kHid * kHid; i += blockDim.x) {
    const int k = i / kHid, n = i % kHid;
    const __nv_bfloat16 w = __float2bfloat16_rn(P[OFF_W2 + i]);
    S.w2[k][n] = w;
    S.w2t[n][k] = w;
  }
  for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
    S.b1[i] = P[OFF_B1 + i];
    S.b2[i] = P[OFF_B2 + i];
    S.w3[i] = P[OFF_W3 + i];
  }
  if (threadIdx.x == 0) S.b3 = P[OFF_B3];
}

// Forward pass of one 16-row tile.  xa0/xa1: the lane's A fragment of the
// input (rows g and g+8, features 2c and 2c+1; features 8..15 are zero).
// Outputs the post-ReLU H1 and H2 accumulators and y for rows g, g+8 (valid
// in every lane of the row's quad).
struct Tile {
  float h1[8][4];
  float h2[8][4];
  float y0, y1;
};

__device__ __forceinline__ void forward_tile(const MlpSmem& S, uint32_t xa0, uint32_t xa1,
                                             Tile& T) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    T.h1[t][0] = T.h1[t][1] = T.h1[t][2] = T.h1[t][3] = 0.0f;
    const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&S.w1t[8 * t + g][2 * c]);
    mma_bf16(T.h1[t], xa0, xa1, 0u, 0u, b0, 0u);
    const float ba = S.b1[8 * t + 2 * c], bb = S.b1[8 * t + 2 * c + 1];
    T.h1[t][0] = fmaxf(T.h1[t][0] + ba, 0.0f);
    T.h1[t][1] = fmaxf(T.h1[t][1] + bb, 0.0f);
    T.h1[t][2] = fmaxf(T.h1[t][2] + ba, 0.0f);
    T.h1[t][3] = fmaxf(T.h1[t][3] + bb, 0.0f);
  }
  uint32_t a[4][4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    a[s][0] = pack_bf16(T.h1[2 * s][0], T.h1[2 * s][1]);
    a[s][1] = pack_bf16(T.h1[2 * s][2], T.h1[2 * s][3]);
    a[s][2] = pack_bf16(T.h1[2 * s + 1][0], T.h1[2 * s + 1][1]);
    a[s][3] = pack_bf16(T.h1[2 * s + 1][2], T.h1[2 * s + 1][3]);
  }
  float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    T.h2[t][0] = T.h2[t][1] = T.h2[t][2] = T.h2[t][3] = 0.0f;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&S.w2t[8 * t + g][16 * s + 2 * c]);
      const uint32_t b1 =
          *reinterpret_cast<const uint32_t*>(&S.w2t[8 * t + g][16 * s + 8 + 2 * c]);
      mma_bf16(T.h2[t], a[s][0], a[s][1], a[s][2], a[s][3], b0, b1);
    }
    const int j = 8 * t + 2 * c;
    T.h2[t][0] = fmaxf(T.h2[t][0] + S.b2[j], 0.0f);
    T.h2[t][1] = fmaxf(T.h2[t][1] + S.b2[j + 1], 0.0f);
    T.h2[t][2] = fmaxf(T.h2[t][2] + S.b2[j], 0.0f);
    T.h2[t][3] = fmaxf(T.h2[t][3] + S.b2[j + 1], 0.0f);
    y0 += T.h2[t][0] * S.w3[j] + T.h2[t][1] * S.w3[j + 1];
    y1 += T.h2[t][2] * S.w3[j] + T.h2[t][3] * S.w3[j + 1];
  }
  y0 += __shfl_xor_sync(0xFFFFFFFFu, y0, 1);
  y0 += __shfl_xor_sync(0xFFFFFFFFu, y0, 2);
  y1 += __shfl_xor_sync(0xFFFFFFFFu, y1, 1);
  y1 += __shfl_xor_sync(0xFFFFFFFFu, y1, 2);
  T.y0 = y0 + S.b3;
  T.y1 = y1 + S.b3;
}

__device__ __forceinline__ void x_fragment(const float* __restrict__ x, uint64_t n, uint64_t r0,
                                           uint32_t& xa0, uint32_t& xa1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  const uint64_t ra = r0 + g, rb = r0 + g + 8;
  const float2 va = ra < n ? *reinterpret_cast<const float2*>(x + ra * kIn + 2 * c)
                           : make_float2(0.0f, 0.0f);
  const float2 vb = rb < n ? *reinterpret_cast<const float2*>(x + rb * kIn + 2 * c)
                           : make_float2(0.0f, 0.0f);
  xa0 = pack_bf16(va.x, va.y);
  xa1 = pack_bf16(vb.x, vb.y);
}

}  // namespace
