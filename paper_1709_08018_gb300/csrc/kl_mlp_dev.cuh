// The level-of-detail network's parameter layout and BF16 packing, shared by
// its kernels (kl_mlp.cu, kl_mlp_tc.cuh) and the pruned render (kl_lod.cu).
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

}  // namespace
