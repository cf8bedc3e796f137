// The level-of-detail network's forward pass on the fifth-generation tensor
// cores, shared by the training kernels (kl_mlp.cu) and the pruned render's
// per-node scoring (kl_lod.cu).
//
// A CTA of 128 threads takes tiles of 128 rows; thread t owns row t of the
// tile, which is lane t of every accumulator in tensor memory (M = 128), so
// bias, ReLU and the last layer's dot product are row-local.  The two layer
// products run as tcgen05 MMAs on BF16 tiles in shared memory (kl_tc.cuh):
//   H1 = X W1 (K = 16: 8 inputs and zero padding), H2 = H1 W2,
// with FP32 accumulators in tensor memory, read back with tcgen05.ld.
#pragma once

#include "kl_mlp_dev.cuh"
#include "kl_tc.cuh"

namespace {

constexpr int kTile = 128;                        // rows per tile = TMEM lanes = threads
constexpr long long kWaitCycles = 2000000000ll;   // bound on an MMA wait (about a second)

// BF16 tiles, K-major where the threads own the rows of the tile (the layer
// inputs) or where the tile is staged once (the weights): LBO = 16 x rows.
constexpr uint32_t kLboW = 64 * 16;           // weight tiles, 64 rows
constexpr uint32_t kLboRow = kTile * 16;      // X, H1, dH2: 128 rows, row-wise

// Forward pass: shared memory (bytes from a 1024-aligned base).
constexpr uint32_t FW_W1 = 0;
constexpr uint32_t FW_W2 = FW_W1 + 2 * kLboW;
constexpr uint32_t FW_X = FW_W2 + 8 * kLboW;
constexpr uint32_t FW_H1 = FW_X + 2 * kLboRow;
constexpr uint32_t FW_PAR = FW_H1 + 8 * kLboRow;   // b1, b2, w3
constexpr uint32_t FW_BAR = FW_PAR + 3 * kHid * 4;
// 52 KB per CTA keeps at most 4 CTAs on an SM (a fifth would need more than
// the SM's 228 KB of shared memory), and 4 x 128 TMEM columns are the SM's
// 512, so a TMEM allocation never waits for another CTA.  4 CTAs per SM made
// the pruned render's scoring 2% faster than 3.
constexpr uint32_t kFwdSmem = 52 * 1024;
static_assert(FW_BAR + 16 <= kFwdSmem, "forward shared memory");

// TMEM columns of the two layer outputs.
constexpr uint32_t TD1 = 0, TD2 = 64;

// Eight values as one 16-byte chunk of BF16.
__device__ __forceinline__ uint4 pack8(const float* v) {
  return make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                    pack_bf16(v[6], v[7]));
}

// Weights as BF16 B operands (K-major, 16-byte chunks of 8 K elements: one
// store per chunk), biases and w3 in FP32.  w2t < 0: no W2 for dH1.
__device__ void stage_weights(unsigned char* sm, uint32_t w1, uint32_t w2, int w2t,
                              uint32_t par, const float* __restrict__ P) {
  // W1 as B of layer 1: (n = h, k = f), f = 0..15 with zeros from 8 on
  for (int i = threadIdx.x; i < kHid * 2; i += blockDim.x) {
    const int h = i % kHid, kc = i / kHid;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = kc == 0 ? P[OFF_W1 + j * kHid + h] : 0.0f;
    *reinterpret_cast<uint4*>(sm + w1 + tc_off(h, 8 * kc, kLboW)) = pack8(v);
  }
  // W2 as B of layer 2: (n = out, k = in), 8 inputs per chunk (a column of W2,
  // read with consecutive threads on consecutive outputs)
  for (int i = threadIdx.x; i < kHid * 8; i += blockDim.x) {
    const int out = i % kHid, kc = i / kHid;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = P[OFF_W2 + (8 * kc + j) * kHid + out];
    *reinterpret_cast<uint4*>(sm + w2 + tc_off(out, 8 * kc, kLboW)) = pack8(v);
  }
  // W2 as B of dH1 = dH2 W2^T: (n = in, k = out), 8 outputs per chunk (part of a row)
  if (w2t >= 0)
    for (int i = threadIdx.x; i < kHid * 8; i += blockDim.x) {
      const int in = i / 8, kc = i % 8;
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = P[OFF_W2 + in * kHid + 8 * kc + j];
      *reinterpret_cast<uint4*>(sm + (uint32_t)w2t + tc_off(in, 8 * kc, kLboW)) = pack8(v);
    }
  float* q = reinterpret_cast<float*>(sm + par);
  for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
    q[i] = P[OFF_B1 + i];
    q[kHid + i] = P[OFF_B2 + i];
    q[2 * kHid + i] = P[OFF_W3 + i];
  }
}

// Hand the tiles just written to the tensor cores and order the TMEM reads
// before the next MMA: every thread fences, then the block synchronises.
__device__ __forceinline__ void sync_for_mma() {
  fence_smem_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// Row t of a row-wise tile: 16 values (columns c .. c+15) as two 16-byte chunks.
__device__ __forceinline__ void st_row16(unsigned char* base, int t, int c, const float* v) {
  *reinterpret_cast<uint4*>(base + tc_off(t, c, kLboRow)) = pack8(v);
  *reinterpret_cast<uint4*>(base + tc_off(t, c + 8, kLboRow)) = pack8(v + 8);
}

// Wait for the MMAs committed last (block-uniform result); on a timeout the
// caller stops issuing work.
__device__ __forceinline__ bool mma_done(uint64_t* bar, uint32_t& phase) {
  const bool ok = mbar_wait(bar, phase, kWaitCycles);
  phase ^= 1u;
  return __syncthreads_and(ok) != 0;
}

// A CTA's forward-pass state: its shared memory (kFwdSmem bytes at sm), its
// TMEM columns, the mbarrier phase, and whether every MMA so far finished.
struct Fwd {
  unsigned char* sm;
  uint64_t* bar;
  uint32_t tm, phase;
  float b3;
  bool ok;
};

// Stage the network P, allocate 128 TMEM columns and set up the mbarrier.
// All threads of the CTA call it.
__device__ __forceinline__ Fwd fwd_begin(unsigned char* sm, const float* __restrict__ P) {
  Fwd F;
  F.sm = sm;
  F.bar = reinterpret_cast<uint64_t*>(sm + FW_BAR);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + FW_BAR + 8);
  stage_weights(sm, FW_W1, FW_W2, -1, FW_PAR, P);
  F.b3 = P[OFF_B3];
  // the input tile's K padding (features 8..15) stays zero
  *reinterpret_cast<uint4*>(sm + FW_X + tc_off(threadIdx.x, 8, kLboRow)) =
      make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) mbar_init(F.bar, 1);
  if ((threadIdx.x >> 5) == 0) tc_alloc(slot, 128);
  sync_for_mma();
  F.tm = *slot;
  F.phase = 0;
  F.ok = true;
  return F;
}

// The network's output for row threadIdx.x of one tile, whose 8 inputs this
// thread holds in x.  All threads of the CTA call it, once per tile.  If an
// MMA does not finish within the bound, F.ok turns false (for the whole CTA)
// and this and every later call return NaN without issuing work.
__device__ __forceinline__ float fwd_tile(Fwd& F, const float (&x)[8]) {
  if (!F.ok) return __int_as_float(0x7FC00000);
  const int t = threadIdx.x, warp = t >> 5;
  const float* b1 = reinterpret_cast<const float*>(F.sm + FW_PAR);
  const float* b2 = b1 + kHid;
  const float* w3 = b2 + kHid;
  const uint32_t la = F.tm + ((uint32_t)(warp * 32) << 16);
  const uint32_t id64 = tc_idesc_bf16(128, 64);
  const uint32_t aX = smem_u32(F.sm + FW_X), aH1 = smem_u32(F.sm + FW_H1);
  const uint32_t aW1 = smem_u32(F.sm + FW_W1), aW2 = smem_u32(F.sm + FW_W2);
  *reinterpret_cast<uint4*>(F.sm + FW_X + tc_off(t, 0, kLboRow)) = pack8(x);
  sync_for_mma();
  if (t == 0) {
    tc_mma(F.tm + TD1, tc_desc(aX, kLboRow), tc_desc(aW1, kLboW), id64, 0u);
    tc_commit(F.bar);
  }
  F.ok = mma_done(F.bar, F.phase);
  if (!F.ok) return __int_as_float(0x7FC00000);
  tc_fence_after();
#pragma unroll
  for (int c = 0; c < kHid; c += 16) {
    float v[16];
    tc_ld16(la + TD1 + c, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j] + b1[c + j], 0.0f);
    st_row16(F.sm + FW_H1, t, c, v);
  }
  sync_for_mma();
  if (t == 0) {
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
      tc_mma(F.tm + TD2, tc_desc(aH1 + 2 * ks * kLboRow, kLboRow),
             tc_desc(aW2 + 2 * ks * kLboW, kLboW), id64, ks > 0 ? 1u : 0u);
    tc_commit(F.bar);
  }
  F.ok = mma_done(F.bar, F.phase);
  if (!F.ok) return __int_as_float(0x7FC00000);
  tc_fence_after();
  float acc = 0.0f;
#pragma unroll
  for (int c = 0; c < kHid; c += 16) {
    float v[16];
    tc_ld16(la + TD2 + c, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) acc += fmaxf(v[j] + b2[c + j], 0.0f) * w3[c + j];
  }
  tc_fence_before();
  return acc + F.b3;
}

// Free the TMEM columns (after letting a late MMA finish if one timed out).
// All threads of the CTA call it.
__device__ __forceinline__ void fwd_end(Fwd& F) {
  if (!F.ok) mbar_wait(F.bar, F.phase ^ 1u, kWaitCycles);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0) tc_dealloc(F.tm, 128);
}

}  // namespace
