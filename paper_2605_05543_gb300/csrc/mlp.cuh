// Learned retarded-time proposal: a 10-64-64-1 perceptron with SiLU activations that predicts, for a
// target and a source, z = log(c (t - t_r) / |d|) with d = r - w_n the present separation. The
// retarded-time search then starts from the slot the predicted delay points at and finishes with the
// same guarded search as the closed-form proposal, so the bracket (and every field) is the one of the
// paper's search whatever the network predicts.
//
// Tensor-core arithmetic: mma.sync m16n8k16 with BF16 operands and FP32 accumulation, one warp per 16
// (or 32) rows. Hidden layers are chained from the accumulator layout of one GEMM to the operand
// layout of the next without data movement.
#pragma once

#include <stdint.h>

#include "emppp_internal.cuh"

namespace emppp {
namespace mlp {

constexpr int kIn = 10;     // features
constexpr int kInPad = 16;  // padded to one k-step
constexpr int kH = 64;      // hidden width

// flat FP32 parameter vector: W1[f][h], b1[h], W2[i][o], b2[o], w3[o], b3
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kIn * kH;
constexpr int kOffW2 = kOffB1 + kH;
constexpr int kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH;
constexpr int kOffB3 = kOffW3 + kH;
constexpr int kNumParams = kOffB3 + 1;  // 4929

// Network image for the tensor-core passes (BF16 pairs packed in uint32, k contiguous per column):
//   w1f[n][k/2]: layer-1 weights as the B operand (n = hidden unit, k = feature)
//   w2f[n][k/2]: layer-2 weights as the B operand (n = output unit, k = input unit)
//   w2b[n][k/2]: layer-2 weights transposed, the B operand of the input-gradient pass
struct __align__(16) NetImage {  // copied with 16-byte vector loads and stores
  uint32_t w1f[kH][kInPad / 2];
  uint32_t w2f[kH][kH / 2];
  uint32_t w2b[kH][kH / 2];
  float b1[kH], b2[kH], w3[kH];
  float b3;
  float pad_[3];
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ float bf16_round(float x) {
  uint32_t p = pack_bf16x2(x, 0.f);
  return __uint_as_float(p << 16);
}

// D = A (16x16, row) * B (16x8, col) + C, BF16 operands, FP32 accumulate
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float sigmoid(float x) { return 1.f / (1.f + __expf(-x)); }
__device__ __forceinline__ float silu(float x) { return x * sigmoid(x); }
__device__ __forceinline__ float dsilu(float x) {
  const float s = sigmoid(x);
  return s * (1.f + x * (1.f - s));
}
// inference form: silu(x) = x (1 + tanh(x / 2)) / 2 with the hardware tanh approximation
__device__ __forceinline__ float silu_fast(float x) {
  float th;
  asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(0.5f * x));
  return 0.5f * x * (1.f + th);
}

// Features of a (target, source) pair: the direction d / |d| of d = r - w_n (3), |d| / L with
// L = c dt D (1), beta_n (3), (beta_n - beta_{n-1}) D (3), with dt the step, D the history depth, w_n,
// beta_n the source's present position and velocity and beta_{n-1} its velocity one slot earlier. For
// uniform motion the target depends on d / |d| and beta_n alone (through d.beta / |d| and |beta|), so the
// direction is given as such rather than as a ratio the network would have to form.
__device__ __forceinline__ void features(float d0, float d1, float d2, float b0, float b1, float b2, float db0,
                                         float db1, float db2, float invL, float Df, float f[kIn]) {
  const float dd = fmaxf(d0 * d0 + d1 * d1 + d2 * d2, 1e-37f);
  const float inv = rsqrtf(dd);
  f[0] = d0 * inv;
  f[1] = d1 * inv;
  f[2] = d2 * inv;
  f[3] = dd * inv * invL;
  f[4] = b0;
  f[5] = b1;
  f[6] = b2;
  f[7] = db0 * Df;
  f[8] = db1 * Df;
  f[9] = db2 * Df;
}

// Forward pass of one 16-row tile held by a warp: a_in is the A fragment of the padded 16 x 16 input
// tile (rows g and g + 8 of lane (g, t)); returns z of rows g and g + 8 (all four lanes of a quad).
template <bool FAST>
__device__ __forceinline__ void forward_tile(const NetImage& net, const uint32_t a_in[4], float& z_g, float& z_g8) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t a1[4][4];
#pragma unroll
  for (int nt = 0; nt < 8; nt += 2) {
    float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
    mma_bf16(c0, a_in, net.w1f[8 * nt + g][t], net.w1f[8 * nt + g][4 + t]);
    mma_bf16(c1, a_in, net.w1f[8 * (nt + 1) + g][t], net.w1f[8 * (nt + 1) + g][4 + t]);
    const float ba = net.b1[8 * nt + 2 * t], bb = net.b1[8 * nt + 2 * t + 1];
    const float bc = net.b1[8 * (nt + 1) + 2 * t], bd = net.b1[8 * (nt + 1) + 2 * t + 1];
    float h[8] = {c0[0] + ba, c0[1] + bb, c0[2] + ba, c0[3] + bb, c1[0] + bc, c1[1] + bd, c1[2] + bc, c1[3] + bd};
#pragma unroll
    for (int k = 0; k < 8; k++) h[k] = FAST ? silu_fast(h[k]) : silu(h[k]);
    const int kk = nt >> 1;
    a1[kk][0] = pack_bf16x2(h[0], h[1]);
    a1[kk][1] = pack_bf16x2(h[2], h[3]);
    a1[kk][2] = pack_bf16x2(h[4], h[5]);
    a1[kk][3] = pack_bf16x2(h[6], h[7]);
  }
  float zg = 0.f, zg8 = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; nt++) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 4; kk++) mma_bf16(c, a1[kk], net.w2f[8 * nt + g][8 * kk + t], net.w2f[8 * nt + g][8 * kk + 4 + t]);
    const int o = 8 * nt + 2 * t;
    const float h0 = c[0] + net.b2[o], h1 = c[1] + net.b2[o + 1], h2 = c[2] + net.b2[o], h3 = c[3] + net.b2[o + 1];
    const float w0 = net.w3[o], w1 = net.w3[o + 1];
    if (FAST) {
      zg += silu_fast(h0) * w0 + silu_fast(h1) * w1;
      zg8 += silu_fast(h2) * w0 + silu_fast(h3) * w1;
    } else {
      zg += silu(h0) * w0 + silu(h1) * w1;
      zg8 += silu(h2) * w0 + silu(h3) * w1;
    }
  }
  zg += __shfl_xor_sync(0xffffffffu, zg, 1);
  zg += __shfl_xor_sync(0xffffffffu, zg, 2);
  zg8 += __shfl_xor_sync(0xffffffffu, zg8, 1);
  zg8 += __shfl_xor_sync(0xffffffffu, zg8, 2);
  z_g = zg + net.b3;
  z_g8 = zg8 + net.b3;
}

// Copies the network image from global memory into shared memory (whole block, then a barrier). Both
// addresses are 16-byte aligned: NetImage is declared with that alignment and the global image comes
// from cudaMalloc.
__device__ __forceinline__ void load_image(NetImage& dst, const NetImage* __restrict__ src) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(&dst);
  for (int k = threadIdx.x; k < (int)(sizeof(NetImage) / 16); k += blockDim.x) d[k] = s[k];
  __syncthreads();
}

// Warp-wide inference for the 32 rows held one per lane: f are this lane's features, stage is a per-warp
// shared buffer of 32 x 8 uint32; returns z of this lane's row. Every lane of the warp must call it.
__device__ __forceinline__ float infer_warp(const NetImage& net, const float f[kIn], uint32_t (*stage)[8]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  stage[lane][0] = pack_bf16x2(f[0], f[1]);
  stage[lane][1] = pack_bf16x2(f[2], f[3]);
  stage[lane][2] = pack_bf16x2(f[4], f[5]);
  stage[lane][3] = pack_bf16x2(f[6], f[7]);
  stage[lane][4] = pack_bf16x2(f[8], f[9]);
  stage[lane][5] = 0u;
  stage[lane][6] = 0u;
  stage[lane][7] = 0u;
  __syncwarp();
  float z[2][2];
#pragma unroll
  for (int m = 0; m < 2; m++) {
    const uint32_t a[4] = {stage[16 * m + g][t], stage[16 * m + g + 8][t], stage[16 * m + g][4 + t],
                           stage[16 * m + g + 8][4 + t]};
    forward_tile<true>(net, a, z[m][0], z[m][1]);
  }
  __syncwarp();
  const int m = lane >> 4, local = lane & 15, src = (local & 7) * 4;
  const float v00 = __shfl_sync(0xffffffffu, z[0][0], src), v01 = __shfl_sync(0xffffffffu, z[0][1], src);
  const float v10 = __shfl_sync(0xffffffffu, z[1][0], src), v11 = __shfl_sync(0xffffffffu, z[1][1], src);
  return m == 0 ? (local < 8 ? v00 : v01) : (local < 8 ? v10 : v11);
}

}  // namespace mlp
}  // namespace emppp
