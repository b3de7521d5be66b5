// Learned retarded-time proposal: a 10-64-64-1 perceptron with SiLU activations that predicts, for a
// target and a source, the correction z = log(tau / tau_u) of the delay tau = t - t_r over the delay
// tau_u that the source's uniform motion from its present record gives (the closed-form guess; the
// network learns what the source's acceleration history does to it). The network is evaluated once per
// (group of 512 targets, source) and step on the mixed path (a kernel of its own, before the pair kernel)
// and once per (warp, source) on the FP64 path, at the mean position of the group's or warp's targets
// (which lie close together in the spatial target order), and every pair scales its own uniform-motion
// delay by e^z; the
// retarded-time search then starts from the slot that delay points at and finishes with the same guarded
// search as the closed-form proposal, so the bracket (and every field) is the one of the paper's search
// whatever the network predicts.
//
// Tensor-core arithmetic: mma.sync m16n8k16 with BF16 operands and FP32 accumulation, one warp per 16
// (or 32) rows. Hidden layers are chained from the accumulator layout of one GEMM to the operand
// layout of the next without data movement.
//
// Two forms of the forward pass:
//   reference form (forward_tile; training and emppp_mlp_forward mode 0): FP32 SiLU of each hidden
//     value, BF16 rounding of the GEMM operands only, FP32 output layer;
//   inference form (infer_warp; the pair kernels and emppp_mlp_forward mode 1): weights and biases of
//     the hidden layers pre-scaled by 1/2 so that the accumulator holds h = x / 2, SiLU evaluated on
//     packed BF16 pairs as h + h tanh(h) (one tanh.approx.bf16x2 and one fma.rn.bf16x2 per two values),
//     and the output layer as one more tensor-core product against w3, so that each hidden value
//     costs about one and a half instructions. Its z differs from the reference form by BF16 rounding
//     of the activations (a few 1e-3), which only moves the starting slot of the guarded search.
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

// Inference image (the pair kernels' form), lane-major B fragments so that a warp's fragment load is
// one contiguous 256-byte row:
//   w1[nt][lane]      B fragment of W1 / 2 for hidden units 8 nt .. 8 nt + 7
//   w2[nt][kk][lane]  B fragment of W2 / 2, output units 8 nt .., input units 16 kk ..
//   b1[nt][t], b2[nt][t]  halved biases of units 8 nt + 2t, 8 nt + 2t + 1
//   w3[kk][t]         B fragment of the output layer (w3 in every column), input units 16 kk ..
struct __align__(16) InferImage {
  uint2 w1[kH / 8][32];
  uint2 w2[kH / 8][kH / 16][32];
  float2 b1[kH / 8][4];
  float2 b2[kH / 8][4];
  uint2 w3[kH / 16][4];
  float b3;
  float pad_[3];
};

// the device image of a network: NetImage (training, reference form) followed by InferImage
constexpr size_t kImageBytes = sizeof(NetImage) + sizeof(InferImage);
static_assert(sizeof(NetImage) % 16 == 0, "InferImage must start 16-byte aligned");
__host__ __device__ inline const InferImage* infer_image(const void* image) {
  return reinterpret_cast<const InferImage*>(static_cast<const char*>(image) + sizeof(NetImage));
}

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
// inference form: silu(x) = h + h tanh(h) with h = x / 2, on two packed BF16 values
__device__ __forceinline__ uint32_t silu_half_bf16x2(float h_lo, float h_hi) {
  const uint32_t h = pack_bf16x2(h_lo, h_hi);
  uint32_t th, r;
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(th) : "r"(h));
  asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(h), "r"(th), "r"(h));
  return r;
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
    for (int k = 0; k < 8; k++) h[k] = silu(h[k]);
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
    zg += silu(h0) * w0 + silu(h1) * w1;
    zg8 += silu(h2) * w0 + silu(h3) * w1;
  }
  zg += __shfl_xor_sync(0xffffffffu, zg, 1);
  zg += __shfl_xor_sync(0xffffffffu, zg, 2);
  zg8 += __shfl_xor_sync(0xffffffffu, zg8, 1);
  zg8 += __shfl_xor_sync(0xffffffffu, zg8, 2);
  z_g = zg + net.b3;
  z_g8 = zg8 + net.b3;
}

// Copies an image (NetImage or InferImage) from global memory into shared memory (whole block, then a
// barrier). Both addresses are 16-byte aligned: the images are declared with that alignment and the
// global image comes from cudaMalloc (InferImage at a multiple of 16 bytes after it).
template <class Image>
__device__ __forceinline__ void load_image(Image& dst, const Image* __restrict__ src) {
  static_assert(sizeof(Image) % 16 == 0, "image size must be a multiple of 16 bytes");
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(&dst);
  for (int k = threadIdx.x; k < (int)(sizeof(Image) / 16); k += blockDim.x) d[k] = s[k];
  __syncthreads();
}

// Inference form of the forward pass for the 32 rows held one per lane: f are this lane's features;
// returns z of this lane's row. The A fragments of the two 16-row input tiles are gathered from the
// lanes that hold the rows by warp shuffles (no shared memory): lane (g, t) takes feature pair t of rows
// g and g + 8 (words 0..3 of those lanes) and pair 4 + t (word 4 for t = 0; the padding is zero). Every
// lane of the warp must call it (converged). Both 16-row tiles share each B-fragment load.
__device__ __forceinline__ float infer_warp(const InferImage& net, const float f[kIn]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t w[5] = {pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]), pack_bf16x2(f[4], f[5]),
                         pack_bf16x2(f[6], f[7]), pack_bf16x2(f[8], f[9])};
  uint32_t a_in[2][4];
#pragma unroll
  for (int m = 0; m < 2; m++) {
    const int r0 = 16 * m + g, r1 = r0 + 8;
    uint32_t lo0 = 0u, lo1 = 0u;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint32_t v0 = __shfl_sync(0xffffffffu, w[q], r0), v1 = __shfl_sync(0xffffffffu, w[q], r1);
      lo0 = (t == q) ? v0 : lo0;
      lo1 = (t == q) ? v1 : lo1;
    }
    const uint32_t h0 = __shfl_sync(0xffffffffu, w[4], r0), h1 = __shfl_sync(0xffffffffu, w[4], r1);
    a_in[m][0] = lo0;
    a_in[m][1] = lo1;
    a_in[m][2] = t == 0 ? h0 : 0u;
    a_in[m][3] = t == 0 ? h1 : 0u;
  }
  // layer 1: accumulators start at b1 / 2, activations packed straight into layer 2's A fragments
  uint32_t a1[2][4][4];
#pragma unroll
  for (int nt = 0; nt < kH / 8; nt++) {
    const uint2 bw = net.w1[nt][lane];
    const float2 bb = net.b1[nt][t];
#pragma unroll
    for (int m = 0; m < 2; m++) {
      float c[4] = {bb.x, bb.y, bb.x, bb.y};
      mma_bf16(c, a_in[m], bw.x, bw.y);
      const int kk = nt >> 1, o = (nt & 1) * 2;
      a1[m][kk][o] = silu_half_bf16x2(c[0], c[1]);
      a1[m][kk][o + 1] = silu_half_bf16x2(c[2], c[3]);
    }
  }
  // layer 2, two n-tiles at a time = one k-step of the output layer
  float zo[2][4];
#pragma unroll
  for (int m = 0; m < 2; m++) zo[m][0] = zo[m][1] = zo[m][2] = zo[m][3] = net.b3;
#pragma unroll
  for (int ko = 0; ko < kH / 16; ko++) {
    uint32_t ao[2][4];
#pragma unroll
    for (int half = 0; half < 2; half++) {
      const int nt = 2 * ko + half;
      const float2 bb = net.b2[nt][t];
      float c[2][4] = {{bb.x, bb.y, bb.x, bb.y}, {bb.x, bb.y, bb.x, bb.y}};
#pragma unroll
      for (int kk = 0; kk < kH / 16; kk++) {
        const uint2 bw = net.w2[nt][kk][lane];
        mma_bf16(c[0], a1[0][kk], bw.x, bw.y);
        mma_bf16(c[1], a1[1][kk], bw.x, bw.y);
      }
#pragma unroll
      for (int m = 0; m < 2; m++) {
        ao[m][2 * half] = silu_half_bf16x2(c[m][0], c[m][1]);
        ao[m][2 * half + 1] = silu_half_bf16x2(c[m][2], c[m][3]);
      }
    }
    const uint2 w3 = net.w3[ko][t];
    mma_bf16(zo[0], ao[0], w3.x, w3.y);
    mma_bf16(zo[1], ao[1], w3.x, w3.y);
  }
  // every column of the output holds z: lane (g, t) has rows g (zo[m][0]) and g + 8 (zo[m][2]) of tile m
  const int m = lane >> 4, local = lane & 15, src = (local & 7) * 4;
  const float v00 = __shfl_sync(0xffffffffu, zo[0][0], src), v01 = __shfl_sync(0xffffffffu, zo[0][2], src);
  const float v10 = __shfl_sync(0xffffffffu, zo[1][0], src), v11 = __shfl_sync(0xffffffffu, zo[1][2], src);
  return m == 0 ? (local < 8 ? v00 : v01) : (local < 8 ? v10 : v11);
}

// Mean of (x0, x1, x2) over the active lanes of the warp (the origin if none is active). Every lane of
// the warp must call it.
__device__ __forceinline__ float3 warp_mean(bool active, float x0, float x1, float x2) {
  float s0 = active ? x0 : 0.f, s1 = active ? x1 : 0.f, s2 = active ? x2 : 0.f;
  float cnt = active ? 1.f : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  const float ic = cnt > 0.f ? 1.f / cnt : 0.f;
  return make_float3(s0 * ic, s1 * ic, s2 * ic);
}

// Delay factor e^z of one source per lane (the warp evaluates up to 32 sources at once): d = r_c - w_n
// from the warp's mean target position r_c to the source's present position, beta_n and
// beta_n - beta_{n-1} of the source. Lanes without a source (valid false) take part in the tensor-core
// pass with zero features and return 1. z is clamped to [-20, 20] (a factor the search absorbs anyway).
// Every lane of the warp must call it (converged).
__device__ __forceinline__ float warp_delay_factor(const InferImage& net, bool valid, float d0, float d1, float d2,
                                                   float b0, float b1, float b2, float db0, float db1, float db2,
                                                   float invL, float Df) {
  float f[kIn];
  if (valid) {
    features(d0, d1, d2, b0, b1, b2, db0, db1, db2, invL, Df, f);
  } else {
#pragma unroll
    for (int k = 0; k < kIn; k++) f[k] = 0.f;
  }
  const float z = infer_warp(net, f);
  return valid ? __expf(fminf(fmaxf(z, -20.f), 20.f)) : 1.f;
}

}  // namespace mlp
}  // namespace emppp
