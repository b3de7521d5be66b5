// Learned retarded-time proposal: training data from the method itself, and the network's training.
//
//   sample_kernel  for given (target, source) pairs at the present state: the 10 features (mlp.cuh)
//                  and the exact retarded delay t - t_r from the FP64 bracket of Sec. 2.2 (the paper's
//                  search) and the smaller root of eq:dt; the training target is
//                  z = log((t - t_r) / tau_u), tau_u the delay of the source's uniform motion from its
//                  present record.
//   train_kernel   one pass over a batch: forward on the tensor cores (BF16 operands, FP32 accumulate),
//                  the mean squared error of z, the input gradients of layer 2 on the tensor cores
//                  (dA1 = dH2 W2^T), the weight gradients reduced in FP32 per warp and summed into a
//                  global gradient vector.
//   adam_kernel    Adam on the FP32 master parameters; the BF16 network image is rebuilt from them.
//
// Rounding points (also followed by the CPU reference in oracle/mlp.py): the GEMM operands X, W1, A1 =
// silu(H1), W2 (forward) and dH2, W2 (input gradient) are rounded to BF16; products accumulate in FP32;
// biases, activations, w3 and every weight gradient are FP32.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/emppp.h"
#include "emppp_internal.cuh"
#include "mlp.cuh"

namespace emppp {
void set_error_text(const char* msg);
}

using namespace emppp;
using namespace emppp::mlp;

namespace {

constexpr int kWarps = 4;  // warps per training block

// ---------------------------------------------------------------------------------------------
// network image
// ---------------------------------------------------------------------------------------------
__global__ void build_image_kernel(const float* __restrict__ p, void* __restrict__ image) {
  NetImage* __restrict__ img = static_cast<NetImage*>(image);
  InferImage* __restrict__ inf = reinterpret_cast<InferImage*>(static_cast<char*>(image) + sizeof(NetImage));
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  // inference image: halved hidden layers, lane-major B fragments (mlp.cuh)
  auto w1h = [&](int f, int n) { return f < kIn ? 0.5f * p[kOffW1 + f * kH + n] : 0.f; };
  auto w2h = [&](int i, int o) { return 0.5f * p[kOffW2 + i * kH + o]; };
  if (k < (kH / 8) * 32) {
    const int nt = k / 32, lane = k % 32, g = lane >> 2, t = lane & 3, n = 8 * nt + g;
    inf->w1[nt][lane] = make_uint2(pack_bf16x2(w1h(2 * t, n), w1h(2 * t + 1, n)),
                                   pack_bf16x2(w1h(2 * t + 8, n), w1h(2 * t + 9, n)));
  }
  if (k < (kH / 8) * (kH / 16) * 32) {
    const int nt = k / 128, kk = (k / 32) % 4, lane = k % 32, g = lane >> 2, t = lane & 3;
    const int n = 8 * nt + g, ki = 16 * kk + 2 * t;
    inf->w2[nt][kk][lane] = make_uint2(pack_bf16x2(w2h(ki, n), w2h(ki + 1, n)), pack_bf16x2(w2h(ki + 8, n), w2h(ki + 9, n)));
  }
  if (k < (kH / 8) * 4) {
    const int nt = k / 4, t = k % 4, o = 8 * nt + 2 * t;
    inf->b1[nt][t] = make_float2(0.5f * p[kOffB1 + o], 0.5f * p[kOffB1 + o + 1]);
    inf->b2[nt][t] = make_float2(0.5f * p[kOffB2 + o], 0.5f * p[kOffB2 + o + 1]);
  }
  if (k < (kH / 16) * 4) {
    const int ko = k / 4, t = k % 4, i = 16 * ko + 2 * t;
    inf->w3[ko][t] = make_uint2(pack_bf16x2(p[kOffW3 + i], p[kOffW3 + i + 1]), pack_bf16x2(p[kOffW3 + i + 8], p[kOffW3 + i + 9]));
  }
  if (k == 0) {
    inf->b3 = p[kOffB3];
    inf->pad_[0] = inf->pad_[1] = inf->pad_[2] = 0.f;
  }
  // reference image
  if (k < kH * (kInPad / 2)) {
    const int n = k / (kInPad / 2), kp = k % (kInPad / 2);
    const int f0 = 2 * kp, f1 = 2 * kp + 1;
    const float a = f0 < kIn ? p[kOffW1 + f0 * kH + n] : 0.f;
    const float b = f1 < kIn ? p[kOffW1 + f1 * kH + n] : 0.f;
    img->w1f[n][kp] = pack_bf16x2(a, b);
  }
  if (k < kH * (kH / 2)) {
    const int n = k / (kH / 2), kp = k % (kH / 2);
    // forward: B(k = in, n = out) = W2[in][out]
    img->w2f[n][kp] = pack_bf16x2(p[kOffW2 + (2 * kp) * kH + n], p[kOffW2 + (2 * kp + 1) * kH + n]);
    // input gradient: B(k = out, n = in) = W2[in][out]
    img->w2b[n][kp] = pack_bf16x2(p[kOffW2 + n * kH + 2 * kp], p[kOffW2 + n * kH + 2 * kp + 1]);
  }
  if (k < kH) {
    img->b1[k] = p[kOffB1 + k];
    img->b2[k] = p[kOffB2 + k];
    img->w3[k] = p[kOffW3 + k];
  }
  if (k == 0) {
    img->b3 = p[kOffB3];
    img->pad_[0] = img->pad_[1] = img->pad_[2] = 0.f;
  }
}

// ---------------------------------------------------------------------------------------------
// training data: features and exact FP64 delays of given pairs at the present state
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ bool node_test64(double r0, double r1, double r2, const double* __restrict__ w,
                                            double lhs) {
  const double d0 = __dsub_rn(r0, w[0]);
  const double d1 = __dsub_rn(r1, w[1]);
  const double d2 = __dsub_rn(r2, w[2]);
  const double rhs = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
  return lhs <= rhs;
}

__global__ void sample_kernel(DeviceState s, const int* __restrict__ pairs, long long m, float* __restrict__ feat,
                              double* __restrict__ delay, float* __restrict__ zt) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  const StepState st = *s.state;
  const int D = s.D;
  const long long i = pairs[2 * q], j = pairs[2 * q + 1];
  const double t = st.t;
  const double* ri = s.rec64 + ((size_t)i * D + st.pn) * 6;
  const double r0 = ri[0], r1 = ri[1], r2 = ri[2];
  const double* src = s.rec64 + (size_t)j * D * 6;
  auto phys = [&](long long k) {
    int p = st.p0 + (int)(k - st.k0);
    return p >= D ? p - D : p;
  };
  // the paper's search (Sec. 2.2)
  long long k1;
  if (node_test64(r0, r1, r2, src + 6 * st.p0, s.tab.lhs64[st.p0])) {
    k1 = st.k0;  // out of history: eq:linear2 from the oldest slot
  } else if (!node_test64(r0, r1, r2, src + 6 * phys(st.n - 1), s.tab.lhs64[phys(st.n - 1)])) {
    k1 = st.n - 1;
  } else {
    long long lo = st.k0, hi = st.n;
    while (hi - lo > 1) {
      const long long mid = (lo + hi) >> 1;
      if (node_test64(r0, r1, r2, src + 6 * phys(mid), s.tab.lhs64[phys(mid)]))
        hi = mid;
      else
        lo = mid;
    }
    k1 = lo;
  }
  const int p1 = phys(k1);
  const double* w1 = src + 6 * p1;
  const double T1 = t - s.slot_t[p1];
  const double c2 = kC * kC;
  const double d0 = r0 - w1[0], d1 = r1 - w1[1], d2 = r2 - w1[2];
  const double C2 = c2 - (w1[3] * w1[3] + w1[4] * w1[4] + w1[5] * w1[5]);
  const double hb = (d0 * w1[3] + d1 * w1[4] + d2 * w1[5]) - c2 * T1;
  const double C0 = c2 * T1 * T1 - (d0 * d0 + d1 * d1 + d2 * d2);
  const double qd = hb * hb - C2 * C0;
  double tau = __longlong_as_double(0x7ff8000000000000LL);
  if (C2 > 0.0 && qd >= 0.0) {
    const double sq = sqrt(qd);
    const double dtr = (hb <= 0.0) ? C0 / (sq - hb) : -(hb + sq) / C2;
    tau = T1 - dtr;  // t - t_r
  }
  // features from the present records
  const double* wn = src + 6 * st.pn;
  const double* vp = (st.n > st.k0) ? src + 6 * phys(st.n - 1) : wn;
  const double e0 = r0 - wn[0], e1 = r1 - wn[1], e2 = r2 - wn[2];
  const double ic = 1.0 / kC;
  const float invL = (float)(1.0 / (kC * st.dt * D));
  float f[kIn];
  features((float)e0, (float)e1, (float)e2, (float)(wn[3] * ic), (float)(wn[4] * ic), (float)(wn[5] * ic),
           (float)((wn[3] - vp[3]) * ic), (float)((wn[4] - vp[4]) * ic), (float)((wn[5] - vp[5]) * ic), invL,
           (float)D, f);
  for (int k = 0; k < kIn; k++) feat[q * kIn + k] = f[k];
  delay[q] = tau;
  // uniform-motion delay from the present record: c tau_u = [d.beta + sqrt((d.beta)^2 + (1 - beta^2) |d|^2)] /
  // (1 - beta^2), d = r - w_n, formed as |d|^2 / (sqrt(...) - d.beta) when d.beta < 0 (no cancellation)
  const double b0 = wn[3] * ic, b1 = wn[4] * ic, b2 = wn[5] * ic;
  const double ig2 = 1.0 - (b0 * b0 + b1 * b1 + b2 * b2);
  const double db = e0 * b0 + e1 * b1 + e2 * b2, dd = e0 * e0 + e1 * e1 + e2 * e2;
  const double sq = sqrt(db * db + ig2 * dd);
  const double ctau_u = db >= 0.0 ? (db + sq) / ig2 : dd / (sq - db);
  zt[q] = (float)log(kC * tau / ctau_u);
}

// ---------------------------------------------------------------------------------------------
// forward pass of many rows (tests and evaluation)
// ---------------------------------------------------------------------------------------------
// the reference form (training's forward pass)
__global__ void forward_kernel(const NetImage* __restrict__ img, const float* __restrict__ X, long long m,
                               float* __restrict__ z) {
  __shared__ NetImage net;
  load_image(net, img);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long tile = warp; tile * 16 < m; tile += nwarps) {
    const long long r0 = tile * 16 + g, r1 = r0 + 8;
    auto feat = [&](long long r, int k) { return (r < m && k < kIn) ? X[r * kIn + k] : 0.f; };
    const uint32_t a[4] = {pack_bf16x2(feat(r0, 2 * t), feat(r0, 2 * t + 1)), pack_bf16x2(feat(r1, 2 * t), feat(r1, 2 * t + 1)),
                           pack_bf16x2(feat(r0, 2 * t + 8), feat(r0, 2 * t + 9)),
                           pack_bf16x2(feat(r1, 2 * t + 8), feat(r1, 2 * t + 9))};
    float zg, zg8;
    forward_tile(net, a, zg, zg8);
    if (t == 0) {
      if (r0 < m) z[r0] = zg;
      if (r1 < m) z[r1] = zg8;
    }
  }
}

// the inference form, exactly as the pair kernels evaluate it: one row per lane, 32 rows per warp
__global__ void forward_infer_kernel(const InferImage* __restrict__ img, const float* __restrict__ X, long long m,
                                     float* __restrict__ z) {
  __shared__ InferImage net;
  load_image(net, img);
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp * 32; base < m; base += nwarps * 32) {
    const long long r = base + lane;
    float f[kIn];
#pragma unroll
    for (int k = 0; k < kIn; k++) f[k] = r < m ? X[r * kIn + k] : 0.f;
    const float zr = infer_warp(net, f);
    if (r < m) z[r] = zr;
  }
}

// ---------------------------------------------------------------------------------------------
// training
// ---------------------------------------------------------------------------------------------
struct TrainSmem {
  NetImage net;
  // per warp: one 16-row tile staged in FP32, and the warp's gradient accumulators
  float X[kWarps][16][kInPad];
  float A1[kWarps][16][kH];
  float dH1[kWarps][16][kH];
  float A2[kWarps][16][kH];
  float dH2[kWarps][16][kH];
  float dz[kWarps][16];
  float g[kWarps][kNumParams];
};

// rows [row0, row0 + rows) of X [m][10] and T [m]; gradient of sum_r (z_r - T_r)^2 / norm
__global__ void __launch_bounds__(kWarps * 32) train_kernel(const NetImage* __restrict__ img,
                                                             const float* __restrict__ X, const float* __restrict__ T,
                                                             long long row0, long long rows, float norm,
                                                             float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  load_image(S.net, img);
  const NetImage& net = S.net;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
  float* gw = S.g[w];
  for (int k = lane; k < kNumParams; k += 32) gw[k] = 0.f;
  float loss_acc = 0.f;
  const long long warp = (long long)blockIdx.x * kWarps + w;
  const long long nwarps = (long long)gridDim.x * kWarps;
  for (long long tile = warp; tile * 16 < rows; tile += nwarps) {
    const long long base = row0 + tile * 16;
    const long long ra = base + g, rb = ra + 8;
    const bool va = ra < row0 + rows, vb = rb < row0 + rows;
    auto feat = [&](long long r, bool v, int k) { return (v && k < kIn) ? X[r * kIn + k] : 0.f; };
    // stage the input tile (FP32, BF16-rounded as the GEMM sees it)
    for (int k = 2 * t; k < 2 * t + 2; k++) {
      S.X[w][g][k] = bf16_round(feat(ra, va, k));
      S.X[w][g][k + 8] = bf16_round(feat(ra, va, k + 8));
      S.X[w][g + 8][k] = bf16_round(feat(rb, vb, k));
      S.X[w][g + 8][k + 8] = bf16_round(feat(rb, vb, k + 8));
    }
    const uint32_t a_in[4] = {pack_bf16x2(feat(ra, va, 2 * t), feat(ra, va, 2 * t + 1)),
                              pack_bf16x2(feat(rb, vb, 2 * t), feat(rb, vb, 2 * t + 1)),
                              pack_bf16x2(feat(ra, va, 2 * t + 8), feat(ra, va, 2 * t + 9)),
                              pack_bf16x2(feat(rb, vb, 2 * t + 8), feat(rb, vb, 2 * t + 9))};
    // layer 1
    float h1[8][4];
    uint32_t a1[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16(c, a_in, net.w1f[8 * nt + g][t], net.w1f[8 * nt + g][4 + t]);
      const int o = 8 * nt + 2 * t;
      h1[nt][0] = c[0] + net.b1[o];
      h1[nt][1] = c[1] + net.b1[o + 1];
      h1[nt][2] = c[2] + net.b1[o];
      h1[nt][3] = c[3] + net.b1[o + 1];
      const float s0 = silu(h1[nt][0]), s1 = silu(h1[nt][1]), s2 = silu(h1[nt][2]), s3 = silu(h1[nt][3]);
      S.A1[w][g][o] = s0;
      S.A1[w][g][o + 1] = s1;
      S.A1[w][g + 8][o] = s2;
      S.A1[w][g + 8][o + 1] = s3;
      const int kk = nt >> 1;
      if ((nt & 1) == 0) {
        a1[kk][0] = pack_bf16x2(s0, s1);
        a1[kk][1] = pack_bf16x2(s2, s3);
      } else {
        a1[kk][2] = pack_bf16x2(s0, s1);
        a1[kk][3] = pack_bf16x2(s2, s3);
      }
    }
    // layer 2 and output
    float h2[8][4];
    float zg = 0.f, zg8 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kk = 0; kk < 4; kk++) mma_bf16(c, a1[kk], net.w2f[8 * nt + g][8 * kk + t], net.w2f[8 * nt + g][8 * kk + 4 + t]);
      const int o = 8 * nt + 2 * t;
      h2[nt][0] = c[0] + net.b2[o];
      h2[nt][1] = c[1] + net.b2[o + 1];
      h2[nt][2] = c[2] + net.b2[o];
      h2[nt][3] = c[3] + net.b2[o + 1];
      const float s0 = silu(h2[nt][0]), s1 = silu(h2[nt][1]), s2 = silu(h2[nt][2]), s3 = silu(h2[nt][3]);
      S.A2[w][g][o] = s0;
      S.A2[w][g][o + 1] = s1;
      S.A2[w][g + 8][o] = s2;
      S.A2[w][g + 8][o + 1] = s3;
      zg += s0 * net.w3[o] + s1 * net.w3[o + 1];
      zg8 += s2 * net.w3[o] + s3 * net.w3[o + 1];
    }
    zg += __shfl_xor_sync(0xffffffffu, zg, 1);
    zg += __shfl_xor_sync(0xffffffffu, zg, 2);
    zg8 += __shfl_xor_sync(0xffffffffu, zg8, 1);
    zg8 += __shfl_xor_sync(0xffffffffu, zg8, 2);
    zg += net.b3;
    zg8 += net.b3;
    const float ea = va ? zg - T[ra] : 0.f, eb = vb ? zg8 - T[rb] : 0.f;
    if (t == 0) loss_acc += ea * ea + eb * eb;
    const float dza = 2.f * ea / norm, dzb = 2.f * eb / norm;
    if (t == 0) {
      S.dz[w][g] = dza;
      S.dz[w][g + 8] = dzb;
    }
    // dH2 = dz w3 silu'(H2); the input gradient of layer 2 on the tensor cores
    uint32_t ad[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
      const int o = 8 * nt + 2 * t;
      const float q0 = dza * net.w3[o] * dsilu(h2[nt][0]);
      const float q1 = dza * net.w3[o + 1] * dsilu(h2[nt][1]);
      const float q2 = dzb * net.w3[o] * dsilu(h2[nt][2]);
      const float q3 = dzb * net.w3[o + 1] * dsilu(h2[nt][3]);
      S.dH2[w][g][o] = q0;
      S.dH2[w][g][o + 1] = q1;
      S.dH2[w][g + 8][o] = q2;
      S.dH2[w][g + 8][o + 1] = q3;
      const int kk = nt >> 1;
      if ((nt & 1) == 0) {
        ad[kk][0] = pack_bf16x2(q0, q1);
        ad[kk][1] = pack_bf16x2(q2, q3);
      } else {
        ad[kk][2] = pack_bf16x2(q0, q1);
        ad[kk][3] = pack_bf16x2(q2, q3);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kk = 0; kk < 4; kk++) mma_bf16(c, ad[kk], net.w2b[8 * nt + g][8 * kk + t], net.w2b[8 * nt + g][8 * kk + 4 + t]);
      const int o = 8 * nt + 2 * t;
      S.dH1[w][g][o] = c[0] * dsilu(h1[nt][0]);
      S.dH1[w][g][o + 1] = c[1] * dsilu(h1[nt][1]);
      S.dH1[w][g + 8][o] = c[2] * dsilu(h1[nt][2]);
      S.dH1[w][g + 8][o + 1] = c[3] * dsilu(h1[nt][3]);
    }
    __syncwarp();
    // weight gradients of this tile, FP32: lane owns hidden units 2 lane and 2 lane + 1
#pragma unroll
    for (int s2 = 0; s2 < 2; s2++) {
      const int u = 2 * lane + s2;
      float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f;
      float gW1[kIn];
#pragma unroll
      for (int f = 0; f < kIn; f++) gW1[f] = 0.f;
      for (int r = 0; r < 16; r++) {
        const float dh1 = S.dH1[w][r][u];
        gb1 += dh1;
#pragma unroll
        for (int f = 0; f < kIn; f++) gW1[f] += S.X[w][r][f] * dh1;
        gb2 += S.dH2[w][r][u];
        gw3 += S.A2[w][r][u] * S.dz[w][r];
      }
      gw[kOffB1 + u] += gb1;
      gw[kOffB2 + u] += gb2;
      gw[kOffW3 + u] += gw3;
#pragma unroll
      for (int f = 0; f < kIn; f++) gw[kOffW1 + f * kH + u] += gW1[f];
      // dW2[u][o] = sum_r A1[r][u] dH2[r][o]
      for (int o = 0; o < kH; o++) {
        float acc = 0.f;
        for (int r = 0; r < 16; r++) acc += S.A1[w][r][u] * S.dH2[w][r][o];
        gw[kOffW2 + u * kH + o] += acc;
      }
    }
    if (lane == 0) {
      float gb3 = 0.f;
      for (int r = 0; r < 16; r++) gb3 += S.dz[w][r];
      gw[kOffB3] += gb3;
    }
    __syncwarp();
  }
  // reduce the warps' gradients of this block and add them to the global gradient
  __syncthreads();
  for (int k = threadIdx.x; k < kNumParams; k += blockDim.x) {
    float acc = 0.f;
    for (int ww = 0; ww < kWarps; ww++) acc += S.g[ww][k];
    atomicAdd(grad + k, acc);
  }
  loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, 4);
  loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, 8);
  loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, 16);
  if (lane == 0) atomicAdd(loss, loss_acc);
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ grad, float* __restrict__ m1,
                            float* __restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kNumParams) return;
  const float gk = grad[k];
  const float a = b1 * m1[k] + (1.f - b1) * gk;
  const float b = b2 * m2[k] + (1.f - b2) * gk * gk;
  m1[k] = a;
  m2[k] = b;
  p[k] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// ---------------------------------------------------------------------------------------------
// delay factors of the mixed path's learned proposal
// ---------------------------------------------------------------------------------------------
// One block per target group (kFacGroup targets in the order the pair kernel takes them): the group's mean
// present position r_c, then e^z of the network for every source j of the bunch at r_c (features from the
// source's present record and its velocity one slot earlier, in the FP32 shadow ring), one source per lane.
constexpr int kFacThreads = 256;

__global__ void __launch_bounds__(kFacThreads, 3) factor_kernel(DeviceState s, const int* __restrict__ order) {
  __shared__ float4 s_part[kFacThreads / 32];
  const int gall = blockIdx.x;
  int b = 0;
  while (b + 1 < s.nbunch && s.bunches[b + 1].grp_off <= gall) b++;
  const BunchDesc& bd = s.bunches[b];
  const int g = gall - bd.grp_off;
  const int t0 = g * kFacGroup, t1 = min(bd.n, t0 + kFacGroup);
  const StepState st = *s.state;
  const int D = s.D, pn = st.pn;
  const int pprev = st.n > st.k0 ? (pn == 0 ? D - 1 : pn - 1) : pn;  // slot n - 1 (or n)
  const float invL = (float)(1.0 / (kC * st.dt * D));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // mean present position of the group (hi parts, relative to the bunch's split origin)
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (int t = t0 + threadIdx.x; t < t1; t += kFacThreads) {
    const long long i = order ? order[bd.off + t] : bd.off + t;
    const float4 q = __ldg(reinterpret_cast<const float4*>(s.rec32) + ((size_t)i * D + pn) * 3);
    sx += q.x;
    sy += q.y;
    sz += q.z;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
    sz += __shfl_xor_sync(0xffffffffu, sz, o);
  }
  if (lane == 0) s_part[w] = make_float4(sx, sy, sz, 0.f);
  __syncthreads();
  float3 rc = make_float3(0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < kFacThreads / 32; k++) {
    rc.x += s_part[k].x;
    rc.y += s_part[k].y;
    rc.z += s_part[k].z;
  }
  const float inv = 1.f / (float)max(t1 - t0, 1);
  rc = make_float3(rc.x * inv, rc.y * inv, rc.z * inv);
  const float b0 = (float)bd.beta_ref[0], b1 = (float)bd.beta_ref[1], b2 = (float)bd.beta_ref[2];
  const InferImage& net = *infer_image(s.mlp_image);
  float* __restrict__ fac = s.mlp_fac + bd.fac_off + (size_t)g * bd.n;
  // block y of the group's gridDim.y blocks, warp w: sources 32 (w + 8 y), then every 256 gridDim.y; the
  // loop bounds are the same for every lane (converged)
  for (int j0 = 32 * (w + (kFacThreads / 32) * (int)blockIdx.y); j0 < bd.n; j0 += kFacThreads * (int)gridDim.y) {
    const int jl = j0 + lane;
    const bool v = jl < bd.n;
    const size_t j = (size_t)bd.off + (v ? jl : j0);
    const float4* q = reinterpret_cast<const float4*>(s.rec32) + (j * D + pn) * 3;
    const float4 q0n = __ldg(q), q2n = __ldg(q + 2);
    const float4 q2p = __ldg(reinterpret_cast<const float4*>(s.rec32) + (j * D + pprev) * 3 + 2);
    const float f = warp_delay_factor(net, v, rc.x - q0n.x, rc.y - q0n.y, rc.z - q0n.z, b0 + q2n.x, b1 + q2n.y,
                                      b2 + q2n.z, q2n.x - q2p.x, q2n.y - q2p.y, q2n.z - q2p.z, invL, (float)D);
    if (v) fac[jl] = f;
  }
}

}  // namespace

namespace emppp {

size_t mlp_image_bytes() { return kImageBytes; }

cudaError_t launch_build_image(const float* params, void* image, cudaStream_t st) {
  static_assert(kH * (kH / 2) >= (kH / 8) * (kH / 16) * 32, "build grid covers every image entry");
  build_image_kernel<<<(kH * (kH / 2) + 255) / 256, 256, 0, st>>>(params, image);
  return cudaGetLastError();
}

cudaError_t launch_sample(const DeviceState& s, const int* pairs, long long m, float* feat, double* delay, float* zt,
                          cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  sample_kernel<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(s, pairs, m, feat, delay, zt);
  return cudaGetLastError();
}

cudaError_t launch_mlp_factors(const DeviceState& s, const int* order, cudaStream_t st) {
  if (s.ngroups <= 0 || !s.mlp_fac) return cudaSuccess;
  // the sources of each group split over enough blocks for about 8 resident blocks per SM (each block
  // forms the group's centroid again: 2 loads per thread)
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int split = std::min(64, std::max(1, (8 * sms + s.ngroups - 1) / s.ngroups));
  factor_kernel<<<dim3(s.ngroups, split), kFacThreads, 0, st>>>(s, order);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const void* image, const float* X, long long m, float* z, int mode, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  if (mode == 0) {
    long long tiles = (m + 15) / 16;
    long long blocks = (tiles + 3) / 4;
    if (blocks > 4096) blocks = 4096;
    forward_kernel<<<(unsigned)blocks, 128, 0, st>>>(static_cast<const NetImage*>(image), X, m, z);
  } else {
    long long blocks = (m + 127) / 128;
    if (blocks > 4096) blocks = 4096;
    forward_infer_kernel<<<(unsigned)blocks, 128, 0, st>>>(infer_image(image), X, m, z);
  }
  return cudaGetLastError();
}

cudaError_t launch_mlp_train_pass(const void* image, const float* X, const float* T, long long row0, long long rows,
                                  float norm, float* grad, float* loss, int num_sms, cudaStream_t st) {
  static_assert(sizeof(TrainSmem) < 227 * 1024, "training tile does not fit in shared memory");
  cudaError_t e = cudaFuncSetAttribute(train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem));
  if (e != cudaSuccess) return e;
  long long tiles = (rows + 15) / 16;
  long long blocks = (tiles + kWarps - 1) / kWarps;
  if (blocks > num_sms) blocks = num_sms;
  if (blocks < 1) blocks = 1;
  train_kernel<<<(unsigned)blocks, kWarps * 32, sizeof(TrainSmem), st>>>(static_cast<const NetImage*>(image), X, T,
                                                                         row0, rows, norm, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* grad, float* m1, float* m2, float lr, float b1, float b2, float eps,
                        int step, cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<(kNumParams + 255) / 256, 256, 0, st>>>(p, grad, m1, m2, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace emppp
