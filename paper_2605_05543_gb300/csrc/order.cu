// Spatial order of the targets for the pair kernels.
//
// Each bunch's present positions are binned into a 2^b x 2^b x 2^b grid over the bunch's bounding box
// (b = 2..5 from the bunch size), the cells are numbered along a Morton (Z-order) curve, and a
// counting sort lists the bunch's particles cell by cell. Threads then take targets in this order, so
// the 32 targets of a warp are close in space: their retarded slots of any one source lie within a
// few cache lines, and they mostly take the same branch of the retarded-time search. One block of 1024 threads sorts one bunch entirely in shared memory. The order is a
// permutation of each bunch's index range (each target is evaluated exactly once whatever the order);
// the order inside a cell comes from shared-memory atomics and may differ run to run, which changes
// which thread evaluates a target but not its result.
#include "emppp_internal.cuh"

namespace emppp {

namespace {

constexpr int kThreads = 1024;
constexpr int kMaxBits = 5;
constexpr int kUnroll = 4;  // particles whose positions a thread loads before it uses any of them

__device__ __forceinline__ unsigned spread3(unsigned v, int bits) {  // bit k -> bit 3k
  unsigned r = 0;
  for (int k = 0; k < bits; k++) r |= ((v >> k) & 1u) << (3 * k);
  return r;
}

__host__ __device__ __forceinline__ int cell_bits(int n) {
  int lg = 0;
  while ((1 << (lg + 1)) <= n) lg++;
  int b = lg / 3;
  return b < 2 ? 2 : (b > kMaxBits ? kMaxBits : b);
}

__global__ void __launch_bounds__(kThreads) order_kernel(DeviceState s, unsigned* __restrict__ key,
                                                         int* __restrict__ order) {
  extern __shared__ int hist[];
  __shared__ float s_lo[3][32], s_hi[3][32];
  __shared__ int s_warp[32];
  const BunchDesc bd = s.bunches[blockIdx.x];
  const int n = bd.n;
  const long long off = bd.off;
  const int bits = cell_bits(n);
  const int cells = 1 << (3 * bits);
  const int pn = (int)(s.state->n % s.D);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  // present FP32 position (hi part) of particle k of the bunch: one record per particle's ring run, so
  // every particle is its own cache line; kUnroll of them are loaded before any is used
  const float4* __restrict__ rec = reinterpret_cast<const float4*>(s.rec32);
  auto position = [&](int k) { return __ldg(rec + ((size_t)(off + k) * s.D + pn) * 3); };
  // bounding box of the present FP32 positions
  float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
  for (int k0 = tid; k0 < n; k0 += kUnroll * kThreads) {
    float4 q[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      const int k = k0 + u * kThreads;
      const float nan = __int_as_float(0x7fc00000);  // skipped by the box below
      q[u] = k < n ? position(k) : make_float4(nan, nan, nan, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      const float x3[3] = {q[u].x, q[u].y, q[u].z};
      for (int c = 0; c < 3; c++) {
        const float x = x3[c];
        if (x == x) {
          lo[c] = fminf(lo[c], x);
          hi[c] = fmaxf(hi[c], x);
        }
      }
    }
  }
  for (int c = 0; c < 3; c++) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
      hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
    }
    if (lane == 0) {
      s_lo[c][wid] = lo[c];
      s_hi[c][wid] = hi[c];
    }
  }
  for (int k = tid; k < cells; k += kThreads) hist[k] = 0;
  __syncthreads();
  float blo[3], bw[3];
  for (int c = 0; c < 3; c++) {
    float a = 3.0e38f, b2 = -3.0e38f;
    for (int w = 0; w < kThreads / 32; w++) {
      a = fminf(a, s_lo[c][w]);
      b2 = fmaxf(b2, s_hi[c][w]);
    }
    blo[c] = a;
    bw[c] = b2 - a;
  }
  // cell keys and histogram
  const float side = (float)(1 << bits);
  for (int k0 = tid; k0 < n; k0 += kUnroll * kThreads) {
    float4 q[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      const int k = k0 + u * kThreads;
      q[u] = k < n ? position(k) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      const int k = k0 + u * kThreads;
      if (k >= n) break;
      const float x3[3] = {q[u].x, q[u].y, q[u].z};
      unsigned cc[3];
      for (int c = 0; c < 3; c++) {
        float f = bw[c] > 0.f ? (x3[c] - blo[c]) / bw[c] : 0.f;
        f = (f == f) ? fminf(fmaxf(f, 0.f), 1.f) : 0.f;
        const int m = (int)(f * side);
        cc[c] = (unsigned)(m >= (1 << bits) ? (1 << bits) - 1 : m);
      }
      const unsigned m = spread3(cc[0], bits) | (spread3(cc[1], bits) << 1) | (spread3(cc[2], bits) << 2);
      key[off + k] = m;
      atomicAdd(hist + m, 1);
    }
  }
  __syncthreads();
  // exclusive scan of the cell counts: each thread owns a contiguous run of cells
  const int per = (cells + kThreads - 1) / kThreads;
  const int c0 = tid * per, c1 = min(cells, c0 + per);
  int sum = 0;
  for (int k = c0; k < c1; k++) sum += hist[k];
  int x = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = s_warp[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  int base = x - sum + (wid > 0 ? s_warp[wid - 1] : 0);
  for (int k = c0; k < c1; k++) {
    const int v = hist[k];
    hist[k] = base;
    base += v;
  }
  __syncthreads();
  // scatter
  for (int k = tid; k < n; k += kThreads) {
    const int pos = atomicAdd(hist + key[off + k], 1);
    order[off + pos] = (int)(off + k);
  }
}

}  // namespace

constexpr size_t kSmem = sizeof(int) << (3 * kMaxBits);

// allows the kernel its shared-memory histogram on the current device (call before launching)
cudaError_t prepare_target_order() {
  return cudaFuncSetAttribute(order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
}

cudaError_t launch_target_order(const DeviceState& s, unsigned* key, int* order, long long max_bunch, cudaStream_t st) {
  // histogram of the largest bunch's cells only: a small system does not reserve 128 KB of shared memory
  const size_t smem = sizeof(int) << (3 * cell_bits((int)(max_bunch < (1LL << 30) ? max_bunch : (1LL << 30))));
  order_kernel<<<s.nbunch, kThreads, smem, st>>>(s, key, order);
  return cudaGetLastError();
}

}  // namespace emppp
