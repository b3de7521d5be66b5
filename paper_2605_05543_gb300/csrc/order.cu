// Spatial order of the targets for the mixed-precision pair kernel.
//
// The particles' present positions are binned into a 32 x 32 x 32 grid over the bunch's bounding box,
// the cells are numbered along a Morton (Z-order) curve, and a counting sort lists the particles cell
// by cell. Threads then take targets in this order, so the 32 targets of a warp are close in space and
// their retarded slots of any one source lie within a few cache lines. The order is a permutation of
// 0..N-1 (each target is evaluated exactly once whatever the order); the order inside a cell comes from
// atomics and may differ run to run, which changes which thread evaluates a target but not its result.
#include "emppp_internal.cuh"

namespace emppp {

namespace {

constexpr int kCellBits = 5;                    // per axis
constexpr int kCells = 1 << (3 * kCellBits);    // 32768

__device__ __forceinline__ int ordered_int(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}

__device__ __forceinline__ float from_ordered_int(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__device__ __forceinline__ unsigned spread3(unsigned v) {  // 5 bits -> every third bit
  unsigned r = 0;
#pragma unroll
  for (int b = 0; b < kCellBits; b++) r |= ((v >> b) & 1u) << (3 * b);
  return r;
}

__global__ void bbox_init_kernel(int* __restrict__ bbox) {
  if (threadIdx.x < 3) {
    bbox[threadIdx.x] = ordered_int(3.0e38f);
    bbox[3 + threadIdx.x] = ordered_int(-3.0e38f);
  }
}

// present positions are the FP32 hi parts of slot n (relative to the split origin)
__global__ void bbox_kernel(const float* __restrict__ rec32, const StepState* __restrict__ state, long long N, int D,
                            int* __restrict__ bbox) {
  const int pn = (int)(state->n % D);
  float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const float* q = rec32 + ((size_t)i * D + pn) * 12;
    for (int c = 0; c < 3; c++) {
      const float x = q[c];
      if (x == x) {
        lo[c] = fminf(lo[c], x);
        hi[c] = fmaxf(hi[c], x);
      }
    }
  }
  for (int c = 0; c < 3; c++) {
    for (int off = 16; off > 0; off >>= 1) {
      lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], off));
      hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], off));
    }
  }
  if ((threadIdx.x & 31) == 0) {
    for (int c = 0; c < 3; c++) {
      atomicMin(bbox + c, ordered_int(lo[c]));
      atomicMax(bbox + 3 + c, ordered_int(hi[c]));
    }
  }
}

__global__ void key_hist_kernel(const float* __restrict__ rec32, const StepState* __restrict__ state, long long N,
                                int D, const int* __restrict__ bbox, unsigned short* __restrict__ key,
                                int* __restrict__ hist) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int pn = (int)(state->n % D);
  const float* q = rec32 + ((size_t)i * D + pn) * 12;
  unsigned cell[3];
  for (int c = 0; c < 3; c++) {
    const float lo = from_ordered_int(bbox[c]), hi = from_ordered_int(bbox[3 + c]);
    const float w = hi - lo;
    float f = w > 0.f ? (q[c] - lo) / w : 0.f;
    f = (f == f) ? fminf(fmaxf(f, 0.f), 1.f) : 0.f;
    const int k = (int)(f * (float)(1 << kCellBits));
    cell[c] = (unsigned)(k >= (1 << kCellBits) ? (1 << kCellBits) - 1 : k);
  }
  const unsigned m = spread3(cell[0]) | (spread3(cell[1]) << 1) | (spread3(cell[2]) << 2);
  key[i] = (unsigned short)m;
  atomicAdd(hist + m, 1);
}

// exclusive scan of kCells counts in one block of 1024 threads (32 cells each)
__global__ void __launch_bounds__(1024) scan_kernel(int* __restrict__ hist) {
  __shared__ int warp_tot[32];
  constexpr int per = kCells / 1024;
  const int t = threadIdx.x;
  int v[per];
  int sum = 0;
#pragma unroll
  for (int k = 0; k < per; k++) {
    v[k] = hist[t * per + k];
    sum += v[k];
  }
  // inclusive scan of the per-thread sums across the block
  int x = sum;
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, off);
    if ((t & 31) >= off) x += y;
  }
  if ((t & 31) == 31) warp_tot[t >> 5] = x;
  __syncthreads();
  if (t < 32) {
    int w = warp_tot[t];
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, off);
      if (t >= off) w += y;
    }
    warp_tot[t] = w;
  }
  __syncthreads();
  int base = x - sum + ((t >> 5) > 0 ? warp_tot[(t >> 5) - 1] : 0);
#pragma unroll
  for (int k = 0; k < per; k++) {
    hist[t * per + k] = base;
    base += v[k];
  }
}

__global__ void scatter_order_kernel(const unsigned short* __restrict__ key, long long N, int* __restrict__ offs,
                                     int* __restrict__ order) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int pos = atomicAdd(offs + key[i], 1);
  order[pos] = (int)i;
}

}  // namespace

size_t order_scratch_ints() { return 6 + kCells; }

// bbox: int[6], hist: int[kCells], key: ushort[N], order: int[N]
cudaError_t launch_target_order(const DeviceState& s, int* bbox, int* hist, unsigned short* key, int* order,
                                cudaStream_t st) {
  bbox_init_kernel<<<1, 32, 0, st>>>(bbox);
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int) * kCells, st);
  if (e != cudaSuccess) return e;
  bbox_kernel<<<152, 256, 0, st>>>(s.rec32, s.state, s.N, s.D, bbox);
  const unsigned nb = (unsigned)((s.N + 255) / 256);
  key_hist_kernel<<<nb, 256, 0, st>>>(s.rec32, s.state, s.N, s.D, bbox, key, hist);
  scan_kernel<<<1, 1024, 0, st>>>(hist);
  scatter_order_kernel<<<nb, 256, 0, st>>>(key, s.N, hist, order);
  return cudaGetLastError();
}

}  // namespace emppp
