// Throughput probes of the plain ALU pipes that bound the pair kernels: FP32 FMA, FP64 FMA and the
// multi-function unit (reciprocal square root). Each thread runs kChains independent dependent chains
// of the operation, so that every SM keeps its pipe full; the count of operations over the
// event-timed duration of the launch is the measured peak at the clock the GPU runs at that moment.
// These are the denominators of the roofline fractions the benchmark reports beside the nominal peaks
// (152 SMs x 128 FP32 lanes / 2 FP64 lanes / 16 MUFU lanes per clock).
#include <cuda_runtime.h>

#include "../../include/emppp.h"
#include "emppp_internal.cuh"

namespace emppp {
void set_error_text(const char* msg);
}

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) ffma_chain_kernel(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) dfma_chain_kernel(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) mufu_chain_kernel(float* out, int iters) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) x[c] = 1.0f + (float)(threadIdx.x + c) * 1e-3f;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = rsqrtf(x[c]);  // stays in [~0.9, ~1.1]: no denormals
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

EMPPP_API emppp_status emppp_measure_peaks(emppp_peaks* out, void* cuda_stream) {
  using namespace emppp;
  if (!out) {
    set_error_text("out is NULL");
    return EMPPP_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ffma_chain_kernel, kThreads, 0);
  if (e != cudaSuccess) {
    set_error_text(cudaGetErrorString(e));
    return EMPPP_ERR_CUDA;
  }
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  const size_t nthreads = (size_t)grid * kThreads;
  void* buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&buf, nthreads * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // best of three timed launches after one warm-up; the iteration counts make each launch a few ms
  auto timed = [&](auto launch, double ops_per_launch, double* rate) {
    launch();
    float best = 3.4e38f;
    for (int r = 0; r < 3 && e == cudaSuccess; r++) {
      e = cudaEventRecord(e0, st);
      launch();
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    *rate = ops_per_launch / (best * 1e-3);
  };
  const int it32 = 1 << 15, it64 = 1 << 10, itmu = 1 << 12;
  if (e == cudaSuccess)
    timed([&] { ffma_chain_kernel<<<grid, kThreads, 0, st>>>(static_cast<float*>(buf), it32, 0.999999f, 1e-6f); },
          2.0 * nthreads * kChains * (double)it32, &out->fp32_flops);
  if (e == cudaSuccess)
    timed([&] { dfma_chain_kernel<<<grid, kThreads, 0, st>>>(static_cast<double*>(buf), it64, 0.999999, 1e-6); },
          2.0 * nthreads * kChains * (double)it64, &out->fp64_flops);
  if (e == cudaSuccess)
    timed([&] { mufu_chain_kernel<<<grid, kThreads, 0, st>>>(static_cast<float*>(buf), itmu); },
          (double)nthreads * kChains * (double)itmu, &out->mufu_ops);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  out->sms = sms;
  out->launches = 12;
  if (e != cudaSuccess) {
    set_error_text(cudaGetErrorString(e));
    return EMPPP_ERR_CUDA;
  }
  return EMPPP_OK;
}

}  // extern "C"
