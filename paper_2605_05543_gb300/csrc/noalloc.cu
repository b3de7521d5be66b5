// emppp_fields_noalloc: the FP64 self-field evaluation for callers that cannot let this library
// allocate device memory.
//
// Some callers own every byte of device memory themselves -- a framework whose caching allocator
// holds the GPU's memory, a service that runs under a fixed device-memory budget, a latency-critical
// loop in which a cudaMalloc could stall or fail once memory is nearly full. They can hand this
// library their inputs and outputs, but not let it take more. This entry point therefore keeps all
// of its working memory (per-slot tables and the per-slice partial field sums of the source-split
// kernel) in one fixed file-scope device array, g_scratch, of kScratchBytes bytes, which every GPU
// that loads the library holds until the process exits. It calls no cudaMalloc, cudaFree or other
// allocating routine.
//
// Because every call shares g_scratch, two calls whose work overlaps on the GPU (different streams,
// or different host threads) race and may corrupt each other's results; serialise them. Each call
// overwrites every scratch word it reads before reading it, so nothing is left to clear between
// calls. The device address of g_scratch is looked up with cudaGetSymbolAddress the first time the
// entry point runs on a device (with that device current); that first call should come before any
// stream capture on the device. The looked-up address is kept for the life of the process, so the
// entry point does not support cudaDeviceReset (or any other replacement of the device's primary
// context) between its calls.
//
// A numeric fault of a pair (|v| >= c in the history, coincident particles, non-finite input) is not
// reported through a status: the affected target's E and B come out NaN and the call returns EMPPP_OK.
//
// The evaluation is the FP64 path with the paper's own search (out-of-history test, near-field
// shortcut, bisection), reading the caller's history in the slot-major layout of emppp_set_history.
#include <mutex>

#include "../../include/emppp.h"
#include "emppp_internal.cuh"

namespace emppp {
void set_error_text(const char* msg);
}

using namespace emppp;

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kMaxSlots = 4096;
constexpr size_t kTabBytes = kMaxSlots * sizeof(double);
constexpr size_t kPartOffset = 2 * kTabBytes;  // lhs table, 1/dt table, then partial sums
constexpr int kMaxSplit = 64;
constexpr int kBlock = 128;
constexpr double kCoulomb = 1.0 / (4.0 * kPi * kEps0);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// (c (t_n - t_k))^2 in the reference operation order and 1 / (t_{k+1} - t_k), k = 0..nslots-1
__global__ void na_tables_kernel(const double* __restrict__ T, int nslots, double* __restrict__ lhs,
                                 double* __restrict__ idt) {
  const double tn = T[nslots - 1];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nslots; k += gridDim.x * blockDim.x) {
    const double ct = __dmul_rn(kC, __dsub_rn(tn, T[k]));
    lhs[k] = __dmul_rn(ct, ct);
    idt[k] = k + 1 < nslots ? 1.0 / (T[k + 1] - T[k]) : 0.0;
  }
}

__device__ __forceinline__ bool na_node_test(double r0, double r1, double r2, const double* __restrict__ w,
                                             double lhs) {
  const double d0 = __dsub_rn(r0, __ldg(w + 0));
  const double d1 = __dsub_rn(r1, __ldg(w + 1));
  const double d2 = __dsub_rn(r2, __ldg(w + 2));
  const double rhs = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
  return lhs <= rhs;
}

// One thread per target; blockIdx.y selects a slice of sources. Slot k of particle j is at
// W[(k * n + j) * 3]; the present slot is nslots - 1 and every slot is usable (k0 = 0).
__global__ void __launch_bounds__(kBlock)
    na_pair_kernel(const double* __restrict__ T, const double* __restrict__ W, const double* __restrict__ V,
                   const double* __restrict__ wts, long long n, int nslots, long long chunk,
                   const double* __restrict__ lhs, const double* __restrict__ idt, double* __restrict__ part) {
  const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  const int kn = nslots - 1;
  const double t = T[kn];
  const double* ri = W + ((size_t)kn * n + i) * 3;
  const double r0 = ri[0], r1 = ri[1], r2 = ri[2];
  const long long j0 = (long long)blockIdx.y * chunk;
  const long long j1 = min(n, j0 + chunk);
  const double c2 = kC * kC;
  const size_t sstride = (size_t)n * 3;  // doubles between consecutive slots of one particle
  double Et[3] = {0, 0, 0}, Bt[3] = {0, 0, 0}, Ep[3] = {0, 0, 0}, Bp[3] = {0, 0, 0};
  int in_block = 0;
  bool bad = false;
  for (long long j = j0; j < j1; ++j) {
    if (j == i) continue;
    const double* wj = W + (size_t)j * 3;
    const double* vj = V + (size_t)j * 3;
    int k1;
    bool ooh = false;
    // with a single slot (kn = 0) every pair is out of history; otherwise a test that is false at slot 0
    // (including a NaN separation) leads to slots kn - 1 >= 0 and, by bisection, 1..kn - 1 only
    if (kn == 0 || na_node_test(r0, r1, r2, wj, lhs[0])) {
      k1 = 0;
      ooh = true;
    } else if (!na_node_test(r0, r1, r2, wj + (size_t)(kn - 1) * sstride, lhs[kn - 1])) {
      k1 = kn - 1;
    } else {
      int lo = 0, hi = kn;
      while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (na_node_test(r0, r1, r2, wj + (size_t)m * sstride, lhs[m]))
          hi = m;
        else
          lo = m;
      }
      k1 = lo;
    }
    const double* w1 = wj + (size_t)k1 * sstride;
    const double* v1 = vj + (size_t)k1 * sstride;
    const double w10 = w1[0], w11 = w1[1], w12 = w1[2];
    const double v10 = v1[0], v11 = v1[1], v12 = v1[2];
    const double T1 = t - T[k1];
    const double d0 = r0 - w10, d1 = r1 - w11, d2 = r2 - w12;
    const double C2 = c2 - (v10 * v10 + v11 * v11 + v12 * v12);
    const double hb = (d0 * v10 + d1 * v11 + d2 * v12) - c2 * T1;
    const double C0 = c2 * T1 * T1 - (d0 * d0 + d1 * d1 + d2 * d2);
    const double qd = hb * hb - C2 * C0;
    if (!(C2 > 0.0) || !(qd >= 0.0)) {
      bad = true;
      continue;
    }
    const double sq = sqrt(qd);
    const double dt = (hb <= 0.0) ? C0 / (sq - hb) : -(hb + sq) / C2;
    const double w0 = w10 + v10 * dt, ww1 = w11 + v11 * dt, w2 = w12 + v12 * dt;
    double vv0 = v10, vv1 = v11, vv2 = v12, a0 = 0.0, a1 = 0.0, a2 = 0.0;
    if (!ooh) {
      const double* v2 = v1 + sstride;
      const double id = idt[k1];
      a0 = (v2[0] - v10) * id;
      a1 = (v2[1] - v11) * id;
      a2 = (v2[2] - v12) * id;
      vv0 = v10 + dt * a0;
      vv1 = v11 + dt * a1;
      vv2 = v12 + dt * a2;
    }
    const double e0 = r0 - w0, e1 = r1 - ww1, e2 = r2 - w2;
    const double R2s = e0 * e0 + e1 * e1 + e2 * e2;
    const double invR = rsqrt(R2s);
    const double R = R2s * invR;
    const double cinvR = kC * invR;
    const double vp0 = e0 * cinvR - vv0, vp1 = e1 * cinvR - vv1, vp2 = e2 * cinvR - vv2;
    const double evp = e0 * vp0 + e1 * vp1 + e2 * vp2;
    if (!(R2s > 0.0) || !(evp > 0.0)) {
      bad = true;
      continue;
    }
    const double c2mv2 = c2 - (vv0 * vv0 + vv1 * vv1 + vv2 * vv2);
    const double xa0 = vp1 * a2 - vp2 * a1, xa1 = vp2 * a0 - vp0 * a2, xa2 = vp0 * a1 - vp1 * a0;
    const double ac0 = e1 * xa2 - e2 * xa1, ac1 = e2 * xa0 - e0 * xa2, ac2 = e0 * xa1 - e1 * xa0;
    const double ievp = 1.0 / evp;
    const double q = -kQe * (wts ? wts[j] : 1.0);
    const double pref = kCoulomb * q * R * (ievp * ievp * ievp);
    const double E0 = pref * (c2mv2 * vp0 + ac0), E1 = pref * (c2mv2 * vp1 + ac1), E2 = pref * (c2mv2 * vp2 + ac2);
    const double bs = invR * (1.0 / kC);
    Ep[0] += E0;
    Ep[1] += E1;
    Ep[2] += E2;
    Bp[0] += (e1 * E2 - e2 * E1) * bs;
    Bp[1] += (e2 * E0 - e0 * E2) * bs;
    Bp[2] += (e0 * E1 - e1 * E0) * bs;
    if (++in_block == 64) {
      in_block = 0;
      for (int c = 0; c < 3; c++) {
        Et[c] += Ep[c];
        Bt[c] += Bp[c];
        Ep[c] = 0.0;
        Bp[c] = 0.0;
      }
    }
  }
  double* o = part + ((size_t)blockIdx.y * n + i) * 6;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int c = 0; c < 3; c++) {
    o[c] = bad ? nan : Et[c] + Ep[c];
    o[3 + c] = bad ? nan : Bt[c] + Bp[c];
  }
}

__global__ void na_reduce_kernel(const double* __restrict__ part, int S, long long n, double* __restrict__ E,
                                 double* __restrict__ B) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int s = 0; s < S; s++) {
    const double* o = part + ((size_t)s * n + i) * 6;
    for (int c = 0; c < 6; c++) acc[c] += o[c];
  }
  for (int c = 0; c < 3; c++) {
    E[3 * i + c] = acc[c];
    B[3 * i + c] = acc[3 + c];
  }
}

// device address of g_scratch, looked up once per device
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

emppp_status scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
      set_error_text(cudaGetErrorString(e));
      return EMPPP_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return EMPPP_OK;
}

}  // namespace

extern "C" EMPPP_API emppp_status emppp_fields_noalloc(int64_t n, int32_t nslots, const double* T, const double* W,
                                                       const double* V, const double* w, double* E, double* B,
                                                       void* cuda_stream) {
  if (n < 1 || !T || !W || !V || !E || !B) {
    set_error_text("emppp_fields_noalloc: n >= 1 and non-NULL T, W, V, E, B are required");
    return EMPPP_ERR_ARG;
  }
  if (nslots < 1 || nslots > kMaxSlots) {
    set_error_text("emppp_fields_noalloc: nslots must be in 1..4096 (fixed scratch size)");
    return EMPPP_ERR_ARG;
  }
  const size_t per_slice = (size_t)n * 6 * sizeof(double);
  const size_t max_slices = (kScratchBytes - kPartOffset) / per_slice;
  if (max_slices < 1) {
    set_error_text("emppp_fields_noalloc: n exceeds the 16 MiB scratch limit (n <= 348160)");
    return EMPPP_ERR_ARG;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error_text(e != cudaSuccess ? cudaGetErrorString(e) : "emppp_fields_noalloc: device index too large");
    return EMPPP_ERR_CUDA;
  }
  void* base = nullptr;
  emppp_status st = scratch_address(dev, &base);
  if (st != EMPPP_OK) return st;
  double* lhs = reinterpret_cast<double*>(base);
  double* idt = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kTabBytes);
  double* part = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kPartOffset);
  // source slices: enough blocks for about four per SM, within the scratch and a cap of 64
  const long long ntb = (n + kBlock - 1) / kBlock;
  long long S = (4LL * sms + ntb - 1) / ntb;
  if (S > kMaxSplit) S = kMaxSplit;
  if (S > (long long)max_slices) S = (long long)max_slices;
  if (S > n) S = n;
  if (S < 1) S = 1;
  const long long chunk = (n + S - 1) / S;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  na_tables_kernel<<<(nslots + 255) / 256, 256, 0, s>>>(T, nslots, lhs, idt);
  na_pair_kernel<<<dim3((unsigned)ntb, (unsigned)S), kBlock, 0, s>>>(T, W, V, w, n, nslots, chunk, lhs, idt, part);
  na_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, (int)S, n, E, B);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error_text(cudaGetErrorString(e));
    return EMPPP_ERR_CUDA;
  }
  return EMPPP_OK;
}
