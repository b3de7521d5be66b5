// History ring (Sec. 2.2: positions and velocities stored at discrete steps; the acceleration is not
// stored) and per-step slot tables.
#include "emppp_internal.cuh"
#include "shadow.cuh"

namespace emppp {

// Writes record (j, p) of both rings from an FP64 position and velocity.
__device__ __forceinline__ void write_record(const DeviceState& s, long long j, int p, double w0, double w1,
                                             double w2, double v0, double v1, double v2) {
  double* r = s.rec64 + ((size_t)j * s.D + p) * 6;
  reinterpret_cast<double2*>(r)[0] = make_double2(w0, w1);
  reinterpret_cast<double2*>(r)[1] = make_double2(w2, v0);
  reinterpret_cast<double2*>(r)[2] = make_double2(v1, v2);
  float4 q[3];
  const BunchDesc& bd = s.bunches[s.bunch_of[j]];
  shadow_record(bd.origin, bd.beta_ref, w0, w1, w2, v0, v1, v2, gamma2_of_v(v0, v1, v2), q);
  float4* o = reinterpret_cast<float4*>(s.rec32 + ((size_t)j * s.D + p) * 12);
  o[0] = q[0];
  o[1] = q[1];
  o[2] = q[2];
}

// v = u / gamma with gamma = sqrt(1 + u.u / c^2), in the operation order of a plain FP64 evaluation
__device__ __forceinline__ void velocity_of(double u0, double u1, double u2, double& v0, double& v1, double& v2) {
  const double uu = __dadd_rn(__dadd_rn(__dmul_rn(u0, u0), __dmul_rn(u1, u1)), __dmul_rn(u2, u2));
  const double g = __dsqrt_rn(__dadd_rn(1.0, __ddiv_rn(uu, __dmul_rn(kC, kC))));
  v0 = __ddiv_rn(u0, g);
  v1 = __ddiv_rn(u1, g);
  v2 = __ddiv_rn(u2, g);
}

__global__ void init_slot0_kernel(DeviceState s, const double* __restrict__ x, const double* __restrict__ u,
                                  const double* __restrict__ w) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    s.slot_t[0] = 0.0;
    *s.err = 0;
  }
  if (i >= s.N) return;
  const double u0 = u[3 * i], u1 = u[3 * i + 1], u2 = u[3 * i + 2];
  double v0, v1, v2;
  velocity_of(u0, u1, u2, v0, v1, v2);
  write_record(s, i, 0, x[3 * i], x[3 * i + 1], x[3 * i + 2], v0, v1, v2);
  s.u[3 * i] = u0;
  s.u[3 * i + 1] = u1;
  s.u[3 * i + 2] = u2;
  s.wts[i] = w ? w[i] : 1.0;
  s.kq32[i] = (float)(-kQe * s.wts[i] / (4.0 * kPi * kEps0));
}

__global__ void scatter_slot_kernel(DeviceState s, int p, const double* __restrict__ W, const double* __restrict__ V) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s.N) return;
  write_record(s, j, p, W[3 * j], W[3 * j + 1], W[3 * j + 2], V[3 * j], V[3 * j + 1], V[3 * j + 2]);
}

__global__ void gather_slot_kernel(DeviceState s, int p, double* __restrict__ W, double* __restrict__ V) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s.N) return;
  const double* r = s.rec64 + ((size_t)j * s.D + p) * 6;
  for (int c = 0; c < 3; c++) {
    if (W) W[3 * j + c] = r[c];
    if (V) V[3 * j + c] = r[3 + c];
  }
}

__global__ void set_state_kernel(DeviceState s, long long n, double t, double dt, long long hist_start,
                                 const double* __restrict__ u, const double* __restrict__ w) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    s.state->n = n;
    s.state->t = t;
    s.state->dt = dt;
    s.state->hist_start = hist_start;
    *s.err = 0;
  }
  if (i >= s.N) return;
  if (u) {
    s.u[3 * i] = u[3 * i];
    s.u[3 * i + 1] = u[3 * i + 1];
    s.u[3 * i + 2] = u[3 * i + 2];
  }
  s.wts[i] = w ? w[i] : 1.0;
  s.kq32[i] = (float)(-kQe * s.wts[i] / (4.0 * kPi * kEps0));
}

// Slot-table entry of window offset l (slot p0 + l, modulo D) at time t_n (Sec. 2.2): the squared
// light-travel distance (c (t_n - t_k))^2 in exactly the operation order of the reference evaluation
// (so that the FP64 node test decides identically), its guard-band thresholds in FP32, c (t_n - t_k) in
// FP32, and 1 / (t_{k+1} - t_k).
constexpr double kGuardHi = (1.0 + kGuardBand) / (1.0 - kGuardBand), kGuardLo = (1.0 - kGuardBand) / (1.0 + kGuardBand);

// FP32 upper threshold of a slot's (c (t_n - t_k))^2 (the node test is true above it)
__device__ __forceinline__ float upper_threshold(double lhs) { return __double2float_ru(lhs * kGuardHi); }

__device__ __forceinline__ void slot_table(const DeviceState& s, int l, int p0, int nwin, double t_n) {
  int p = p0 + l;
  if (p >= s.D) p -= s.D;
  const double tk = s.slot_t[p];
  const double ct = __dmul_rn(kC, __dsub_rn(t_n, tk));
  const double lhs = __dmul_rn(ct, ct);
  s.tab.lhs64[p] = lhs;
  float icdt = 0.f;
  if (l + 1 < nwin) {
    int q = p + 1 == s.D ? 0 : p + 1;
    const double dtk = s.slot_t[q] - tk;
    s.tab.inv_dtk[p] = 1.0 / dtk;
    icdt = (float)(1.0 / (kC * dtk));
  } else {
    s.tab.inv_dtk[p] = 0.0;
  }
  s.tab.tab32[p] = make_float4(upper_threshold(lhs), __double2float_rd(lhs * kGuardLo), (float)ct, icdt);
}

// Per-step slot tables over the usable window k0..n alone (used before the delay sampler).
__global__ void prep_kernel(DeviceState s) {
  const long long n = s.state->n;
  const double t_n = s.state->t;
  const long long hs = s.state->hist_start;
  const long long k0 = n - s.D + 1 > hs ? n - s.D + 1 : hs;
  const int p0 = (int)(k0 % s.D);
  const int pn = (int)(n % s.D);
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    s.state->k0 = k0;
    s.state->p0 = p0;
    s.state->pn = pn;
  }
  const int nwin = (int)(n - k0 + 1);
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nwin; l += gridDim.x * blockDim.x) slot_table(s, l, p0, nwin, t_n);
}

// Per-step set-up, one launch before the pair kernel: the window k0..n and its slot tables (as
// prep_kernel), the pair kernel's work counter, and, for the mixed path, per-source vectors (eq:linear at
// t_n):
//   P_j = w_{j,n-1} + v_{j,n-1} (t_n - t_{n-1}), the end of the last history segment, split hi/lo about
//     the bunch origin. For a pair in the near-field shortcut bracket [n-1, n] the retarded point is
//     written as P_j - v_{j,n-1} tau with tau = t_n - t_r: the same point as w_{j,n-1} + v_{j,n-1}
//     (t_r - t_{n-1}), with FP32 precision kept when c tau is far below c (t_n - t_{n-1}).
//   X_j = w_{j,k0} + v_{j,k0} (t_n - t_{k0}) - w_{j,n}, where the straight line of eq:linear2 (the
//     out-of-history case) is at t_n, relative to the source's present position. Along that line the
//     source moves uniformly, so its field is Heaviside's field about the point w_{j,n} + X_j; the
//     separation from a target is then (r - w_{j,n}) - X_j, formed without cancellation.
//   c_j = w_{j,n} - w_{j,k0} and T (1 + 32u) - |c_j|^2 (1 - 32u), rounded up, with T the FP32 upper
//     threshold of slot k0: the oldest-slot bound (kChordMargin), by which an out-of-history pair's
//     node test of slot k0 needs no record of that slot; and the FP32 record's beta - beta_ref,
//     1/gamma^2 and gamma^2 of slot k0, which Heaviside's field of that pair reads.
__global__ void setup_kernel(DeviceState s, int extrap) {
  const long long n = s.state->n;
  const double t_n = s.state->t;
  const long long hs = s.state->hist_start;
  const long long k0 = n - s.D + 1 > hs ? n - s.D + 1 : hs;
  const int p0 = (int)(k0 % s.D);
  const int pn = (int)(n % s.D);
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid == 0) {
    s.state->k0 = k0;
    s.state->p0 = p0;
    s.state->pn = pn;
    *s.work = 0;
  }
  const int nwin = (int)(n - k0 + 1);
  if (gid < nwin) slot_table(s, (int)gid, p0, nwin, t_n);
  if (!extrap || gid >= s.N) return;
  const long long j = gid;
  const double* rn = s.rec64 + ((size_t)j * s.D + pn) * 6;
  const double* r0 = s.rec64 + ((size_t)j * s.D + p0) * 6;
  const float* q0 = s.rec32 + ((size_t)j * s.D + p0) * 12;  // FP32 record of slot k0
  float4* ext = s.ext32 + (size_t)j * kExtCount;
  const double dt0 = s.slot_t[pn] - s.slot_t[p0];
  ext[kExtLine] = make_float4((float)((r0[0] + r0[3] * dt0) - rn[0]), (float)((r0[1] + r0[4] * dt0) - rn[1]),
                              (float)((r0[2] + r0[5] * dt0) - rn[2]), q0[11]);
  ext[kExtOldest] = make_float4(q0[8], q0[9], q0[10], q0[3]);
  {
    const double c0 = rn[0] - r0[0], c1 = rn[1] - r0[1], c2 = rn[2] - r0[2];
    const double ct = __dmul_rn(kC, __dsub_rn(t_n, s.slot_t[p0]));
    const double cc = c0 * c0 + c1 * c1 + c2 * c2;
    const double rhs = (double)upper_threshold(__dmul_rn(ct, ct)) * (1.0 + kChordMargin) - cc * (1.0 - kChordMargin);
    const float inf = __int_as_float(0x7f800000);
    ext[kExtChord] = make_float4((float)c0, (float)c1, (float)c2, n > k0 ? __double2float_ru(rhs) : inf);
  }
  if (n <= k0) return;  // no segment [n-1, n] in the window
  const int p1 = pn == 0 ? s.D - 1 : pn - 1;
  const double dtl = s.slot_t[pn] - s.slot_t[p1];
  const double* r = s.rec64 + ((size_t)j * s.D + p1) * 6;
  const BunchDesc& bd = s.bunches[s.bunch_of[j]];
  const double d0 = (r[0] + r[3] * dtl) - bd.origin[0];
  const double d1 = (r[1] + r[4] * dtl) - bd.origin[1];
  const double d2 = (r[2] + r[5] * dtl) - bd.origin[2];
  const float h0 = (float)d0, h1 = (float)d1, h2 = (float)d2;
  ext[kExtSegHi] = make_float4(h0, h1, h2, 0.f);
  ext[kExtSegLo] = make_float4((float)(d0 - (double)h0), (float)(d1 - (double)h1), (float)(d2 - (double)h2), 0.f);
}

__global__ void reset_scale_kernel(DeviceState s) {
  for (int b = 0; b < s.nbunch; b++) {
    s.scale[2 * b] = (unsigned long long)0x7ff0000000000000ULL;
    s.scale[2 * b + 1] = 0ull;
  }
  s.adapt_info[0] = s.state->dt;
  s.adapt_info[1] = 0.0;
  s.adapt_info[2] = 0.0;
}

__global__ void gather_positions_kernel(DeviceState s, double* __restrict__ x) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s.N) return;
  const int pn = (int)(s.state->n % s.D);
  const double* r = s.rec64 + ((size_t)j * s.D + pn) * 6;
  x[3 * j] = r[0];
  x[3 * j + 1] = r[1];
  x[3 * j + 2] = r[2];
}

static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

cudaError_t launch_init_slot0(const DeviceState& s, const double* x, const double* u, const double* w,
                              cudaStream_t st) {
  init_slot0_kernel<<<blocks_for(s.N, 256), 256, 0, st>>>(s, x, u, w);
  return cudaGetLastError();
}

cudaError_t launch_scatter_slot(const DeviceState& s, int p, const double* W, const double* V, cudaStream_t st) {
  scatter_slot_kernel<<<blocks_for(s.N, 256), 256, 0, st>>>(s, p, W, V);
  return cudaGetLastError();
}

cudaError_t launch_gather_slot(const DeviceState& s, int p, double* W, double* V, cudaStream_t st) {
  gather_slot_kernel<<<blocks_for(s.N, 256), 256, 0, st>>>(s, p, W, V);
  return cudaGetLastError();
}

cudaError_t launch_set_state(const DeviceState& s, long long n, double t, double dt, long long hist_start,
                             const double* u, const double* w, cudaStream_t st) {
  set_state_kernel<<<blocks_for(s.N, 256), 256, 0, st>>>(s, n, t, dt, hist_start, u, w);
  return cudaGetLastError();
}

cudaError_t launch_prep(const DeviceState& s, cudaStream_t st) {
  prep_kernel<<<1, 1024, 0, st>>>(s);
  return cudaGetLastError();
}

cudaError_t launch_setup(const DeviceState& s, bool extrap, cudaStream_t st) {
  const long long n = extrap ? (s.N > s.D ? s.N : s.D) : s.D;
  // small blocks: the per-slot and per-source FP64 work spreads over more SMs (an FP64 warp instruction
  // holds an SM's FP64 pipe for 16 cycles)
  setup_kernel<<<blocks_for(n, 64), 64, 0, st>>>(s, extrap ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_reset_scale(const DeviceState& s, cudaStream_t st) {
  reset_scale_kernel<<<1, 1, 0, st>>>(s);
  return cudaGetLastError();
}

cudaError_t launch_gather_positions(const DeviceState& s, double* x, cudaStream_t st) {
  gather_positions_kernel<<<blocks_for(s.N, 256), 256, 0, st>>>(s, x);
  return cudaGetLastError();
}

}  // namespace emppp
