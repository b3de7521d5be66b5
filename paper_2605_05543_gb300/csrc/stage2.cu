// Stage-1 -> stage-2 handoff and stage-2 transport (Sec. 2.7): after the switch the pair interaction is
// turned off (E = 0, B = B_geo) and the particles are advanced with a larger step in the background
// field alone. Particles are then independent: the transport kernel keeps each particle in registers
// for many steps, with the same per-step arithmetic as the stage-1 push (push_math.cuh), and writes the
// final state back as the single present history slot.
#include "emppp_internal.cuh"
#include "push_math.cuh"
#include "shadow.cuh"

namespace emppp {

namespace {

constexpr int kSumThreads = 256;

// per bunch: sum_i w_i x_i (3) and sum_i w_i over the present positions, in a fixed order
__global__ void __launch_bounds__(kSumThreads) bunch_sums_kernel(DeviceState s) {
  __shared__ double sh[4][kSumThreads];
  const BunchDesc bd = s.bunches[blockIdx.x];
  const int pn = (int)(s.state->n % s.D);
  double acc[4] = {0, 0, 0, 0};
  for (int k = threadIdx.x; k < bd.n; k += kSumThreads) {
    const long long i = bd.off + k;
    const double* r = s.rec64 + ((size_t)i * s.D + pn) * 6;
    const double w = s.wts[i];
    acc[0] += w * r[0];
    acc[1] += w * r[1];
    acc[2] += w * r[2];
    acc[3] += w;
  }
  for (int c = 0; c < 4; c++) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = kSumThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 4; c++) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 4; c++) s.bsum[4 * blockIdx.x + c] = sh[c][0];
}

// x += shift of the particle's bunch on the present slot; the history restarts at the present slot
__global__ void translate_kernel(DeviceState s, const double* __restrict__ shifts) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = s.state->n;
  const int pn = (int)(n % s.D);
  if (i == 0) s.state->hist_start = n;
  if (i >= s.N) return;
  const int b = s.bunch_of[i];
  double* r = s.rec64 + ((size_t)i * s.D + pn) * 6;
  const double x0 = r[0] + shifts[3 * b], x1 = r[1] + shifts[3 * b + 1], x2 = r[2] + shifts[3 * b + 2];
  r[0] = x0;
  r[1] = x1;
  r[2] = x2;
  float4 q[3];
  const BunchDesc& bd = s.bunches[b];
  shadow_record(bd.origin, bd.beta_ref, x0, x1, x2, r[3], r[4], r[5], gamma2_of_u(s.u[3 * i], s.u[3 * i + 1], s.u[3 * i + 2]),
                q);
  float4* o = reinterpret_cast<float4*>(s.rec32 + ((size_t)i * s.D + pn) * 12);
  o[0] = q[0];
  o[1] = q[1];
  o[2] = q[2];
}

// nsteps transport steps of every particle from the present slot n; the result is written as slot
// n + nsteps (state advanced by the host-side caller through the slot time stamp argument)
__global__ void transport_kernel(DeviceState s, BextParams bp, double dt, int nsteps, double t_end) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = s.state->n;
  const int pn = (int)(n % s.D);
  const int pe = (int)((n + nsteps) % s.D);
  if (i >= s.N) return;
  const double* rec = s.rec64 + ((size_t)i * s.D + pn) * 6;
  double x[3] = {rec[0], rec[1], rec[2]};
  double u[3] = {s.u[3 * i], s.u[3 * i + 1], s.u[3 * i + 2]};
  const double E[3] = {0.0, 0.0, 0.0};
  double v[3] = {rec[3], rec[4], rec[5]}, B[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < nsteps; k++) push_particle<false>(x, u, E, E, bp, dt, v, B);
  if (!isfinite(x[0] + x[1] + x[2] + u[0] + u[1] + u[2])) atomicOr(s.err, kErrNonFinite);
  for (int c = 0; c < 3; c++) {
    s.u[3 * i + c] = u[c];
    s.Eself[3 * i + c] = 0.0;
    s.Bself[3 * i + c] = 0.0;
    s.Bout[3 * i + c] = B[c];
  }
  double* r = s.rec64 + ((size_t)i * s.D + pe) * 6;
  reinterpret_cast<double2*>(r)[0] = make_double2(x[0], x[1]);
  reinterpret_cast<double2*>(r)[1] = make_double2(x[2], v[0]);
  reinterpret_cast<double2*>(r)[2] = make_double2(v[1], v[2]);
  float4 q[3];
  const BunchDesc& bd = s.bunches[s.bunch_of[i]];
  shadow_record(bd.origin, bd.beta_ref, x[0], x[1], x[2], v[0], v[1], v[2], gamma2_of_u(u[0], u[1], u[2]), q);
  float4* o = reinterpret_cast<float4*>(s.rec32 + ((size_t)i * s.D + pe) * 12);
  o[0] = q[0];
  o[1] = q[1];
  o[2] = q[2];
  if (i == 0) s.slot_t[pe] = t_end;
}

__global__ void transport_advance_kernel(StepState* st, int nsteps, double t_end) {
  st->n += nsteps;
  st->t = t_end;
  st->hist_start = st->n;
}

}  // namespace

cudaError_t launch_bunch_sums(const DeviceState& s, cudaStream_t st) {
  bunch_sums_kernel<<<s.nbunch, kSumThreads, 0, st>>>(s);
  return cudaGetLastError();
}

cudaError_t launch_translate(const DeviceState& s, const double* shifts, cudaStream_t st) {
  translate_kernel<<<(unsigned)((s.N + 255) / 256), 256, 0, st>>>(s, shifts);
  return cudaGetLastError();
}

// nsteps transport steps ending at time t_end (accumulated by the caller one step at a time)
cudaError_t launch_transport_chunk(const DeviceState& s, const BextParams& b, double dt, int nsteps, double t_end,
                                   cudaStream_t st) {
  transport_kernel<<<(unsigned)((s.N + 127) / 128), 128, 0, st>>>(s, b, dt, nsteps, t_end);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  transport_advance_kernel<<<1, 1, 0, st>>>(s.state, nsteps, t_end);
  return cudaGetLastError();
}

}  // namespace emppp
