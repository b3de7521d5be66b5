// Stage-switch monitor (Sec. 2.7): the weighted mean kinetic energy per electron of each bunch,
//   E(t) = sum_i w_i (gamma_i - 1) m_e c^2 / sum_i w_i,
// and the criterion |dE/dt| < eps_E on its backward difference between consecutive steps. The
// criterion arms once the rate has reached eps_E (the rate "falls below" the threshold, so a bunch at
// rest does not switch at once); the switch step is the first step at which the rate has stayed below
// eps_E, after arming, for `hold` consecutive steps.
//
// One block per bunch. Each thread sums a fixed strided subset of its bunch's particles, then a fixed
// tree in shared memory adds the partial sums, so the result does not depend on scheduling. gamma - 1
// is formed as (u.u / c^2) / (gamma + 1), without the cancellation of 1 from gamma. The kernel runs
// after the push of every step (state n+1 at t_{n+1}) and is part of a captured step graph.
#include "emppp_internal.cuh"

namespace emppp {

namespace {
constexpr int kThreads = 256;
}

__global__ void __launch_bounds__(kThreads) energy_kernel(DeviceState s, EnergyParams ep, EnergyMon* __restrict__ mon,
                                                          int reset) {
  __shared__ double s_num[kThreads];
  __shared__ double s_den[kThreads];
  const int b = blockIdx.x;
  const BunchDesc& bd = s.bunches[b];
  double num = 0.0, den = 0.0;
  for (long long i = bd.off + threadIdx.x; i < bd.off + bd.n; i += kThreads) {
    const double u0 = s.u[3 * i], u1 = s.u[3 * i + 1], u2 = s.u[3 * i + 2];
    const double uu = (u0 * u0 + u1 * u1 + u2 * u2) / (kC * kC);
    const double w = s.wts[i];
    num += w * (uu / (sqrt(1.0 + uu) + 1.0));
    den += w;
  }
  s_num[threadIdx.x] = num;
  s_den[threadIdx.x] = den;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s_num[threadIdx.x] += s_num[threadIdx.x + h];
      s_den[threadIdx.x] += s_den[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double ebar = s_num[0] / s_den[0] * (kMe * kC * kC);
  const long long n = s.state->n;
  const double t = s.state->t;
  EnergyMon m = mon[b];
  if (reset) {
    m.ebar = ebar;
    m.rate = 0.0;
    m.t_prev = t;
    m.t_sw = 0.0;
    m.n_sw = -1;
    m.armed = 0;
    m.run = 0;
    m.switched = 0;
  } else {
    const double rate = (ebar - m.ebar) / (t - m.t_prev);
    m.rate = rate;
    m.ebar = ebar;
    m.t_prev = t;
    if (fabs(rate) >= ep.eps) m.armed = 1;
    m.run = (m.armed && fabs(rate) < ep.eps) ? m.run + 1 : 0;
    if (!m.switched && m.run >= ep.hold) {
      m.switched = 1;
      m.n_sw = n;
      m.t_sw = t;
    }
  }
  mon[b] = m;
}

cudaError_t launch_energy(const DeviceState& s, const EnergyParams& ep, EnergyMon* mon, bool reset, cudaStream_t st) {
  energy_kernel<<<s.nbunch, kThreads, 0, st>>>(s, ep, mon, reset ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace emppp
