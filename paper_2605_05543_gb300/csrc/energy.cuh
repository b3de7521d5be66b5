// Energy monitor of the stage switch (Sec. 2.7), one bunch per call by one block of threads: shared by
// the monitor's own launch and the last block of the post-pair launch, so that both compute the same
// values with the same operations.
#pragma once

#include "emppp_internal.cuh"

namespace emppp {

// the monitor of bunch b, by one block of kEnergyThreads threads (also called by the last block of the
// post-pair launch, which has the same size); n, t: the present step and time. Reads of the particles
// go to L2 (__ldcg): they were written by other blocks of the same launch in that case.
__device__ __forceinline__ void energy_block(const DeviceState& s, const EnergyParams& ep, EnergyMon* __restrict__ mon, int reset,
                             int b, long long n, double t, double* s_num, double* s_den) {
  const BunchDesc& bd = s.bunches[b];
  double num = 0.0, den = 0.0;
  for (long long i = bd.off + threadIdx.x; i < bd.off + bd.n; i += kEnergyThreads) {
    const double u0 = __ldcg(s.u + 3 * i), u1 = __ldcg(s.u + 3 * i + 1), u2 = __ldcg(s.u + 3 * i + 2);
    const double uu = (u0 * u0 + u1 * u1 + u2 * u2) / (kC * kC);
    const double w = __ldcg(s.wts + i);
    num += w * (uu / (sqrt(1.0 + uu) + 1.0));
    den += w;
  }
  s_num[threadIdx.x] = num;
  s_den[threadIdx.x] = den;
  __syncthreads();
  for (int h = kEnergyThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s_num[threadIdx.x] += s_num[threadIdx.x + h];
      s_den[threadIdx.x] += s_den[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double ebar = s_num[0] / s_den[0] * (kMe * kC * kC);
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
  __syncthreads();  // the shared arrays are reused for the next bunch
}

}  // namespace emppp
