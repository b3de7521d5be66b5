// Energy monitor of the stage switch (Sec. 2.7), one bunch per call by one block of threads: shared by
// the monitor's own launch and the last block of the post-pair launch, so that both compute the same
// values with the same operations.
#pragma once

#include "emppp_internal.cuh"

namespace emppp {

// kinetic-energy term of one particle, w (gamma - 1) / (m_e c^2) with gamma - 1 = (u.u / c^2) /
// (gamma + 1), in a fixed sequence of correctly rounded operations, so that the pushing thread and the
// monitor's own launch form the same value
__device__ __forceinline__ double kinetic_term(double u0, double u1, double u2, double w) {
  const double su = __fma_rn(u2, u2, __fma_rn(u1, u1, __dmul_rn(u0, u0)));
  const double uu = __ddiv_rn(su, kC * kC);
  return __dmul_rn(w, __ddiv_rn(uu, __dadd_rn(__dsqrt_rn(__dadd_rn(1.0, uu)), 1.0)));
}

// the monitor of bunch b, by one block of kEnergyThreads threads (also called by the last block of the
// post-pair launch, which has the same size); n, t: the present step and time. terms: the particles'
// kinetic_term values when already formed (by the pushing threads of the same launch), else nullptr.
// Reads of the particles go to L2 (__ldcg): they were written by other blocks of the same launch.
__device__ __forceinline__ void energy_block(const DeviceState& s, const EnergyParams& ep, EnergyMon* __restrict__ mon,
                                             int reset, int b, long long n, double t, const double* terms,
                                             double* s_num, double* s_den) {
  const BunchDesc& bd = s.bunches[b];
  double num = 0.0, den = 0.0;
  for (long long i = bd.off + threadIdx.x; i < bd.off + bd.n; i += kEnergyThreads) {
    const double w = __ldcg(s.wts + i);
    if (terms) {
      num += __ldcg(terms + i);
    } else {
      num += kinetic_term(__ldcg(s.u + 3 * i), __ldcg(s.u + 3 * i + 1), __ldcg(s.u + 3 * i + 2), w);
    }
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
