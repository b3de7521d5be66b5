// Stage-switch monitor (Sec. 2.7): the weighted mean kinetic energy per electron of each bunch,
//   E(t) = sum_i w_i (gamma_i - 1) m_e c^2 / sum_i w_i,
// and the criterion |dE/dt| < eps_E on its backward difference between consecutive steps. The
// criterion arms once the rate has reached eps_E (the rate "falls below" the threshold, so a bunch at
// rest does not switch at once); the switch step is the first step at which the rate has stayed below
// eps_E, after arming, for `hold` consecutive steps.
//
// One block per bunch (or, for small systems, the last block of the post-pair launch for all bunches).
// Each thread sums a fixed strided subset of its bunch's particles, then a fixed tree in shared memory
// adds the partial sums, so the result does not depend on scheduling or on which launch computes it. gamma - 1
// is formed as (u.u / c^2) / (gamma + 1), without the cancellation of 1 from gamma. The kernel runs
// after the push of every step (state n+1 at t_{n+1}) and is part of a captured step graph.
#include "energy.cuh"

namespace emppp {

__global__ void __launch_bounds__(kEnergyThreads) energy_kernel(DeviceState s, EnergyParams ep,
                                                                EnergyMon* __restrict__ mon, int reset) {
  __shared__ double s_num[kEnergyThreads];
  __shared__ double s_den[kEnergyThreads];
  energy_block(s, ep, mon, reset, blockIdx.x, s.state->n, s.state->t, nullptr, s_num, s_den);
}

cudaError_t launch_energy(const DeviceState& s, const EnergyParams& ep, EnergyMon* mon, bool reset, cudaStream_t st) {
  energy_kernel<<<s.nbunch, kEnergyThreads, 0, st>>>(s, ep, mon, reset ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace emppp
