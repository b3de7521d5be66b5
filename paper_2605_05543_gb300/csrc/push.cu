// Higuera-Cary push (Sec. 2.3, Ripperda form) with the background field (Sec. 2.6) and the append of
// the new history slot (Sec. 2.2).
//
// Per particle: x^{n+1/2} = x^n + (dt/2) v^n; B = B_self + B_ext(x^{n+1/2}); h = q dt / (2 m);
//   u^- = u^n + h E;  gamma^- = sqrt(1 + u^-.u^- / c^2);  tau = h B;  u* = u^-.tau / c;
//   sigma = gamma^-^2 - tau^2;  gamma^+ = sqrt((sigma + sqrt(sigma^2 + 4 (tau^2 + u*^2))) / 2);
//   t = tau / gamma^+;  s = 1 / (1 + t^2);  u^+ = s [u^- + (u^-.t) t + u^- x t];
//   u^{n+1} = u^+ + h E + u^+ x t   (u^+ x t, not the u^- x t misprint the paper warns about);
//   v^{n+1} = u^{n+1} / gamma^{n+1};  x^{n+1} = x^{n+1/2} + (dt/2) v^{n+1}.
// Then slot n+1 (modulo D) receives (x^{n+1}, v^{n+1}) and the time stamp t_n + dt.
// O(N) work; FP64 throughout (the momentum update needs it). The launch also sums the pair kernel's
// per-chunk partial fields, picks the adaptive step and advances the clock, so that a step after the
// pair kernel is one launch.
#include "emppp_internal.cuh"
#include "energy.cuh"
#include "push_math.cuh"
#include "shadow.cuh"

namespace emppp {

// Step size of the push from the pair kernel's per-bunch interaction scales (Sec. 2.4): each bunch's
// dt_b = c_dt eta_min,b / v_max,b clamped to [dt_min, dt_max] (dt_max when no pair qualified or v_max = 0);
// the step of all bunches (one clock) is the smallest dt_b. eta_rep and v_rep are the binding bunch's.
__device__ __forceinline__ double adaptive_step(const DeviceState& s, const AdaptParams& ap, double& eta_rep,
                                                double& v_rep) {
  double dt = ap.dt_max;
  eta_rep = 0.0;
  v_rep = 0.0;
  for (int b = 0; b < s.nbunch; b++) {
    const double eta_min = __longlong_as_double((long long)s.scale[2 * b]);
    const double v_max = sqrt(__longlong_as_double((long long)s.scale[2 * b + 1]));
    const bool bounded = v_max > 0.0 && eta_min < __longlong_as_double(0x7ff0000000000000LL);
    const double dtb = fmin(ap.dt_max, fmax(ap.dt_min, bounded ? ap.c_dt * eta_min / v_max : ap.dt_max));
    if (b == 0 || dtb < dt) {
      dt = dtb;
      eta_rep = bounded ? eta_min : 0.0;
      v_rep = v_max;
    }
  }
  return dt;
}

// Half-step field point (comparison variant, fixed dt): before the pair evaluation of step n every
// particle's history gains a provisional slot n+1 holding its half-drifted position
// x^{n+1/2} = x^n + (dt/2) v^n (the push's own half drift, same operations) and v^n, stamped t_n + dt/2,
// and the clock moves to (n+1, t_n + dt/2), so that the set-up and pair launches evaluate the fields
// there. The post-pair launch (half = 1) then pushes from slot n and overwrites slot n+1. The last block
// to finish moves the clock, as in the post-pair launch.
__global__ void half_slot_kernel(DeviceState s) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const StepState st = *s.state;
  const int pn = (int)(st.n % s.D);
  const int pnext = pn + 1 == s.D ? 0 : pn + 1;
  if (i == 0) s.slot_t[pnext] = st.t + 0.5 * st.dt;
  if (i < s.N) {
    const double* rec = s.rec64 + ((size_t)i * s.D + pn) * 6;
    const double u0 = s.u[3 * i], u1 = s.u[3 * i + 1], u2 = s.u[3 * i + 2];
    const double ig0 = rsqrt(1.0 + (u0 * u0 + u1 * u1 + u2 * u2) * (1.0 / (kC * kC)));
    const double hdt = 0.5 * st.dt;
    const double v0 = u0 * ig0, v1 = u1 * ig0, v2 = u2 * ig0;
    const double x0 = rec[0] + hdt * v0, x1 = rec[1] + hdt * v1, x2 = rec[2] + hdt * v2;
    double* r = s.rec64 + ((size_t)i * s.D + pnext) * 6;
    reinterpret_cast<double2*>(r)[0] = make_double2(x0, x1);
    reinterpret_cast<double2*>(r)[1] = make_double2(x2, v0);
    reinterpret_cast<double2*>(r)[2] = make_double2(v1, v2);
    float4 q[3];
    const BunchDesc& bd = s.bunches[s.bunch_of[i]];
    shadow_record(bd.origin, bd.beta_ref, x0, x1, x2, v0, v1, v2, gamma2_of_u(u0, u1, u2), q);
    float4* o = reinterpret_cast<float4*>(s.rec32 + ((size_t)i * s.D + pnext) * 12);
    o[0] = q[0];
    o[1] = q[1];
    o[2] = q[2];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(s.done, 1u);
    if (prev == gridDim.x - 1) {
      s.state->n = st.n + 1;
      s.state->t = st.t + 0.5 * st.dt;
      *s.done = 0u;
    }
  }
}

// The rest of a step after the pair kernel, in one launch: the sum of each target's per-chunk partial
// fields (fixed chunk order), the adaptive step size, the push of every particle and the append of slot
// n+1, then (by the last block to finish) the clock advance n -> n+1, t -> t + dt and the reset of the
// interaction-scale reduction. The last block is found with a counter that every block increments once
// after its work; nothing waits on it. With half = 1 (half-step field point) the clock already stands at
// the provisional slot n+1: the push starts from slot n, the provisional slot is overwritten and the
// clock moves from t_n + dt/2 to t_n + dt (formed from t_n, as without the variant).
__global__ void __launch_bounds__(kEnergyThreads) step_post_kernel(DeviceState s, BextParams bp, AdaptParams ap,
                                                                   int chunked, int half, int wide, EnergyParams ep,
                                                                   EnergyMon* __restrict__ mon) {
  // wide = 1: one warp per particle, whose lanes read the per-chunk partial sums in parallel (small
  // systems, where a bunch is split into many short chunks); else one thread per particle
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long i = wide ? (g >> 5) : g;
  const int lane = threadIdx.x & 31;
  const bool owner = !wide || lane == 0;
  const StepState st = *s.state;
  double dt = st.dt, eta_rep = 0.0, v_rep = 0.0;
  if (ap.on) {
    // the step size, once per block (FP64 root and division) and shared
    __shared__ double s_step[3];
    if (threadIdx.x == 0) {
      s_step[0] = adaptive_step(s, ap, s_step[1], s_step[2]);
    }
    __syncthreads();
    dt = s_step[0];
    eta_rep = s_step[1];
    v_rep = s_step[2];
  }
  // slot of x^n, the slot the push writes and t_n
  const int pfrom = half ? (st.pn == 0 ? s.D - 1 : st.pn - 1) : st.pn;
  const int pnext = half ? st.pn : (st.pn + 1 == s.D ? 0 : st.pn + 1);
  const double t_n = half ? s.slot_t[pfrom] : st.t;
  if (g == 0) {
    s.slot_t[pnext] = t_n + dt;
    if (ap.on) {
      s.adapt_info[0] = dt;
      s.adapt_info[1] = eta_rep;
      s.adapt_info[2] = v_rep;
    }
  }
  if (i < s.N) {
    if (chunked) {
      // E_i = sum over the source chunks c of partial[c][i], in a fixed order
      const int S = s.sched[s.bunch_of[i]].nchunk;
      if (S > 1) {
        double acc[6] = {0, 0, 0, 0, 0, 0};
        if (wide) {
          // lane l adds chunks l, l + 32, ... in order; then a butterfly over the lanes, which leaves the
          // same sum in every lane (each step adds two equal-order partial sums, a commutative operation)
          for (int c = lane; c < S; c += 32) {
            const double* o = s.partial + ((size_t)c * s.N + i) * 6;
#pragma unroll
            for (int k = 0; k < 6; k++) acc[k] += o[k];
          }
#pragma unroll
          for (int m = 16; m >= 1; m >>= 1) {
#pragma unroll
            for (int k = 0; k < 6; k++) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], m);
          }
        } else {
          for (int c = 0; c < S; c++) {
            const double* o = s.partial + ((size_t)c * s.N + i) * 6;
#pragma unroll
            for (int k = 0; k < 6; k++) acc[k] += o[k];
          }
        }
        if (owner) {
          for (int c = 0; c < 3; c++) {
            s.Eself[3 * i + c] = acc[c];
            s.Bself[3 * i + c] = acc[3 + c];
          }
        }
      }
    }
  }
  // the particle this thread pushes: its own, or (wide) one of the block's particles by the lanes of the
  // first warp, so that the FP64 push occupies one warp per block rather than one lane of each warp
  long long ip = i;
  bool pusher = i < s.N && owner;
  if (wide) {
    __syncthreads();  // the block's field sums are written
    ip = (long long)blockIdx.x * (blockDim.x >> 5) + threadIdx.x;
    pusher = threadIdx.x < (blockDim.x >> 5) && ip < s.N;
  }
  if (pusher) {
    const long long i = ip;
    const double* rec = s.rec64 + ((size_t)i * s.D + pfrom) * 6;
    double x[3] = {rec[0], rec[1], rec[2]};
    double u[3] = {s.u[3 * i], s.u[3 * i + 1], s.u[3 * i + 2]};
    const double E[3] = {s.Eself[3 * i], s.Eself[3 * i + 1], s.Eself[3 * i + 2]};
    const double Bs[3] = {s.Bself[3 * i], s.Bself[3 * i + 1], s.Bself[3 * i + 2]};
    double v[3], B[3];
    push_particle(x, u, E, Bs, bp, dt, v, B);
    const double x0 = x[0], x1 = x[1], x2 = x[2], v0 = v[0], v1 = v[1], v2 = v[2];
    if (!isfinite(x0 + x1 + x2 + u[0] + u[1] + u[2])) atomicOr(s.err, kErrNonFinite);
    s.u[3 * i] = u[0];
    s.u[3 * i + 1] = u[1];
    s.u[3 * i + 2] = u[2];
    if (ep.on) s.ke[i] = kinetic_term(u[0], u[1], u[2], s.wts[i]);  // for the monitor in the last block
    for (int c = 0; c < 3; c++) s.Bout[3 * i + c] = B[c];
    // append slot n+1 (both rings)
    double* r = s.rec64 + ((size_t)i * s.D + pnext) * 6;
    reinterpret_cast<double2*>(r)[0] = make_double2(x0, x1);
    reinterpret_cast<double2*>(r)[1] = make_double2(x2, v0);
    reinterpret_cast<double2*>(r)[2] = make_double2(v1, v2);
    float4 q[3];
    const BunchDesc& bd = s.bunches[s.bunch_of[i]];
    shadow_record(bd.origin, bd.beta_ref, x0, x1, x2, v0, v1, v2, gamma2_of_u(u[0], u[1], u[2]), q);
    float4* o = reinterpret_cast<float4*>(s.rec32 + ((size_t)i * s.D + pnext) * 12);
    o[0] = q[0];
    o[1] = q[1];
    o[2] = q[2];
  }
  // the last block to finish advances the clock and resets the reduction for the next step (and, with
  // ep.on, evaluates the energy monitor of every bunch on the pushed state)
  __shared__ bool s_last;
  __shared__ double s_num[kEnergyThreads], s_den[kEnergyThreads];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(s.done, 1u);
    s_last = (prev == gridDim.x - 1);
    if (s_last) {
      s.state->n = half ? st.n : st.n + 1;
      s.state->t = t_n + dt;
      s.state->dt = dt;
      if (ap.on) {
        for (int b = 0; b < s.nbunch; b++) {
          s.scale[2 * b] = (unsigned long long)0x7ff0000000000000ULL;  // +inf
          s.scale[2 * b + 1] = 0ull;
        }
      }
      *s.done = 0u;
    }
  }
  __syncthreads();
  if (ep.on && s_last) {
    __threadfence();
    for (int b = 0; b < s.nbunch; b++)
      energy_block(s, ep, mon, 0, b, half ? st.n : st.n + 1, t_n + dt, s.ke, s_num, s_den);
  }
}

cudaError_t launch_step_post(const DeviceState& s, const BextParams& b, const AdaptParams& ap, bool chunked,
                             bool half, bool wide, const EnergyParams* ep, EnergyMon* mon, cudaStream_t st) {
  const long long threads = wide ? 32 * s.N : s.N;
  EnergyParams e{0, 1, 0.0};
  if (ep) e = *ep;  // the energy monitor in the last block (small systems)
  step_post_kernel<<<(unsigned)((threads + kEnergyThreads - 1) / kEnergyThreads), kEnergyThreads, 0, st>>>(
      s, b, ap, chunked ? 1 : 0, half ? 1 : 0, wide ? 1 : 0, e, mon);
  return cudaGetLastError();
}

cudaError_t launch_half_slot(const DeviceState& s, cudaStream_t st) {
  half_slot_kernel<<<(unsigned)((s.N + 255) / 256), 256, 0, st>>>(s);
  return cudaGetLastError();
}

}  // namespace emppp
