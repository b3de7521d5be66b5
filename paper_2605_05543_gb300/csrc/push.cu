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
// O(N) work; FP64 throughout (the momentum update needs it).
#include "emppp_internal.cuh"
#include "push_math.cuh"
#include "shadow.cuh"

namespace emppp {

__global__ void push_kernel(DeviceState s, BextParams bp) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const StepState st = *s.state;
  const int pnext = st.pn + 1 == s.D ? 0 : st.pn + 1;
  if (i == 0) s.slot_t[pnext] = st.t + st.dt;
  if (i >= s.N) return;
  const double* rec = s.rec64 + ((size_t)i * s.D + st.pn) * 6;
  double x[3] = {rec[0], rec[1], rec[2]};
  double u[3] = {s.u[3 * i], s.u[3 * i + 1], s.u[3 * i + 2]};
  const double E[3] = {s.Eself[3 * i], s.Eself[3 * i + 1], s.Eself[3 * i + 2]};
  const double Bs[3] = {s.Bself[3 * i], s.Bself[3 * i + 1], s.Bself[3 * i + 2]};
  double v[3], B[3];
  push_particle(x, u, E, Bs, bp, st.dt, v, B);
  const double x0 = x[0], x1 = x[1], x2 = x[2], v0 = v[0], v1 = v[1], v2 = v[2];
  if (!isfinite(x0 + x1 + x2 + u[0] + u[1] + u[2])) atomicOr(s.err, kErrNonFinite);
  s.u[3 * i] = u[0];
  s.u[3 * i + 1] = u[1];
  s.u[3 * i + 2] = u[2];
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

cudaError_t launch_push(const DeviceState& s, const BextParams& b, cudaStream_t st) {
  push_kernel<<<(unsigned)((s.N + 255) / 256), 256, 0, st>>>(s, b);
  return cudaGetLastError();
}

}  // namespace emppp
