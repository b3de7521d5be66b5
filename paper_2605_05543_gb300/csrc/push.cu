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
#include "shadow.cuh"

namespace emppp {

namespace {

__device__ __forceinline__ void background_b(const BextParams& b, double x0, double x1, double x2, double B[3]) {
  B[0] = B[1] = B[2] = 0.0;
  if (b.kind == 1) {
    B[0] = b.b[0];
    B[1] = b.b[1];
    B[2] = b.b[2];
  } else if (b.kind == 2) {
    const double r0 = x0 - b.center[0], r1 = x1 - b.center[1], r2 = x2 - b.center[2];
    const double r = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
    const double ir = 1.0 / r;
    const double h0 = r0 * ir, h1 = r1 * ir, h2 = r2 * ir;
    const double Mr = b.m0 * h2;  // M = m0 e_z
    const double k = (kMu0 / (4.0 * kPi)) * ir * ir * ir;
    B[0] = k * (3.0 * Mr * h0);
    B[1] = k * (3.0 * Mr * h1);
    B[2] = k * (3.0 * Mr * h2 - b.m0);
  }
}

}  // namespace

// Shared by the stage-1 step and the stage-2 transport: one HC update of u with fields E, B.
__device__ __forceinline__ void hc_kick(double u[3], const double E[3], const double B[3], double h) {
  const double um0 = u[0] + h * E[0], um1 = u[1] + h * E[1], um2 = u[2] + h * E[2];
  const double ic2 = 1.0 / (kC * kC);
  const double gm2 = 1.0 + (um0 * um0 + um1 * um1 + um2 * um2) * ic2;
  const double ta0 = h * B[0], ta1 = h * B[1], ta2 = h * B[2];
  const double tau2 = ta0 * ta0 + ta1 * ta1 + ta2 * ta2;
  const double us = (um0 * ta0 + um1 * ta1 + um2 * ta2) * (1.0 / kC);
  const double sigma = gm2 - tau2;
  const double gp = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (tau2 + us * us))));
  const double igp = 1.0 / gp;
  const double t0 = ta0 * igp, t1 = ta1 * igp, t2 = ta2 * igp;
  const double s = 1.0 / (1.0 + (t0 * t0 + t1 * t1 + t2 * t2));
  const double umt = um0 * t0 + um1 * t1 + um2 * t2;
  const double up0 = s * (um0 + umt * t0 + (um1 * t2 - um2 * t1));
  const double up1 = s * (um1 + umt * t1 + (um2 * t0 - um0 * t2));
  const double up2 = s * (um2 + umt * t2 + (um0 * t1 - um1 * t0));
  u[0] = up0 + h * E[0] + (up1 * t2 - up2 * t1);
  u[1] = up1 + h * E[1] + (up2 * t0 - up0 * t2);
  u[2] = up2 + h * E[2] + (up0 * t1 - up1 * t0);
}

__global__ void push_kernel(DeviceState s, BextParams bp) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const StepState st = *s.state;
  const int pnext = st.pn + 1 == s.D ? 0 : st.pn + 1;
  if (i == 0) s.slot_t[pnext] = st.t + st.dt;
  if (i >= s.N) return;
  const double dt = st.dt;
  const double* rec = s.rec64 + ((size_t)i * s.D + st.pn) * 6;
  double u[3] = {s.u[3 * i], s.u[3 * i + 1], s.u[3 * i + 2]};
  const double g0 = sqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / (kC * kC));
  const double hdt = 0.5 * dt;
  const double xh0 = rec[0] + hdt * (u[0] / g0), xh1 = rec[1] + hdt * (u[1] / g0), xh2 = rec[2] + hdt * (u[2] / g0);
  double Bg[3];
  background_b(bp, xh0, xh1, xh2, Bg);
  const double E[3] = {s.Eself[3 * i], s.Eself[3 * i + 1], s.Eself[3 * i + 2]};
  const double B[3] = {s.Bself[3 * i] + Bg[0], s.Bself[3 * i + 1] + Bg[1], s.Bself[3 * i + 2] + Bg[2]};
  const double h = -kQe * dt / (2.0 * kMe);
  hc_kick(u, E, B, h);
  const double g1 = sqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / (kC * kC));
  const double v0 = u[0] / g1, v1 = u[1] / g1, v2 = u[2] / g1;
  const double x0 = xh0 + hdt * v0, x1 = xh1 + hdt * v1, x2 = xh2 + hdt * v2;
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
  shadow_record(s.origin, s.beta_ref, x0, x1, x2, v0, v1, v2, gamma2_of_u(u[0], u[1], u[2]), q);
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
