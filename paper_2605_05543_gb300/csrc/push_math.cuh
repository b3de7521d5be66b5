// Per-particle arithmetic of the Higuera-Cary push (Sec. 2.3, Ripperda form) and of the background
// field (Sec. 2.6), shared by the stage-1 push and the stage-2 transport kernels so that both advance a
// particle with the same operations.
#pragma once

#include "emppp_internal.cuh"

namespace emppp {

// Background field at x: none, uniform b, or a centred dipole with moment m0 e_z about `center`:
// B = mu0/(4 pi) [3 (M.rhat) rhat - M] / r^3.
__device__ __forceinline__ void background_b(const BextParams& b, double x0, double x1, double x2, double B[3]) {
  B[0] = B[1] = B[2] = 0.0;
  if (b.kind == 1) {
    B[0] = b.b[0];
    B[1] = b.b[1];
    B[2] = b.b[2];
  } else if (b.kind == 2) {
    const double r0 = x0 - b.center[0], r1 = x1 - b.center[1], r2 = x2 - b.center[2];
    const double ir = rsqrt(r0 * r0 + r1 * r1 + r2 * r2);
    const double h0 = r0 * ir, h1 = r1 * ir, h2 = r2 * ir;
    const double Mr = b.m0 * h2;  // M = m0 e_z
    const double k = (kMu0 / (4.0 * kPi)) * ir * ir * ir;
    B[0] = k * (3.0 * Mr * h0);
    B[1] = k * (3.0 * Mr * h1);
    B[2] = k * (3.0 * Mr * h2 - b.m0);
  }
}

// One Higuera-Cary update of the proper velocity u with fields E, B and h = q dt / (2 m). With
// HAS_E = false the electric half-kicks are left out: for E = 0 they add a zero, so the values are the
// same.
template <bool HAS_E = true>
__device__ __forceinline__ void hc_kick(double u[3], const double E[3], const double B[3], double h) {
  const double um0 = HAS_E ? u[0] + h * E[0] : u[0];
  const double um1 = HAS_E ? u[1] + h * E[1] : u[1];
  const double um2 = HAS_E ? u[2] + h * E[2] : u[2];
  const double ic2 = 1.0 / (kC * kC);
  const double gm2 = 1.0 + (um0 * um0 + um1 * um1 + um2 * um2) * ic2;
  const double ta0 = h * B[0], ta1 = h * B[1], ta2 = h * B[2];
  const double tau2 = ta0 * ta0 + ta1 * ta1 + ta2 * ta2;
  const double us = (um0 * ta0 + um1 * ta1 + um2 * ta2) * (1.0 / kC);
  const double sigma = gm2 - tau2;
  // 1 / gamma+ directly: only its reciprocal is used
  const double igp = rsqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (tau2 + us * us))));
  const double t0 = ta0 * igp, t1 = ta1 * igp, t2 = ta2 * igp;
  const double s = 1.0 / (1.0 + (t0 * t0 + t1 * t1 + t2 * t2));
  const double umt = um0 * t0 + um1 * t1 + um2 * t2;
  const double up0 = s * (um0 + umt * t0 + (um1 * t2 - um2 * t1));
  const double up1 = s * (um1 + umt * t1 + (um2 * t0 - um0 * t2));
  const double up2 = s * (um2 + umt * t2 + (um0 * t1 - um1 * t0));
  if (HAS_E) {
    u[0] = up0 + h * E[0] + (up1 * t2 - up2 * t1);
    u[1] = up1 + h * E[1] + (up2 * t0 - up0 * t2);
    u[2] = up2 + h * E[2] + (up0 * t1 - up1 * t0);
  } else {
    u[0] = up0 + (up1 * t2 - up2 * t1);
    u[1] = up1 + (up2 * t0 - up0 * t2);
    u[2] = up2 + (up0 * t1 - up1 * t0);
  }
}

// One full push of a particle (x, u): half drift, kick with E and B_self + B_ext(x^{n+1/2}), half drift.
// Returns the new velocity in v and the total B used in Btot. HAS_E = false: E = 0 (stage 2).
template <bool HAS_E = true>
__device__ __forceinline__ void push_particle(double x[3], double u[3], const double E[3], const double Bself[3],
                                              const BextParams& bp, double dt, double v[3], double Btot[3]) {
  // 1 / gamma = 1 / sqrt(1 + u.u / c^2), then v = u / gamma as three products (FP64 throughout; each
  // division or square root costs several operations of GB300's FP64 pipe)
  const double ic2 = 1.0 / (kC * kC);
  const double ig0 = rsqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * ic2);
  const double hdt = 0.5 * dt;
  const double xh0 = x[0] + hdt * (u[0] * ig0), xh1 = x[1] + hdt * (u[1] * ig0), xh2 = x[2] + hdt * (u[2] * ig0);
  double Bg[3];
  background_b(bp, xh0, xh1, xh2, Bg);
  for (int c = 0; c < 3; c++) Btot[c] = Bself[c] + Bg[c];
  const double h = -kQe * dt / (2.0 * kMe);
  hc_kick<HAS_E>(u, E, Btot, h);
  const double ig1 = rsqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * ic2);
  v[0] = u[0] * ig1;
  v[1] = u[1] * ig1;
  v[2] = u[2] * ig1;
  x[0] = xh0 + hdt * v[0];
  x[1] = xh1 + hdt * v[1];
  x[2] = xh2 + hdt * v[2];
}

}  // namespace emppp
