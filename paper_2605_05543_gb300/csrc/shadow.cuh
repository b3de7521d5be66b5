// FP32 shadow record of one history slot, used by the mixed-precision pair path and by the FP32
// delay guess. Three float4 per (particle, slot):
//   q0 = (hi.x, hi.y, hi.z, 1/gamma^2)   hi = fl32(w - origin)
//   q1 = (lo.x, lo.y, lo.z, 0)           lo = fl32((w - origin) - hi), so hi + lo carries ~48 bits
//   q2 = (dbeta.x, dbeta.y, dbeta.z, gamma^2)  dbeta = v/c - beta_ref
// 1/gamma^2 = 1 - beta^2 is formed in FP64, so the FP32 path never subtracts beta^2 from 1. Velocities
// are stored relative to a reference velocity beta_ref (the velocity of one particle of the bunch when
// the state was set): the spread of a bunch's velocities is small, so the FP32 difference of two stored
// velocities (the acceleration of eq:linear) keeps its relative precision; beta itself is
// beta_ref + dbeta.
#pragma once

#include "emppp_internal.cuh"

namespace emppp {

__device__ __forceinline__ void shadow_record(const double origin[3], const double beta_ref[3], double w0, double w1,
                                              double w2, double v0, double v1, double v2, double gamma2, float4 q[3]) {
  const double d0 = w0 - origin[0], d1 = w1 - origin[1], d2 = w2 - origin[2];
  const float h0 = (float)d0, h1 = (float)d1, h2 = (float)d2;
  const double ic = 1.0 / kC;
  q[0] = make_float4(h0, h1, h2, (float)(1.0 / gamma2));
  q[1] = make_float4((float)(d0 - (double)h0), (float)(d1 - (double)h1), (float)(d2 - (double)h2), 0.f);
  q[2] = make_float4((float)(v0 * ic - beta_ref[0]), (float)(v1 * ic - beta_ref[1]), (float)(v2 * ic - beta_ref[2]),
                     (float)gamma2);
}

// gamma^2 of a stored velocity: 1 / (1 - v.v / c^2)
__device__ __forceinline__ double gamma2_of_v(double v0, double v1, double v2) {
  return 1.0 / (1.0 - (v0 * v0 + v1 * v1 + v2 * v2) / (kC * kC));
}

// gamma^2 of a proper velocity: 1 + u.u / c^2 (no cancellation)
__device__ __forceinline__ double gamma2_of_u(double u0, double u1, double u2) {
  return 1.0 + (u0 * u0 + u1 * u1 + u2 * u2) / (kC * kC);
}

// Uniform-motion guess of the older bracket node: the source at its present record (q0n, q2n)
// keeps its velocity; c (t - t_r) = [d.beta + sqrt((d.beta)^2 + (1 - beta^2) d^2)] / (1 - beta^2),
// d = r - w_n. Returns a slot index clamped to [k0, n - 1] (requires n > k0).
__device__ __forceinline__ long long uniform_motion_guess(float r0, float r1, float r2, float4 q0n, float4 q2n,
                                                          float3 bref, float inv_cdt, long long k0, long long n) {
  const float d0 = r0 - q0n.x, d1 = r1 - q0n.y, d2 = r2 - q0n.z;
  const float db = d0 * (bref.x + q2n.x) + d1 * (bref.y + q2n.y) + d2 * (bref.z + q2n.z);
  const float dd = d0 * d0 + d1 * d1 + d2 * d2;
  const float ctau = (db + sqrtf(fmaxf(db * db + q0n.w * dd, 0.f))) * q2n.w;
  const float steps = floorf(ctau * inv_cdt);
  long long k = n - 1 - (long long)fminf(fmaxf(steps, 0.f), 1e9f);
  if (k < k0) k = k0;
  if (k > n - 1) k = n - 1;
  return k;
}

}  // namespace emppp
