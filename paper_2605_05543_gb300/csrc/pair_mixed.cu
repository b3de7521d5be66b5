// Mixed-precision all-pairs Lienard-Wiechert kernel (Sec. 2.1-2.2): pair geometry and fields in FP32,
// time stamps, the bracket decision and (in the push) the momentum update in FP64.
//
// Per pair (target i at r = x_i^n, t = t_n; source j):
//   bracket   the node test P(k): (c (t - t_k))^2 <= |r - w_k|^2 is evaluated in FP32 on hi/lo split
//             coordinates; the FP32 margin M = |d|^2 - L^2 carries an error below 8u (|d|^2 + L^2)
//             (u = 2^-24: two roundings in each component of d, three in |d|^2, one in the table value
//             L^2 and one in M), so |M| > kBand (|d|^2 + L^2) with kBand = 32u decides exactly as the
//             FP64 test would; otherwise the FP64 test itself (reference operation order) decides. The
//             bracket is therefore the FP64 one. Search: the paper's bisection or the guarded galloping
//             search from the uniform-motion guess.
//   retarded  in light units (lengths in m, velocities as beta = v/c): with L1 = c (t - t1) and d = r - w1,
//             (1 - beta1^2) s^2 + 2 (d.beta1 - L1) s + (L1^2 - |d|^2) = 0 for s = c (t_r - t1) (eq:dt),
//             smaller root without cancellation; eta = d - beta1 s (eq:linear, retarded position w1 + v1 dt);
//             beta = beta1 + (s / (c dt)) (beta2 - beta1), alpha = a / c^2 = (beta2 - beta1) / (c dt)
//             (eq:linear2 out of history: beta = beta1, alpha = 0); 1 - beta^2 = 1/gamma1^2 - dbeta.(2 beta1
//             + dbeta), so 1 - beta^2 is never formed by cancellation.
//   fields    with u' = eta_hat - beta: E = (q / 4 pi eps0) R [(1 - beta^2) u' + eta x (u' x alpha)] / (eta.u')^3
//             (eq:LW_E with v' = c u', a = c^2 alpha), B = eta_hat x E / c (eq:LW_B).
//   sums      Kahan-compensated FP32 per target, converted to FP64 at the end.
// Targets are taken in the spatial order of order.cu so that a warp's retarded slots of a source are
// close together in the source-major FP32 shadow ring.
#include "emppp_internal.cuh"
#include "shadow.cuh"

namespace emppp {

namespace {

constexpr int kBlock = 128;
constexpr float kBand = 32.0f * 5.9604645e-8f;  // 32 u, u = 2^-24
constexpr double kCoulomb = 1.0 / (4.0 * kPi * kEps0);

struct MixedArgs {
  const float4* __restrict__ rec32;
  const double* __restrict__ rec64;
  const double* __restrict__ lhs64;
  const float* __restrict__ lhs32;
  const float* __restrict__ ct32;
  const float* __restrict__ icdt32;
  const double* __restrict__ wts;
  const int* __restrict__ order;
  const StepState* __restrict__ state;
  double* __restrict__ out;
  double* __restrict__ E;
  double* __restrict__ B;
  unsigned long long* stats;
  int* err;
  long long N;
  int D;
  long long chunk;
};

struct Target {
  float h0, h1, h2, l0, l1, l2;
  double r0, r1, r2;
  bool exact_only;  // coordinates too far from the split origin for the FP32 band: FP64 tests only
};

struct Window {
  long long k0, n;
  int p0, D;
  __device__ __forceinline__ int phys(long long k) const {
    int p = p0 + (int)(k - k0);
    return p >= D ? p - D : p;
  }
};

__device__ __forceinline__ bool exact_test(const Target& r, const double* __restrict__ w, double lhs) {
  const double d0 = __dsub_rn(r.r0, __ldg(w + 0));
  const double d1 = __dsub_rn(r.r1, __ldg(w + 1));
  const double d2 = __dsub_rn(r.r2, __ldg(w + 2));
  const double rhs = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
  return lhs <= rhs;
}

// P(k) at physical slot p of the source whose rings start at src32 / src64
__device__ __forceinline__ bool node_test(const Target& r, const float4* __restrict__ src32,
                                          const double* __restrict__ src64, int p, const MixedArgs& a,
                                          unsigned& n_fb) {
  const float4 q0 = __ldg(src32 + 3 * p);
  const float4 q1 = __ldg(src32 + 3 * p + 1);
  const float d0 = (r.h0 - q0.x) + (r.l0 - q1.x);
  const float d1 = (r.h1 - q0.y) + (r.l1 - q1.y);
  const float d2 = (r.h2 - q0.z) + (r.l2 - q1.z);
  const float D2 = d0 * d0 + d1 * d1 + d2 * d2;
  const float L2 = __ldg(a.lhs32 + p);
  const float M = D2 - L2;
  const float band = kBand * (D2 + L2);
  if (!r.exact_only) {
    if (M > band) return true;
    if (M < -band) return false;
  }
  n_fb++;
  return exact_test(r, src64 + 6 * p, __ldg(a.lhs64 + p));
}

}  // namespace

template <int PROP>
__global__ void __launch_bounds__(kBlock) pair_mixed_kernel(MixedArgs a) {
  const long long N = a.N;
  const int D = a.D;
  const long long t = (long long)blockIdx.x * kBlock + threadIdx.x;
  const bool active = t < N;
  const long long i = active ? (a.order ? (long long)a.order[t] : t) : 0;

  Window win;
  win.n = a.state->n;
  win.k0 = a.state->k0;
  win.p0 = a.state->p0;
  win.D = D;
  const int pn = a.state->pn;
  const float inv_cdt = (float)(1.0 / (kC * a.state->dt));

  Target r;
  {
    const float4 q0 = a.rec32[((size_t)i * D + pn) * 3];
    const float4 q1 = a.rec32[((size_t)i * D + pn) * 3 + 1];
    r.h0 = q0.x;
    r.h1 = q0.y;
    r.h2 = q0.z;
    r.l0 = q1.x;
    r.l1 = q1.y;
    r.l2 = q1.z;
    const double* rr = a.rec64 + ((size_t)i * D + pn) * 6;
    r.r0 = rr[0];
    r.r1 = rr[1];
    r.r2 = rr[2];
    r.exact_only = fmaxf(fabsf(r.h0), fmaxf(fabsf(r.h1), fabsf(r.h2))) > 0.5f;
  }

  const long long j_begin = (long long)blockIdx.y * a.chunk;
  const long long j_end = min(N, j_begin + a.chunk);

  float Es[3] = {0.f, 0.f, 0.f}, Ec[3] = {0.f, 0.f, 0.f}, Bs[3] = {0.f, 0.f, 0.f}, Bc[3] = {0.f, 0.f, 0.f};
  unsigned n_ooh = 0, n_sc = 0, n_bi = 0, n_tests = 0, n_fb = 0;
  int errbits = 0;
  const float kq_unit = (float)(-kQe * kCoulomb);

  for (long long j = j_begin; active && j < j_end; ++j) {
    if (j == i) continue;
    const float4* src32 = a.rec32 + (size_t)j * D * 3;
    const double* src64 = a.rec64 + (size_t)j * D * 6;
    // ---- bracket --------------------------------------------------------------------------------
    long long k1;
    int br;
    if (PROP == kPropBisect) {
      n_tests += 1;
      if (node_test(r, src32, src64, win.p0, a, n_fb)) {
        k1 = win.k0;
        br = 0;
      } else {
        n_tests += 1;
        if (!node_test(r, src32, src64, win.phys(win.n - 1), a, n_fb)) {
          k1 = win.n - 1;
          br = 1;
        } else {
          long long lo = win.k0, hi = win.n;
          while (hi - lo > 1) {
            const long long m = (lo + hi) >> 1;
            n_tests += 1;
            if (node_test(r, src32, src64, win.phys(m), a, n_fb))
              hi = m;
            else
              lo = m;
          }
          k1 = lo;
          br = 2;
        }
      }
    } else {
      if (win.n == win.k0) {
        k1 = win.k0;
        br = 0;
        n_tests += 1;
      } else {
        const long long kg = uniform_motion_guess(r.h0, r.h1, r.h2, __ldg(src32 + 3 * pn), __ldg(src32 + 3 * pn + 2),
                                                  inv_cdt, win.k0, win.n);
        long long lo = kg, hi = kg;
        bool ooh = false;
        n_tests += 1;
        if (node_test(r, src32, src64, win.phys(kg), a, n_fb)) {
          long long s = 1;
          for (;;) {
            if (hi == win.k0) {
              ooh = true;
              break;
            }
            lo = hi - s;
            if (lo < win.k0) lo = win.k0;
            n_tests += 1;
            if (!node_test(r, src32, src64, win.phys(lo), a, n_fb)) break;
            hi = lo;
            s <<= 1;
          }
        } else {
          long long s = 1;
          for (;;) {
            hi = lo + s;
            if (hi >= win.n) {
              hi = win.n;
              break;
            }
            n_tests += 1;
            if (node_test(r, src32, src64, win.phys(hi), a, n_fb)) break;
            lo = hi;
            s <<= 1;
          }
        }
        if (ooh) {
          k1 = win.k0;
          br = 0;
        } else {
          while (hi - lo > 1) {
            const long long m = (lo + hi) >> 1;
            n_tests += 1;
            if (node_test(r, src32, src64, win.phys(m), a, n_fb))
              hi = m;
            else
              lo = m;
          }
          k1 = lo;
          br = (k1 == win.n - 1) ? 1 : 2;
        }
      }
    }
    if (br == 0)
      n_ooh++;
    else if (br == 1)
      n_sc++;
    else
      n_bi++;

    // ---- retarded state (light units) --------------------------------------------------------------
    const int p1 = win.phys(k1);
    const float4 q0 = __ldg(src32 + 3 * p1);
    const float4 q1 = __ldg(src32 + 3 * p1 + 1);
    const float4 q2 = __ldg(src32 + 3 * p1 + 2);
    const float d0 = (r.h0 - q0.x) + (r.l0 - q1.x);
    const float d1 = (r.h1 - q0.y) + (r.l1 - q1.y);
    const float d2 = (r.h2 - q0.z) + (r.l2 - q1.z);
    const float L1 = __ldg(a.ct32 + p1);
    const float b10 = q2.x, b11 = q2.y, b12 = q2.z;
    const float ig2 = q0.w, g2 = q2.w;
    const float hb = (d0 * b10 + d1 * b11 + d2 * b12) - L1;
    const float C0 = fmaf(L1, L1, -(d0 * d0 + d1 * d1 + d2 * d2));
    const float qd = fmaf(hb, hb, -ig2 * C0);
    if (!(qd >= 0.f) || !(ig2 > 0.f)) {
      errbits |= kErrDisc;
      continue;
    }
    const float sq = qd > 0.f ? qd * rsqrtf(qd) : 0.f;
    const float s = (hb <= 0.f) ? __fdividef(C0, sq - hb) : -(hb + sq) * g2;
    const float e0 = fmaf(-b10, s, d0), e1 = fmaf(-b11, s, d1), e2 = fmaf(-b12, s, d2);
    float be0 = b10, be1 = b11, be2 = b12, al0 = 0.f, al1 = 0.f, al2 = 0.f, ug = ig2;
    if (br != 0) {
      const int p2 = p1 + 1 == D ? 0 : p1 + 1;
      const float4 q2b = __ldg(src32 + 3 * p2 + 2);
      const float icdt = __ldg(a.icdt32 + p1);
      const float db0 = q2b.x - b10, db1 = q2b.y - b11, db2 = q2b.z - b12;
      al0 = db0 * icdt;
      al1 = db1 * icdt;
      al2 = db2 * icdt;
      const float df = s * icdt;
      const float x0 = db0 * df, x1 = db1 * df, x2 = db2 * df;
      be0 = b10 + x0;
      be1 = b11 + x1;
      be2 = b12 + x2;
      ug = ig2 - (x0 * (2.f * b10 + x0) + x1 * (2.f * b11 + x1) + x2 * (2.f * b12 + x2));
    }
    // ---- Lienard-Wiechert fields -------------------------------------------------------------------
    const float R2 = e0 * e0 + e1 * e1 + e2 * e2;
    const float invR = rsqrtf(R2);
    const float R = R2 * invR;
    const float n0 = e0 * invR, n1 = e1 * invR, n2 = e2 * invR;
    const float u0 = n0 - be0, u1 = n1 - be1, u2 = n2 - be2;
    const float eu = R - (e0 * be0 + e1 * be1 + e2 * be2);
    if (!(R2 > 0.f) || !(eu > 0.f)) {
      errbits |= kErrCoincide;
      continue;
    }
    const float ieu = __fdividef(1.f, eu);
    const float kq = kq_unit * (float)__ldg(a.wts + j);
    const float pref = kq * (R * ieu) * ieu * ieu;
    // eta x (u' x alpha)
    const float c0 = u1 * al2 - u2 * al1, c1 = u2 * al0 - u0 * al2, c2 = u0 * al1 - u1 * al0;
    const float F0 = fmaf(ug, u0, e1 * c2 - e2 * c1);
    const float F1 = fmaf(ug, u1, e2 * c0 - e0 * c2);
    const float F2 = fmaf(ug, u2, e0 * c1 - e1 * c0);
    const float E0 = pref * F0, E1 = pref * F1, E2 = pref * F2;
    const float ic = (float)(1.0 / kC);
    const float B0 = (n1 * E2 - n2 * E1) * ic, B1 = (n2 * E0 - n0 * E2) * ic, B2 = (n0 * E1 - n1 * E0) * ic;
    // ---- Kahan-compensated sums ---------------------------------------------------------------------
    const float xs[6] = {E0, E1, E2, B0, B1, B2};
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const float y = xs[c] - Ec[c];
      const float tt = Es[c] + y;
      Ec[c] = (tt - Es[c]) - y;
      Es[c] = tt;
      const float yb = xs[3 + c] - Bc[c];
      const float tb = Bs[c] + yb;
      Bc[c] = (tb - Bs[c]) - yb;
      Bs[c] = tb;
    }
  }
  if (active) {
    double Et[3], Bt[3];
    for (int c = 0; c < 3; c++) {
      Et[c] = (double)Es[c] - (double)Ec[c];
      Bt[c] = (double)Bs[c] - (double)Bc[c];
    }
    if (gridDim.y == 1) {
      for (int c = 0; c < 3; c++) {
        a.E[3 * i + c] = Et[c];
        a.B[3 * i + c] = Bt[c];
      }
    } else {
      double* o = a.out + ((size_t)blockIdx.y * N + i) * 6;
      for (int c = 0; c < 3; c++) {
        o[c] = Et[c];
        o[3 + c] = Bt[c];
      }
    }
  }
  n_ooh = __reduce_add_sync(0xffffffffu, n_ooh);
  n_sc = __reduce_add_sync(0xffffffffu, n_sc);
  n_bi = __reduce_add_sync(0xffffffffu, n_bi);
  n_tests = __reduce_add_sync(0xffffffffu, n_tests);
  n_fb = __reduce_add_sync(0xffffffffu, n_fb);
  errbits = __reduce_or_sync(0xffffffffu, errbits);
  if ((threadIdx.x & 31) == 0) {
    if (n_ooh) atomicAdd(a.stats + kStatOOH, (unsigned long long)n_ooh);
    if (n_sc) atomicAdd(a.stats + kStatShortcut, (unsigned long long)n_sc);
    if (n_bi) atomicAdd(a.stats + kStatBisect, (unsigned long long)n_bi);
    if (n_tests) atomicAdd(a.stats + kStatNodeTests, (unsigned long long)n_tests);
    if (n_fb) atomicAdd(a.stats + kStatGuard, (unsigned long long)n_fb);
    if (errbits) atomicOr(a.err, errbits);
  }
}

cudaError_t launch_pair_mixed(const DeviceState& s, const int* order, int proposal, int split, cudaStream_t st) {
  MixedArgs a;
  a.rec32 = reinterpret_cast<const float4*>(s.rec32);
  a.rec64 = s.rec64;
  a.lhs64 = s.tab.lhs64;
  a.lhs32 = s.tab.lhs32;
  a.ct32 = s.tab.ct32;
  a.icdt32 = s.tab.icdt32;
  a.wts = s.wts;
  a.order = order;
  a.state = s.state;
  a.out = s.partial;
  a.E = s.Eself;
  a.B = s.Bself;
  a.stats = s.stats;
  a.err = s.err;
  a.N = s.N;
  a.D = s.D;
  if (split < 1) split = 1;
  a.chunk = (s.N + split - 1) / split;
  dim3 grid((unsigned)((s.N + kBlock - 1) / kBlock), (unsigned)split);
  if (proposal == kPropClosedForm)
    pair_mixed_kernel<kPropClosedForm><<<grid, kBlock, 0, st>>>(a);
  else
    pair_mixed_kernel<kPropBisect><<<grid, kBlock, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace emppp
