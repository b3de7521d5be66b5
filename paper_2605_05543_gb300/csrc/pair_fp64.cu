// FP64 all-pairs Lienard-Wiechert field evaluation with the retarded-time solve (Sec. 2.1-2.2).
//
// One thread owns one target i (present position r = x_i^n at t = t_n) and walks the sources j of
// its slice. Per pair:
//   1. bracket the retarded time in j's history with the node test
//        P(k):  (c (t - t_k))^2 <= |r - w_{j,k}|^2       (true: t_r at or before t_k)
//      evaluated in FP32 on the shadow ring's hi/lo split against guard-band thresholds of the slot
//      tables, and in FP64 in the reference operation order between them (so decisions agree bit for
//      bit): out-of-history if P(k0), near-field shortcut if not P(n-1), else bisection (Sec. 2.2);
//      or, with the closed-form proposal, a guarded galloping search started at the slot predicted
//      by uniform motion from j's present state. Both return the unique sign change of P.
//   2. linear reconstruction (eq:dt, eq:linear): delta t from the quadratic, w = w1 + v1 dt,
//      v = v1 + (dt / (t2 - t1)) (v2 - v1), a = (v2 - v1) / (t2 - t1); or, in the comparison variant MID,
//      the bracket's midpoint values of eq:mid.
//   3. Lienard-Wiechert E (eq:LW_E) and B = eta_hat x E / c (eq:LW_B), summed over j != i in
//      blocks of kSumBlock sources (blocked summation keeps the FP64 rounding error of a 65536-term
//      sum near 1e-14 of the sum of magnitudes).
//   Out of history (eq:linear2) the source moves uniformly with v1 along the line through w_{k0}, and its
//   Lienard-Wiechert field is Heaviside's field about the line's point at t_n: with X = r - w_{k0} -
//   v1 (t_n - t_{k0}), E = kq c (c^2 - v1^2) X / [|X|^2 (c^2 - v1^2) + (X.v1)^2]^{3/2}, B = v1 x E / c^2.
//   It is the same field, without the quadratic and the retarded reconstruction.
// Targets are taken in the spatial order of order.cu (when given), so that the pairs of a warp mostly
// take the same branch; which thread evaluates a target does not change its result.
// The arithmetic is FP64-pipe bound (GB300: 2 DFMA/clk/SM); everything that is not an FP64 result
// (the guess, the node tests outside the guard band, indices, loads) runs on the FP32/INT pipes beside it.
#include "../../include/emppp.h"
#include "emppp_internal.cuh"
#include "mlp.cuh"
#include "shadow.cuh"

namespace emppp {

namespace {

constexpr int kSumBlock = 64;
constexpr double kCoulomb = 1.0 / (4.0 * kPi * kEps0);
// the sums run over w_j-weighted fields without the electron's charge constant -e / (4 pi eps0), and over
// c^2 B; both are scaled once per target
constexpr double kFieldScale = -kQe * kCoulomb;

// 1 / x for finite x > 0: the hardware's approximate reciprocal refined by two Newton-Raphson steps
// y <- y + y (1 - x y). Each step squares the relative error, so the approximation's error falls below
// FP64 rounding after two steps (within a few units in the last place, not correctly rounded), for
// five FP64-pipe operations instead of a correctly rounded division.
__device__ __forceinline__ double recip_newton(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}


struct PairArgs {
  const double* __restrict__ rec64;
  const float* __restrict__ rec32;
  const double* __restrict__ slot_t;
  const double* __restrict__ lhs64;
  const float4* __restrict__ tab32;  // per slot: FP32 guard-band thresholds of (c (t_n - t_k))^2
  const double* __restrict__ inv_dtk;
  const double* __restrict__ wts;
  const StepState* __restrict__ state;
  double* __restrict__ out;  // [S][N][6] (S = 1: [N][6] temporary) -- see launch
  double* __restrict__ E;
  double* __restrict__ B;
  unsigned long long* stats;
  int* err;
  long long N;
  int D;
  int nbunch;
  const BunchDesc* __restrict__ bunches;
  const BunchSched* __restrict__ sched;
  int nitems;  // work items of all bunches
  int* work;   // work-item counter (zero at launch)
  const mlp::InferImage* __restrict__ net;  // proposal network, inference form (EMPPP_PROPOSAL_MLP)
  unsigned long long* scale;  // adaptive time step: eta_min / v_max^2 reduction
  double eta_allow;
  const int* __restrict__ order;  // spatial order of the targets (nullptr: index order)
  int* __restrict__ dump;  // [N][N] bracket of every evaluated pair, 4 (k1 - k0) + branch (DUMP instances only)
};

// node test P(k) with the reference operation order (no contraction)
__device__ __forceinline__ bool node_test(double r0, double r1, double r2, const double* __restrict__ w,
                                          double lhs) {
  const double d0 = __dsub_rn(r0, __ldg(w + 0));
  const double d1 = __dsub_rn(r1, __ldg(w + 1));
  const double d2 = __dsub_rn(r2, __ldg(w + 2));
  const double rhs = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
  return lhs <= rhs;
}

struct Window {
  long long k0, n;
  int p0, D;
  int* err;  // device error word (the debug build's range checks)
  __device__ __forceinline__ int phys(long long k) const {
    int p = p0 + (int)(debug_index(k, k0, n + 1, err) - k0);
    return p >= D ? p - D : p;
  }
};

}  // namespace

// SHAPE: targets per block (kBlock = shape_block(SHAPE); shapes 3 and 4 run as shape 0)
template <int PROP, bool ADAPT, bool MID, bool DUMP, int SHAPE>
__global__ void __launch_bounds__(shape_block(SHAPE)) pair_fp64_kernel(PairArgs a) {
  constexpr int kBlock = shape_block(SHAPE);
  __shared__ int s_item;
  const long long N = a.N;
  const int D = a.D;

  Window win;
  win.n = a.state->n;
  win.k0 = a.state->k0;
  win.p0 = a.state->p0;
  win.D = D;
  win.err = a.err;
  const int pn = a.state->pn;
  const double t = a.state->t;
  const float inv_cdt = PROP != kPropBisect ? (float)(1.0 / (kC * a.state->dt)) : 0.f;
  const float invL = (float)(1.0 / (kC * a.state->dt * D));
  const int pprev = win.n > win.k0 ? win.phys(win.n - 1) : pn;  // slot n - 1 (or n)

  unsigned n_ooh = 0, n_sc = 0, n_bi = 0, n_tests = 0, n_fb = 0;
  double emin = __longlong_as_double(0x7ff0000000000000LL), vmax2 = 0.0;  // adaptive time step (Sec. 2.4)
  int errbits = 0;

  // persistent blocks pull (source chunk, target tile) items, chunk-major, until none is left
  for (;;) {
  __syncthreads();
  if (threadIdx.x == 0) s_item = atomicAdd(a.work, 1);
  __syncthreads();
  const int item = s_item;
  if (item >= a.nitems) break;
  int b, chunk_id, tb;
  decode_item(a.sched, a.nbunch, item, b, chunk_id, tb);
  const BunchDesc& bd = a.bunches[b];
  const BunchSched& bs = a.sched[b];
  const float3 bref = make_float3((float)bd.beta_ref[0], (float)bd.beta_ref[1], (float)bd.beta_ref[2]);
  const long long i_loc = (long long)tb * kBlock + threadIdx.x;
  const bool active = i_loc < bd.n;
  const long long i = debug_index<long long>(a.order ? a.order[bd.off + (active ? i_loc : 0)] : bd.off + (active ? i_loc : 0),
                                            bd.off, bd.off + bd.n, a.err);
  const long long ic = i;

  const double* rr = a.rec64 + ((size_t)ic * D + pn) * 6;
  const double r0 = rr[0], r1 = rr[1], r2 = rr[2];
  const double vi0 = ADAPT ? rr[3] : 0.0, vi1 = ADAPT ? rr[4] : 0.0, vi2 = ADAPT ? rr[5] : 0.0;  // v_i(t_n)
  // FP32 hi/lo split of the target's position: node tests run in FP32 against the guard-band thresholds
  // of the slot tables and fall back to the FP64 test between them (the decision is the FP64 one)
  const float* tq = a.rec32 + ((size_t)ic * D + pn) * 12;
  const float rh0 = tq[0], rh1 = tq[1], rh2 = tq[2];
  const float rl0 = tq[4], rl1 = tq[5], rl2 = tq[6];
  const bool far_target = fmaxf(fabsf(rh0), fmaxf(fabsf(rh1), fabsf(rh2))) > 0.5f;
  // learned proposal: the mean position of the warp's targets, where the network is evaluated
  float3 rc = make_float3(0.f, 0.f, 0.f);
  if (PROP == kPropMlp) rc = mlp::warp_mean(active, rh0, rh1, rh2);
  float fac_lane = 1.f;  // delay factor of source j0 + lane of the current group of 32

  const long long j_begin = bd.off + (long long)chunk_id * bs.chunk;
  const long long j_end = min(bd.off + bd.n, j_begin + bs.chunk);

  double Et[3] = {0, 0, 0}, Bt[3] = {0, 0, 0};
  double Ep[3] = {0, 0, 0}, Bp[3] = {0, 0, 0};
  int in_block = 0;

  const double c2 = kC * kC;
  for (long long j = j_begin; (PROP == kPropMlp || active) && j < j_end; ++j) {
    float fac = 1.f;
    if (PROP == kPropMlp) {
      // every 32 sources, the warp evaluates the network for the next 32 (one per lane) at its mean target
      // position; each pair then scales its uniform-motion delay by its source's factor
      const int l = (int)((j - j_begin) & 31);
      if (l == 0) {
        __syncwarp();
        const long long js = j + (threadIdx.x & 31);
        const bool v = js < j_end;
        const long long jr = v ? js : j;
        const float4* qn = reinterpret_cast<const float4*>(a.rec32 + ((size_t)jr * D + pn) * 12);
        const float4 q0n = __ldg(qn), q2n = __ldg(qn + 2);
        const float4 q2p = __ldg(reinterpret_cast<const float4*>(a.rec32 + ((size_t)jr * D + pprev) * 12) + 2);
        fac_lane = mlp::warp_delay_factor(*a.net, v, rc.x - q0n.x, rc.y - q0n.y, rc.z - q0n.z, bref.x + q2n.x,
                                          bref.y + q2n.y, bref.z + q2n.z, q2n.x - q2p.x, q2n.y - q2p.y,
                                          q2n.z - q2p.z, invL, (float)D);
      }
      fac = __shfl_sync(0xffffffffu, fac_lane, l);
    }
    if (!active) continue;  // and stay in the loop for the next group's evaluation
    if (j == i) continue;
    const long long jc = debug_index(j, bd.off, bd.off + bd.n, a.err);  // j itself in a release build
    const double* src = a.rec64 + (size_t)jc * D * 6;
    const float4* src32 = reinterpret_cast<const float4*>(a.rec32 + (size_t)jc * D * 12);
    // P(k) at physical slot p: FP32 on the hi/lo split outside the guard band, else the FP64 test
    auto ntest = [&](int p) -> bool {
      const float4 q0 = __ldg(src32 + 3 * p), q1 = __ldg(src32 + 3 * p + 1);
      const float d0 = (rh0 - q0.x) + (rl0 - q1.x), d1 = (rh1 - q0.y) + (rl1 - q1.y), d2 = (rh2 - q0.z) + (rl2 - q1.z);
      const float D2 = d0 * d0 + d1 * d1 + d2 * d2;
      const float4 tb = __ldg(a.tab32 + p);
      if (!far_target) {
        if (D2 > tb.x) return true;
        if (D2 < tb.y) return false;
      }
      n_fb += 1;
      return node_test(r0, r1, r2, src + p * 6, __ldg(a.lhs64 + p));
    };
    // ---- 1. bracket ------------------------------------------------------------------------
    long long k1;
    int br;
    if (PROP == kPropBisect) {
      n_tests += 1;
      if (ntest(win.p0)) {
        k1 = win.k0;
        br = 0;
      } else {
        n_tests += 1;
        const int pm1 = win.phys(win.n - 1);
        if (!ntest(pm1)) {
          k1 = win.n - 1;
          br = 1;
        } else {
          long long lo = win.k0, hi = win.n;
          while (hi - lo > 1) {
            const long long m = (lo + hi) >> 1;
            const int pm = win.phys(m);
            n_tests += 1;
            if (ntest(pm))
              hi = m;
            else
              lo = m;
          }
          k1 = lo;
          br = 2;
        }
      }
    } else {
      // guarded galloping search from the closed-form guess
      if (win.n == win.k0) {
        k1 = win.k0;
        br = 0;
        n_tests += 1;
      } else {
        // the uniform-motion delay (scaled by the network's factor with the learned proposal)
        const float4* qn = reinterpret_cast<const float4*>(a.rec32 + ((size_t)j * D + pn) * 12);
        const long long kg = uniform_motion_guess(rh0, rh1, rh2, __ldg(qn), __ldg(qn + 2), bref,
                                                  PROP == kPropMlp ? inv_cdt * fac : inv_cdt, win.k0, win.n);
        long long lo, hi;
        bool ooh = false;
        n_tests += 1;
        int pg = win.phys(kg);
        if (ntest(pg)) {
          hi = kg;
          long long s = 1;
          for (;;) {
            if (hi == win.k0) {
              ooh = true;
              break;
            }
            lo = hi - s;
            if (lo < win.k0) lo = win.k0;
            const int pl = win.phys(lo);
            n_tests += 1;
            if (!ntest(pl)) break;
            hi = lo;
            s <<= 1;
          }
        } else {
          lo = kg;
          long long s = 1;
          for (;;) {
            hi = lo + s;
            if (hi >= win.n) {
              hi = win.n;
              break;
            }
            const int ph = win.phys(hi);
            n_tests += 1;
            if (ntest(ph)) break;
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
            const int pm = win.phys(m);
            n_tests += 1;
            if (ntest(pm))
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
    if (DUMP) a.dump[(size_t)i * N + j] = 4 * (int)(k1 - win.k0) + br;

    // ---- 2. reconstruction (eq:dt, eq:linear; eq:mid in the MID variant) ----------------------
    const int p1 = win.phys(k1);
    const double2* R1 = reinterpret_cast<const double2*>(src + p1 * 6);
    const double2 x01 = __ldg(R1), x23 = __ldg(R1 + 1), x45 = __ldg(R1 + 2);
    const double w10 = x01.x, w11 = x01.y, w12 = x23.x;
    const double v10 = x23.y, v11 = x45.x, v12 = x45.y;
    if (br == 0) {
      // ---- out of history (eq:linear2): Heaviside's field of the uniformly moving source -------
      const double T1 = t - __ldg(a.slot_t + p1);
      const double X0 = (r0 - w10) - v10 * T1, X1 = (r1 - w11) - v11 * T1, X2 = (r2 - w12) - v12 * T1;
      const double c2mv2 = c2 - (v10 * v10 + v11 * v11 + v12 * v12);
      const double XX = X0 * X0 + X1 * X1 + X2 * X2;
      const double Xv = X0 * v10 + X1 * v11 + X2 * v12;
      const double Dh = XX * c2mv2 + Xv * Xv;  // c^2 [|X|^2 (1 - beta^2) + (X.beta)^2]
      if (!(c2mv2 > 0.0)) {
        errbits |= kErrDisc;
        continue;
      }
      if (!(Dh > 0.0)) {
        errbits |= kErrCoincide;
        continue;
      }
      const double iD = rsqrt(Dh);
      // E / (-e / (4 pi eps0)): the source's charge constant is applied once per target (kFieldScale)
      const double pref = (kC * __ldg(a.wts + j)) * c2mv2 * (iD * iD * iD);
      const double E0 = pref * X0, E1 = pref * X1, E2 = pref * X2;
      if (ADAPT) {
        // retarded distance R = c (t - t_r), the positive root of R^2 (c^2 - v^2) - 2 R c (X.v) - c^2 |X|^2
        // = 0, formed without cancellation; v(t_r) = v1
        const double sD = Dh * iD;
        const double R = (Xv >= 0.0) ? kC * (Xv + sD) / c2mv2 : kC * XX / (sD - Xv);
        if (R >= a.eta_allow) {
          emin = fmin(emin, R);
          const double dv0 = vi0 - v10, dv1 = vi1 - v11, dv2 = vi2 - v12;
          vmax2 = fmax(vmax2, dv0 * dv0 + dv1 * dv1 + dv2 * dv2);
        }
      }
      // c^2 B = v x E (the 1 / c^2 is applied once per target)
      Ep[0] += E0;
      Ep[1] += E1;
      Ep[2] += E2;
      Bp[0] += v11 * E2 - v12 * E1;
      Bp[1] += v12 * E0 - v10 * E2;
      Bp[2] += v10 * E1 - v11 * E0;
      if (++in_block == kSumBlock) {
        in_block = 0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          Et[c] += Ep[c];
          Bt[c] += Bp[c];
          Ep[c] = 0.0;
          Bp[c] = 0.0;
        }
      }
      continue;
    }
    double w0, w1, w2, v0 = v10, v1 = v11, v2 = v12, a0 = 0.0, a1 = 0.0, a2 = 0.0;
    if (MID && br != 0) {
      // eq:mid: the midpoint of the bracket stands for the retarded time
      const int p2 = p1 + 1 == D ? 0 : p1 + 1;
      const double2* R2 = reinterpret_cast<const double2*>(src + p2 * 6);
      const double2 y01 = __ldg(R2), y23 = __ldg(R2 + 1), y45 = __ldg(R2 + 2);
      const double idt = __ldg(a.inv_dtk + p1);
      w0 = 0.5 * (w10 + y01.x);
      w1 = 0.5 * (w11 + y01.y);
      w2 = 0.5 * (w12 + y23.x);
      v0 = 0.5 * (v10 + y23.y);
      v1 = 0.5 * (v11 + y45.x);
      v2 = 0.5 * (v12 + y45.y);
      a0 = (y23.y - v10) * idt;
      a1 = (y45.x - v11) * idt;
      a2 = (y45.y - v12) * idt;
    } else {
      const double T1 = t - __ldg(a.slot_t + p1);
      const double d0 = r0 - w10, d1 = r1 - w11, d2 = r2 - w12;
      const double C2 = c2 - (v10 * v10 + v11 * v11 + v12 * v12);
      const double hb = (d0 * v10 + d1 * v11 + d2 * v12) - c2 * T1;  // C1 / 2
      const double C0 = c2 * T1 * T1 - (d0 * d0 + d1 * d1 + d2 * d2);
      const double qd = hb * hb - C2 * C0;  // disc / 4
      if (!(C2 > 0.0) || !(qd >= 0.0)) {
        errbits |= kErrDisc;
        continue;
      }
      const double sq = qd * rsqrt(fmax(qd, 1e-300));  // sqrt(qd); the reciprocal root costs fewer FP64-pipe operations
      // smaller root of C2 x^2 + 2 hb x + C0 without cancellation
      const double dt = (hb <= 0.0) ? C0 * recip_newton(sq - hb) : -(hb + sq) * recip_newton(C2);
      w0 = w10 + v10 * dt;
      w1 = w11 + v11 * dt;
      w2 = w12 + v12 * dt;
      if (br != 0) {
        const int p2 = p1 + 1 == D ? 0 : p1 + 1;
        const double2* R2 = reinterpret_cast<const double2*>(src + p2 * 6);
        const double2 y23 = __ldg(R2 + 1), y45 = __ldg(R2 + 2);
        const double idt = __ldg(a.inv_dtk + p1);
        a0 = (y23.y - v10) * idt;
        a1 = (y45.x - v11) * idt;
        a2 = (y45.y - v12) * idt;
        v0 = v10 + dt * a0;
        v1 = v11 + dt * a1;
        v2 = v12 + dt * a2;
      }
    }
    // ---- 3. Lienard-Wiechert fields ----------------------------------------------------------
    const double e0 = r0 - w0, e1 = r1 - w1, e2 = r2 - w2;
    const double R2s = e0 * e0 + e1 * e1 + e2 * e2;
    const double invR = rsqrt(R2s);
    const double R = R2s * invR;
    const double cinvR = kC * invR;
    const double vp0 = e0 * cinvR - v0, vp1 = e1 * cinvR - v1, vp2 = e2 * cinvR - v2;
    const double evp = e0 * vp0 + e1 * vp1 + e2 * vp2;
    if (!(R2s > 0.0) || !(evp > 0.0)) {
      errbits |= kErrCoincide;
      continue;
    }
    const double c2mv2 = c2 - (v0 * v0 + v1 * v1 + v2 * v2);
    // eta x (v' x a)
    const double xa0 = vp1 * a2 - vp2 * a1, xa1 = vp2 * a0 - vp0 * a2, xa2 = vp0 * a1 - vp1 * a0;
    const double ac0 = e1 * xa2 - e2 * xa1, ac1 = e2 * xa0 - e0 * xa2, ac2 = e0 * xa1 - e1 * xa0;
    const double ievp = recip_newton(evp);
    const double pref = (__ldg(a.wts + j) * R) * (ievp * ievp * ievp);  // charge constant once per target
    const double E0 = pref * (c2mv2 * vp0 + ac0), E1 = pref * (c2mv2 * vp1 + ac1), E2 = pref * (c2mv2 * vp2 + ac2);
    const double bs = invR * kC;  // c^2 B = c eta_hat x E
    if (ADAPT && R >= a.eta_allow) {
      // interaction scale of the adaptive step: |eta_ij| and |v_i(t_n) - v_j(t_r)|
      emin = fmin(emin, R);
      const double dv0 = vi0 - v0, dv1 = vi1 - v1, dv2 = vi2 - v2;
      vmax2 = fmax(vmax2, dv0 * dv0 + dv1 * dv1 + dv2 * dv2);
    }
    Ep[0] += E0;
    Ep[1] += E1;
    Ep[2] += E2;
    Bp[0] += (e1 * E2 - e2 * E1) * bs;
    Bp[1] += (e2 * E0 - e0 * E2) * bs;
    Bp[2] += (e0 * E1 - e1 * E0) * bs;
    if (++in_block == kSumBlock) {
      in_block = 0;
#pragma unroll
      for (int c = 0; c < 3; c++) {
        Et[c] += Ep[c];
        Bt[c] += Bp[c];
        Ep[c] = 0.0;
        Bp[c] = 0.0;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; c++) {
    Et[c] = (Et[c] + Ep[c]) * kFieldScale;
    Bt[c] = (Bt[c] + Bp[c]) * (kFieldScale / (kC * kC));
  }
  if (active) {
    if (bs.nchunk == 1) {
      for (int c = 0; c < 3; c++) {
        a.E[3 * i + c] = Et[c];
        a.B[3 * i + c] = Bt[c];
      }
    } else {
      double* o = a.out + ((size_t)chunk_id * N + i) * 6;
      for (int c = 0; c < 3; c++) {
        o[c] = Et[c];
        o[3 + c] = Bt[c];
      }
    }
  }
  if (ADAPT) {
    // this item's interaction scale into its bunch's slots (every lane of the warp takes part)
    reduce_scale(a.scale + 2 * b, emin, vmax2);
    emin = __longlong_as_double(0x7ff0000000000000LL);
    vmax2 = 0.0;
  }
  }  // work items
  // counters: one atomic per warp and counter
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

// E_i = sum over the source chunks c of partial[c][i] (fixed order), for bunches split in chunks
__global__ void reduce_partials_kernel(const double* __restrict__ part, const BunchSched* __restrict__ sched,
                                       const int* __restrict__ bunch_of, long long N, double* __restrict__ E,
                                       double* __restrict__ B) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int S = sched[bunch_of[i]].nchunk;
  if (S == 1) return;  // written directly by the pair kernel
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int c = 0; c < S; c++) {
    const double* o = part + ((size_t)c * N + i) * 6;
#pragma unroll
    for (int k = 0; k < 6; k++) acc[k] += o[k];
  }
  for (int c = 0; c < 3; c++) {
    E[3 * i + c] = acc[c];
    B[3 * i + c] = acc[3 + c];
  }
}

__global__ void zero_kernel(double* __restrict__ a, double* __restrict__ b, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    a[i] = 0.0;
    b[i] = 0.0;
  }
}

template <bool ADAPT, bool MID, int SHAPE>
int max_blocks_fp64(int proposal) {
  int nb = 0;
  constexpr int B = shape_block(SHAPE);
  if (proposal == kPropClosedForm)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_fp64_kernel<kPropClosedForm, ADAPT, MID, false, SHAPE>, B, 0);
  else if (proposal == kPropMlp)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_fp64_kernel<kPropMlp, ADAPT, MID, false, SHAPE>, B, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_fp64_kernel<kPropBisect, ADAPT, MID, false, SHAPE>, B, 0);
  return nb > 0 ? nb : 1;
}

// the adaptive-step and eq:mid instances and the bracket dump run the default shape only
int max_blocks_pair_fp64(int proposal, int variant, int shape) {
  if (variant == 2) return max_blocks_fp64<false, true, 0>(proposal);
  if (variant == 1) return max_blocks_fp64<true, false, 0>(proposal);
  if (shape == 1) return max_blocks_fp64<false, false, 1>(proposal);
  if (shape == 2) return max_blocks_fp64<false, false, 2>(proposal);
  return max_blocks_fp64<false, false, 0>(proposal);
}

template <bool ADAPT, bool MID, bool DUMP, int SHAPE>
void launch_fp64(int proposal, const PairLaunch& pl, const PairArgs& a, cudaStream_t st) {
  constexpr int B = shape_block(SHAPE);
  if (proposal == kPropClosedForm)
    pair_fp64_kernel<kPropClosedForm, ADAPT, MID, DUMP, SHAPE><<<pl.grid, B, 0, st>>>(a);
  else if (proposal == kPropMlp)
    pair_fp64_kernel<kPropMlp, ADAPT, MID, DUMP, SHAPE><<<pl.grid, B, 0, st>>>(a);
  else
    pair_fp64_kernel<kPropBisect, ADAPT, MID, DUMP, SHAPE><<<pl.grid, B, 0, st>>>(a);
}

cudaError_t launch_pair_fp64(const DeviceState& s, const int* order, int proposal, int reconstruction,
                             const AdaptParams& ap, const PairLaunch& pl, cudaStream_t st, int* dump) {
  PairArgs a;
  a.rec64 = s.rec64;
  a.rec32 = s.rec32;
  a.slot_t = s.slot_t;
  a.lhs64 = s.tab.lhs64;
  a.tab32 = s.tab.tab32;
  a.inv_dtk = s.tab.inv_dtk;
  a.wts = s.wts;
  a.state = s.state;
  a.out = s.partial;
  a.E = s.Eself;
  a.B = s.Bself;
  a.stats = s.stats;
  a.err = s.err;
  a.N = s.N;
  a.D = s.D;
  a.nbunch = s.nbunch;
  a.bunches = s.bunches;
  a.sched = s.sched;
  a.nitems = pl.nitems;
  a.work = s.work;
  a.net = s.mlp_image ? mlp::infer_image(s.mlp_image) : nullptr;
  a.scale = s.scale;
  a.eta_allow = ap.eta_allow;
  a.order = order;
  a.dump = dump;
  // the work counter is zeroed by the set-up launch that precedes every pair launch
  // the midpoint reconstruction runs with a fixed time step only (the host refuses the combination);
  // the bracket dump runs the method's instance (the brackets depend on neither variant)
  if (dump)
    launch_fp64<false, false, true, 0>(proposal, pl, a, st);
  else if (reconstruction == 1)
    launch_fp64<false, true, false, 0>(proposal, pl, a, st);
  else if (ap.on)
    launch_fp64<true, false, false, 0>(proposal, pl, a, st);
  else if (pl.shape == 1)
    launch_fp64<false, false, false, 1>(proposal, pl, a, st);
  else if (pl.shape == 2)
    launch_fp64<false, false, false, 2>(proposal, pl, a, st);
  else
    launch_fp64<false, false, false, 0>(proposal, pl, a, st);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const DeviceState& s, cudaStream_t st) {
  reduce_partials_kernel<<<(unsigned)((s.N + 255) / 256), 256, 0, st>>>(s.partial, s.sched, s.bunch_of, s.N, s.Eself,
                                                                          s.Bself);
  return cudaGetLastError();
}

cudaError_t launch_zero_self(const DeviceState& s, cudaStream_t st) {
  zero_kernel<<<(unsigned)((3 * s.N + 255) / 256), 256, 0, st>>>(s.Eself, s.Bself, 3 * s.N);
  return cudaGetLastError();
}

namespace {
__global__ void recip_probe_kernel(const double* __restrict__ x, double* __restrict__ y, long long n) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) y[k] = recip_newton(x[k]);
}
}  // namespace

void set_error_text(const char* msg);

}  // namespace emppp

extern "C" EMPPP_API emppp_status emppp_reciprocal_probe(const double* x, double* y, int64_t n, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!x || !y))) {
    emppp::set_error_text("emppp_reciprocal_probe: n >= 0 and device arrays x, y are required");
    return EMPPP_ERR_ARG;
  }
  if (n == 0) return EMPPP_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  emppp::recip_probe_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, (long long)n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    emppp::set_error_text(cudaGetErrorString(e));
    return EMPPP_ERR_CUDA;
  }
  return EMPPP_OK;
}
