// Mixed-precision all-pairs Lienard-Wiechert kernel (Sec. 2.1-2.2): pair geometry and fields in FP32,
// time stamps, the bracket decision and (in the push) the momentum update in FP64.
//
// Per pair (target i at r = x_i^n, t = t_n; source j):
//   bracket   the node test P(k): (c (t - t_k))^2 <= |r - w_k|^2 is evaluated in FP32 on hi/lo split
//             coordinates against two per-slot thresholds, L^2 widened and narrowed by the guard band
//             (kGuardBand, emppp_internal.cuh); beyond them the FP32 decision is the FP64 one, between
//             them the FP64 test itself (reference operation order) decides. The bracket is therefore
//             the FP64 one. Search: the paper's bisection, or the guarded galloping
//             search from the uniform-motion guess; with the guess, the records of the one or two slots
//             the guess points at are loaded together, so a correct guess needs a single gather round.
//             A pair the guess places beyond the history first tries the oldest-slot bound (kChordMargin,
//             emppp_internal.cuh): from the staged present separation and the source's chord, it shows the
//             oldest slot's FP32 test true at its first comparison without loading that slot's record.
//   retarded  in light units (lengths in m, velocities as beta = v/c): with L1 = c (t - t1) and d = r - w1,
//             (1 - beta1^2) s^2 + 2 (d.beta1 - L1) s + (L1^2 - |d|^2) = 0 for s = c (t_r - t1) (eq:dt),
//             smaller root without cancellation; eta = d - beta1 s (eq:linear, retarded position w1 + v1 dt);
//             in the near-field shortcut bracket the same point is formed from the segment's end
//             P = w1 + v1 (t_n - t1) as eta = (r - P) + beta1 tau, tau = c (t_n - t_r) = R, which avoids the
//             cancellation in L1^2 - |d|^2 when R is far below c (t_n - t_{n-1});
//             beta = beta1 + (s / (c dt)) (beta2 - beta1), alpha = a / c^2 = (beta2 - beta1) / (c dt)
//             (eq:linear2 out of history: beta = beta1, alpha = 0); 1 - beta^2 = 1/gamma1^2 - dbeta.(2 beta1
//             + dbeta), so 1 - beta^2 is never formed by cancellation.
//   fields    with u' = eta_hat - beta: E = (q / 4 pi eps0) R [(1 - beta^2) u' + eta x (u' x alpha)] / (eta.u')^3
//             (eq:LW_E with v' = c u', a = c^2 alpha), B = eta_hat x E / c (eq:LW_B). eta.u' = R - eta.beta
//             cancels for a source moving towards the target; there it is formed as
//             [R^2 (1 - beta^2) + |eta x beta|^2] / (R + eta.beta), a sum of non-negative terms.
//   sums      FP32 partial sums over kSub sources (8, 16 or 32 by tile shape), added with Kahan
//             compensation into FP32 running totals (kept in shared memory, which leaves the registers to
//             the pair loop: 64 registers, 8 blocks of 128 threads per SM), converted to FP64 at the end.
// Vector arithmetic takes x and y in one packed FP32x2 instruction where both operands come as pairs
// (separations, velocity differences, the retarded point, u', F, the sums) and z as a scalar.
// Sources are walked in tiles of kTile (half a block's targets) whose present records, out-of-history
// lines, oldest-slot chords and FP32 charges are staged in shared memory; targets are taken in the spatial order of order.cu so that a warp's retarded slots of a
// source are close together in the source-major FP32 shadow ring. The window instance (shape_win)
// also copies, per warp and one source ahead, the ring slots its lanes' guessed brackets fall in to
// shared memory by bulk copy (bulk.cuh) and reads the predicted brackets' records there; the search,
// the arithmetic and the work split are those of the same shape without it, so the fields are too.
#include "bulk.cuh"
#include "emppp_internal.cuh"
#include "shadow.cuh"

namespace emppp {

namespace {

#ifndef EMPPP_MIXED_MIN_BLOCKS
#define EMPPP_MIXED_MIN_BLOCKS 8  // resident blocks per SM the register budget is fitted to (64 registers)
#endif

// FP64 recomputation of C0 when u L1^2 |s| / (C0 (L1 - s)) exceeds 2e-6: kC0Guard = 2e-6 / u
constexpr float kC0Guard = 2.0e-6f / 5.9604644775390625e-08f;
// FP64 recomputation of X.beta (out-of-history pairs) when 2 u |X| |X.beta| / denominator exceeds 1.3e-6
constexpr float kXbGuard = 2.0f * 5.9604644775390625e-08f / 1.3e-6f;

struct MixedArgs {
  const float4* __restrict__ rec32;
  const double* __restrict__ rec64;
  const double* __restrict__ lhs64;
  const double* __restrict__ slot_t;  // time stamps of the physical slots
  const float4* __restrict__ tab32;  // per slot: guard-band thresholds of L^2, c (t - t_k), 1 / (c dt_k)
  const float* __restrict__ kq32;  // -e w_j / (4 pi eps0), FP32
  const int* __restrict__ order;
  const StepState* __restrict__ state;
  double* __restrict__ out;
  double* __restrict__ E;
  double* __restrict__ B;
  unsigned long long* stats;
  int* err;
  int N;
  int D;
  int nbunch;
  const BunchDesc* __restrict__ bunches;
  const BunchSched* __restrict__ sched;
  int nitems;  // work items of all bunches
  int* work;   // work-item counter (zero at launch)
  const float* __restrict__ fac;  // learned proposal: delay factors [groups][n] per bunch (factor kernel)
  unsigned long long* scale;  // adaptive time step: eta_min / v_max^2 reduction
  float eta_allow;
  const float4* __restrict__ ext32;  // [N][kExtCount] per source: segment end hi/lo, out-of-history line, oldest slot
  int* __restrict__ dump;  // [N][N] bracket of every evaluated pair, 4 (k1 - k0) + branch (DUMP instances only)
  int wait_limit;          // probes of a bounded wait on a staged history window (window shapes)
};

// probes of the wait, before a block exits, on a window copy whose own wait gave up
constexpr int kDrainLimit = 1 << 20;

struct Target {
  float2 h01, l01;  // x and y of the hi and lo parts (packed FP32x2 operands)
  float h2, l2;
  int idx;          // particle index (its FP64 present record is formed only for the rare FP64 node tests)
  bool exact_only;  // coordinates too far from the split origin for the FP32 band: FP64 tests only
};

// slots of the usable window k0..n are addressed by their offset l = k - k0 (0..nw-1)
struct Window {
  int p0, D, nw;
  int* err;  // device error word (the debug build's range checks)
  __device__ __forceinline__ int phys(int l) const {
    const int p = p0 + debug_index(l, 0, nw, err);
    return p >= D ? p - D : p;
  }
};

struct Rec {  // one FP32 shadow record
  float4 q0, q1, q2;
};

__device__ __forceinline__ Rec load_rec(const float4* __restrict__ src32, int p) {
  Rec r;
  r.q0 = __ldg(src32 + 3 * p);
  r.q1 = __ldg(src32 + 3 * p + 1);
  r.q2 = __ldg(src32 + 3 * p + 2);
  return r;
}

// FP64 node tests (those between the guard-band thresholds) of the block, for the instances that count
// in shared memory (SH); the others count per thread in n_fb
__shared__ unsigned long long s_fallbacks;

template <bool SH>
__device__ __forceinline__ void count_fallback(unsigned& n_fb) {
  if (SH)
    atomicAdd(&s_fallbacks, 1ull);
  else
    n_fb++;
}

__device__ __forceinline__ bool exact_test(const double* __restrict__ rr, const double* __restrict__ w, double lhs) {
  const double d0 = __dsub_rn(__ldg(rr + 0), __ldg(w + 0));
  const double d1 = __dsub_rn(__ldg(rr + 1), __ldg(w + 1));
  const double d2 = __dsub_rn(__ldg(rr + 2), __ldg(w + 2));
  const double rhs = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
  return lhs <= rhs;
}

// a0 b0 + a1 b1 + a2 b2 and a0 b1 - a1 b0 in a fixed rounding sequence (no compiler contraction)
__device__ __forceinline__ float dot3(float a0, float a1, float a2, float b0, float b1, float b2) {
  return __fmaf_rn(a2, b2, __fmaf_rn(a1, b1, __fmul_rn(a0, b0)));
}
__device__ __forceinline__ float cross1(float a0, float a1, float b0, float b1) {
  return __fmaf_rn(a0, b1, -__fmul_rn(a1, b0));
}

// a - (b.x, b.y) by one packed FP32x2 addition of the negation (the same rounding as two subtractions)
__device__ __forceinline__ float2 sub2(float2 a, float4 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// r - w of a record, from the hi and lo parts (each component exact to two roundings); x and y packed
__device__ __forceinline__ float3 separation(const Target& r, float4 q0, float4 q1) {
  const float2 d = __fadd2_rn(sub2(r.h01, q0), sub2(r.l01, q1));
  return make_float3(d.x, d.y, (r.h2 - q0.z) + (r.l2 - q1.z));
}

// P(k) from a separation d already formed at physical slot p, with that slot's table entry tab
template <bool SH>
__device__ __forceinline__ bool node_test_d(const Target& r, float3 d, float4 tab, const double* __restrict__ src64,
                                            int p, const MixedArgs& a, unsigned& n_fb) {
  const float D2 = d.x * d.x + d.y * d.y + d.z * d.z;
  if (!r.exact_only) {
    if (D2 > tab.x) return true;
    if (D2 < tab.y) return false;
  }
  count_fallback<SH>(n_fb);
  return exact_test(a.rec64 + ((size_t)r.idx * a.D + a.state->pn) * 6, src64 + 6 * p, __ldg(a.lhs64 + p));
}

template <bool SH>
__device__ __forceinline__ bool node_test(const Target& r, const float4* __restrict__ src32,
                                          const double* __restrict__ src64, int p, const MixedArgs& a, unsigned& n_fb) {
  return node_test_d<SH>(r, separation(r, __ldg(src32 + 3 * p), __ldg(src32 + 3 * p + 1)), __ldg(a.tab32 + p), src64,
                         p, a, n_fb);
}

// uniform-motion guess of the retarded delay, from the staged present record of the source:
// c tau = gamma^2 [d.beta + sqrt((d.beta)^2 + |d|^2 / gamma^2)] with d from the hi parts only (g2.w is
// gamma^2, times the learned delay factor with that proposal)
__device__ __forceinline__ float closed_form_ctau(const Target& r, float4 g0, float4 g2) {
  const float2 x01 = sub2(r.h01, g0);
  const float x0 = x01.x, x1 = x01.y, x2 = r.h2 - g0.z;
  const float db = x0 * g2.x + x1 * g2.y + x2 * g2.z;
  const float dd = x0 * x0 + x1 * x1 + x2 * x2;
  const float x = fmaxf(fmaf(db, db, g0.w * dd), 0.f);
  return (db + x * rsqrtf(fmaxf(x, 1e-37f))) * g2.w;
}

// offset of the guessed older node for a delay of sc steps: (nw - 2) - floor(sc); -1 ("older than the
// history") when floor(sc) > nw - 2, i.e. sc >= nw - 1, decided before any rounding; a negative or NaN
// delay guesses the newest bracket
__device__ __forceinline__ int guessed_offset(float sc, int nw, float nw1) {
  return (sc >= nw1) ? -1 : (nw - 2) - (int)fmaxf(sc, 0.f);
}

// bisection between offsets lo (P false) and hi (P true); returns lo
template <bool SH>
__device__ __forceinline__ int bisect(const Target& r, const float4* __restrict__ src32, const double* __restrict__ src64,
                                      const Window& w, int lo, int hi, const MixedArgs& a, unsigned& n_tests,
                                      unsigned& n_fb) {
  while (hi - lo > 1) {
    const int m = (lo + hi) >> 1;
    n_tests += 1;
    if (node_test<SH>(r, src32, src64, w.phys(m), a, n_fb))
      hi = m;
    else
      lo = m;
  }
  return lo;
}

}  // namespace

// SHAPE: targets per block (kBlock), sources per FP32 partial sum (kSub); the
// register budget stays at 64 per thread for every block size
template <int PROP, bool ADAPT, bool DUMP, int SHAPE>
__global__ void __launch_bounds__(shape_block(SHAPE), EMPPP_MIXED_MIN_BLOCKS * 128 / shape_block(SHAPE))
    pair_mixed_kernel(MixedArgs a) {
  constexpr int kBlock = shape_block(SHAPE);
  // sources per staged tile: half a block's targets, which keeps 8 blocks of the (128, *) shapes within the
  // 132 KB shared-memory carveout (the rest of the SM's 256 KB is the L1 of the pair gathers)
  constexpr int kTile = kBlock / 2;
  constexpr int kSub = shape_sub(SHAPE);
  // history windows (shape_win): one elected lane per warp copies, one source ahead, the slots its lanes'
  // guessed brackets of the next source fall in from the FP32 shadow ring to shared memory (bulk copy,
  // two buffers per warp); the lanes whose predicted bracket lies in the window read its two records
  // there instead of gathering them
  constexpr bool WIN = shape_win(SHAPE) > 0 && PROP != kPropBisect;
  constexpr int kWin = WIN ? shape_win(SHAPE) : 1;
  constexpr int kWarps = kBlock / 32;
  __shared__ __align__(128) float4 s_win[WIN ? kWarps * 2 * kWin * 3 : 1];
  __shared__ __align__(8) unsigned long long s_bar[WIN ? kWarps * 2 : 1];
  __shared__ int2 s_wd[WIN ? kWarps * 2 : 1];  // (first offset, slots) of each staged window
  __shared__ float4 s_q0[kTile];  // present record (hi, 1/gamma^2) of the tile's sources
  // (beta, gamma^2) of the same records; with the learned proposal the w component carries gamma^2 times the
  // network's delay factor for the block's target group, which only the delay guess reads
  __shared__ float4 s_q2[kTile];
  __shared__ float s_kq[kTile];
  __shared__ float4 s_q1[kTile];  // present record (lo, 0) of the tile's sources
  __shared__ float4 s_x[kTile];   // out-of-history line at t_n, relative to the present position; gamma^2 of slot k0
  // with the uniform-motion guess: the chord w_n - w_k0 and the oldest-slot bound's threshold, and slot k0's
  // (beta - beta_ref, 1/gamma^2) (ext32)
  constexpr int kTileG = PROP != kPropBisect ? kTile : 1;
  __shared__ float4 s_ck[kTileG];
  __shared__ float4 s_k0[kTileG];
  __shared__ float s_acc[12][kBlock];  // per-thread compensated sums

  __shared__ int s_item;
  const int N = a.N;
  const int D = a.D;

  Window win;
  const long long n_abs = a.state->n;
  const long long k0_abs = a.state->k0;
  win.p0 = a.state->p0;
  win.D = D;
  win.err = a.err;
  win.nw = (int)(n_abs - k0_abs) + 1;
  const int pn = a.state->pn;
  const float inv_cdt = (float)(1.0 / (kC * a.state->dt));
  const float nw1 = (float)(win.nw - 1);  // a guessed delay of at least nw - 1 steps is out of history

  // Counts and error bits. Node tests are counted per thread. The branch counts (added once per tile), the
  // FP64 fallbacks and the error bits (both rare) are kept in shared memory by the guessed-search
  // instances without the adaptive step (kShared), which frees their registers for the pair loop; the
  // bisection and adaptive instances keep them per thread, where the register allocation comes out better.
  constexpr bool kShared = PROP != kPropBisect && !ADAPT;
  __shared__ unsigned long long s_cnt[3];  // out of history, shortcut, bisection
  __shared__ int s_err;
  if (threadIdx.x == 0) {
    s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
    s_fallbacks = 0;
    s_err = 0;
  }
  unsigned n_tests = 0, n_ooh = 0, n_sc = 0, n_bi = 0, n_fb = 0;
  int errbits = 0;
  auto set_err = [&](int bits) {
    if (kShared)
      atomicOr(&s_err, bits);
    else
      errbits |= bits;
  };
  float emin = __int_as_float(0x7f800000), vmax2 = 0.f;  // adaptive time step (Sec. 2.4), vmax2 in units of c^2
  // history windows: phase parity and pending copy of each of the warp's two buffers (warp-uniform), and
  // whether the warp still stages (a wait that gave up stops it; the pairs then gather from the ring)
  unsigned wph = 0, wpend = 0;
  bool wok = true;
  int g_nxt = -1;  // the lane's guessed offset for the next source (-1: out of history)
  if (WIN) {
    if (threadIdx.x < kWarps * 2) {
      mbar_init(smem_u32(&s_bar[threadIdx.x]), 1);
      fence_mbar_init();
    }
  }

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
  const int boff = (int)bd.off;
  const float2 bref01 = make_float2((float)bd.beta_ref[0], (float)bd.beta_ref[1]);
  const float bref2 = (float)bd.beta_ref[2];
  const int t_loc = tb * kBlock + threadIdx.x;
  const bool active = t_loc < bd.n;
  const int t = boff + (active ? t_loc : 0);
  const int i = debug_index(a.order ? a.order[t] : t, boff, boff + bd.n, a.err);

  Target r;
  {
    const float4 q0 = a.rec32[((size_t)i * D + pn) * 3];
    const float4 q1 = a.rec32[((size_t)i * D + pn) * 3 + 1];
    r.h01 = make_float2(q0.x, q0.y);
    r.h2 = q0.z;
    r.l01 = make_float2(q1.x, q1.y);
    r.l2 = q1.z;
    r.idx = i;
    r.exact_only = fmaxf(fabsf(r.h01.x), fmaxf(fabsf(r.h01.y), fabsf(r.h2))) > 0.5f;
  }
  // learned proposal: the delay factors of this target tile's group (kFacGroup targets, a multiple of the
  // tile), one per source of the bunch
  // (as an index of a.fac relative to the bunch's first particle: the table has fewer than 2^31 entries)
  const int fac_row = PROP == kPropMlp ? (int)(bd.fac_off + (long long)((tb * kBlock) / kFacGroup) * bd.n) - boff : 0;
  // the lane's guessed older-node offset for staged source jj of the tile (-1: predicted out of history)
  auto guess_of = [&](int jj) -> int {
    const float sc = closed_form_ctau(r, s_q0[jj], s_q2[jj]) * inv_cdt;
    return guessed_offset(sc, win.nw, nw1);
  };
  // beta_i(t_n) - beta_ref of the target (adaptive time step; target and sources share the bunch's beta_ref,
  // so relative velocities are formed from these small differences at full FP32 relative precision)
  float bi0 = 0.f, bi1 = 0.f, bi2 = 0.f;
  if (ADAPT) {
    const float4 q2 = a.rec32[((size_t)i * D + pn) * 3 + 2];
    bi0 = q2.x;
    bi1 = q2.y;
    bi2 = q2.z;
  }

  const int j_begin = boff + chunk_id * bs.chunk;
  const int j_end = min(boff + bd.n, j_begin + bs.chunk);

  // compensated running sums of E and of c B, kept in shared memory (rows: E sums, E compensations,
  // c B sums, c B compensations) to leave registers to the pair loop
#pragma unroll
  for (int c = 0; c < 12; c++) s_acc[c][threadIdx.x] = 0.f;

  for (int tile = j_begin; tile < j_end; tile += kTile) {
    const int tn = min(kTile, j_end - tile);
    unsigned brc = 0;  // out-of-history, shortcut and bisection counts of this tile (at most kTile each)
    __syncthreads();
    if (threadIdx.x < tn) {
      const int j = debug_index<int>(tile + (int)threadIdx.x, boff, boff + bd.n, a.err);
      const float4* q = a.rec32 + ((size_t)j * D + pn) * 3;
      s_q0[threadIdx.x] = q[0];
      const float4 q2 = q[2];
      s_q2[threadIdx.x] = make_float4(bref01.x + q2.x, bref01.y + q2.y, bref2 + q2.z,
                                      PROP == kPropMlp ? q2.w * __ldg(a.fac + (fac_row + j)) : q2.w);
      s_kq[threadIdx.x] = a.kq32[j];
      s_q1[threadIdx.x] = q[1];
      const float4* e = a.ext32 + (size_t)j * kExtCount;
      s_x[threadIdx.x] = __ldg(e + kExtLine);
      if (PROP != kPropBisect) {
        s_ck[threadIdx.x] = __ldg(e + kExtChord);
        s_k0[threadIdx.x] = __ldg(e + kExtOldest);
      }
    }
    __syncthreads();
    // window of staged source jn into buffer sb: the offsets lo .. hi + 1 of the guessed brackets [lg, lg + 1]
    // of the warp's lanes that predict one in history, at most kWin slots from lo (one or two contiguous
    // runs of the ring)
    auto win_issue = [&](int jn, int g, int sb) {
      const bool want = wok && active && (tile + jn != i) && g >= 0;
      const int lo = __reduce_min_sync(0xffffffffu, want ? g : 0x7fffffff);
      const int hi = __reduce_max_sync(0xffffffffu, want ? g : -1);
      if (lo > hi) return;
      const int nsl = min(hi + 2 - lo, kWin);
      if (kDebug && (lo < 0 || lo + nsl > win.nw)) {  // the staged run lies inside the usable window
        if ((threadIdx.x & 31) == 0) atomicOr(a.err, kErrBounds);
        return;
      }
      if ((threadIdx.x & 31) == 0) {
        const int wb = (threadIdx.x >> 5) * 2 + sb;
        s_wd[wb] = make_int2(lo, nsl);
        const uint32_t bar = smem_u32(&s_bar[wb]);
        mbar_arrive_expect_tx(bar, (uint32_t)nsl * 48u);
        const int p = win.phys(lo);
        const int n1 = min(nsl, D - p);
        const size_t base = (size_t)(tile + jn) * D;
        float4* dst = s_win + (size_t)wb * kWin * 3;
        bulk_copy_g2s(smem_u32(dst), a.rec32 + (base + p) * 3, (uint32_t)n1 * 48u, bar);
        if (nsl > n1) bulk_copy_g2s(smem_u32(dst + 3 * n1), a.rec32 + base * 3, (uint32_t)(nsl - n1) * 48u, bar);
      }
      wpend |= 1u << sb;
    };
    if (WIN && win.nw > 1) {
      g_nxt = guess_of(0);
      win_issue(0, g_nxt, 0);
    }
    for (int jj0 = 0; jj0 < tn; jj0 += kSub) {
      float P[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const int jend = min(jj0 + kSub, tn);
      for (int jj = jj0; (WIN || active) && jj < jend; ++jj) {
        const int j = debug_index(tile + jj, boff, boff + bd.n, a.err);
        // history window of this source (WIN): guessed offset, first offset and slots of the staged run
        int g_cur = -1, w_lo = 0, w_n = 1;
        const int sb = jj & 1;
        if (WIN && win.nw > 1) {
          g_cur = g_nxt;
          __syncwarp();  // every lane is done with the buffer the next copy overwrites
          if (jj + 1 < tn) {
            g_nxt = guess_of(jj + 1);
            win_issue(jj + 1, g_nxt, sb ^ 1);
          }
          if (wpend & (1u << sb)) {
            const uint32_t bar = smem_u32(&s_bar[(threadIdx.x >> 5) * 2 + sb]);
            const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, (wph >> sb) & 1u, a.wait_limit));
            if (ok) {
              wph ^= 1u << sb;
              wpend &= ~(1u << sb);
              const int2 wd = s_wd[(threadIdx.x >> 5) * 2 + sb];
              w_lo = wd.x;
              w_n = wd.y;
            } else {
              // the copy stays pending (drained before the block exits); no further windows
              set_err(kErrTimeout);
              wok = false;
            }
          }
        }
        if (WIN && !active) continue;
        if (j == i) continue;
        const float4* src32 = a.rec32 + (size_t)j * D * 3;
        const double* src64 = a.rec64 + (size_t)j * D * 6;
        auto heaviside = [&](float2 dn01, float dn2, float4 o, float g2, int pk) {
          // ---- out of history (eq:linear2): the source moves uniformly with beta1 along the line through
          // w1; its Lienard-Wiechert field is Heaviside's field about the line's point at t_n,
          //   E = kq (1 - beta^2) X / [X^2 (1 - beta^2) + (X.beta)^2]^{3/2},  c B = beta x E,
          // with X = (r - w_n) - (line at t_n - w_n) from the staged present record and line offset.
          const float4 gx = s_x[jj];
          const float2 X01 = sub2(dn01, gx);
          float X0 = X01.x, X1 = X01.y;
          float X2 = __fsub_rn(dn2, gx.z);
          const float2 b101 = __fadd2_rn(bref01, make_float2(o.x, o.y));
          const float b10 = b101.x, b11 = b101.y, b12 = __fadd_rn(bref2, o.z);
          const float ig2 = o.w;
          float Xb = dot3(X0, X1, X2, b10, b11, b12);
          float XX = dot3(X0, X1, X2, X0, X1, X2);
          // The FP32 rounding of X.beta (absolute about u |X|) moves the denominator by 2 u |X| |X.beta| /
          // denominator relative, at most u gamma. Above 1.3e-6 (only for gamma above ~20, at directions
          // near perpendicular to beta) X and X.beta are formed in FP64 from the FP64 records instead.
          // (as the shift is at most u gamma, sources with gamma^2 < 100 never need it)
          if (ig2 < 0.01f && __fmul_rn(kXbGuard, __fmul_rn(sqrtf(XX), fabsf(Xb))) > __fmaf_rn(XX, ig2, __fmul_rn(Xb, Xb))) {
            const double* w0 = src64 + 6 * pk;  // FP64 record of slot k0: X = r - w_k0 - v_k0 (t_n - t_k0)
            const double ct = kC * (a.state->t - __ldg(a.slot_t + pk));  // c (t_n - t_k0)
            const double ic = 1.0 / kC;
            const double* rr = a.rec64 + ((size_t)i * D + pn) * 6;
            const double y0 = (__ldg(rr + 0) - __ldg(w0 + 0)) - __ldg(w0 + 3) * ic * ct;
            const double y1 = (__ldg(rr + 1) - __ldg(w0 + 1)) - __ldg(w0 + 4) * ic * ct;
            const double y2 = (__ldg(rr + 2) - __ldg(w0 + 2)) - __ldg(w0 + 5) * ic * ct;
            X0 = (float)y0;
            X1 = (float)y1;
            X2 = (float)y2;
            Xb = (float)((y0 * __ldg(w0 + 3) + y1 * __ldg(w0 + 4) + y2 * __ldg(w0 + 5)) * ic);
            XX = dot3(X0, X1, X2, X0, X1, X2);
            count_fallback<kShared>(n_fb);
          }
          const float Dh = __fmaf_rn(XX, ig2, __fmul_rn(Xb, Xb));
          const float iD = rsqrtf(Dh);
          if (!(Dh > 0.f) || !(ig2 > 0.f)) {
            set_err((ig2 > 0.f) ? kErrCoincide : kErrDisc);
            return;
          }
          const float pref = __fmul_rn(__fmul_rn(s_kq[jj], ig2), __fmul_rn(__fmul_rn(iD, iD), iD));
          if (ADAPT) {
            // retarded distance c (t - t_r) = gamma^2 [X.beta + sqrt(Dh)], and v(t_r) = v1
            const float sD = __fmul_rn(Dh, iD);
            const float R = (Xb >= 0.f) ? __fmul_rn(__fadd_rn(Xb, sD), g2)
                                        : __fdividef(dot3(X0, X1, X2, X0, X1, X2), __fsub_rn(sD, Xb));
            if (R >= a.eta_allow) {
              emin = fminf(emin, R);
              const float dv0 = bi0 - o.x, dv1 = bi1 - o.y, dv2 = bi2 - o.z;
              vmax2 = fmaxf(vmax2, dv0 * dv0 + dv1 * dv1 + dv2 * dv2);
            }
          }
          const float2 p01 = __ffma2_rn(make_float2(pref, pref), make_float2(X0, X1), make_float2(P[0], P[1]));
          P[0] = p01.x;
          P[1] = p01.y;
          P[2] = __fmaf_rn(pref, X2, P[2]);
          // c B = beta x E = pref (beta x X)
          const float2 p34 = __ffma2_rn(make_float2(pref, pref),
                                        make_float2(cross1(b11, b12, X1, X2), cross1(b12, b10, X2, X0)),
                                        make_float2(P[3], P[4]));
          P[3] = p34.x;
          P[4] = p34.y;
          P[5] = __fmaf_rn(pref, cross1(b10, b11, X0, X1), P[5]);
        };
        // ---- bracket: offset l1 of the older node, its slot pA, record A, separation dA and table -------
        int l1;
        int br;
        int pA;         // physical slot of the older node
        Rec A;          // record of the older node
        float3 dA;      // r - w at the older node
        float4 tabA;    // slot table entry of the older node
        float4 q2b;     // (dbeta, gamma^2) of the newer node (regular brackets)
        bool have_b = false;
        bool fast = true;  // pA, A, dA and tabA already belong to l1
        if (win.nw == 1) {
          // n = k0: only the present slot exists; every pair is out of history
          n_tests += 1;
          l1 = 0;
          br = 0;
          pA = win.phys(0);
          A = load_rec(src32, pA);
          dA = separation(r, A.q0, A.q1);
          tabA = __ldg(a.tab32 + pA);
        } else if (PROP == kPropBisect) {
          n_tests += 1;
          pA = win.phys(0);
          A = load_rec(src32, pA);
          dA = separation(r, A.q0, A.q1);
          tabA = __ldg(a.tab32 + pA);
          if (node_test_d<kShared>(r, dA, tabA, src64, pA, a, n_fb)) {
            l1 = 0;
            br = 0;
          } else {
            n_tests += 1;
            if (!node_test<kShared>(r, src32, src64, win.phys(win.nw - 2), a, n_fb)) {
              l1 = win.nw - 2;
              br = 1;
            } else {
              l1 = bisect<kShared>(r, src32, src64, win, 0, win.nw - 1, a, n_tests, n_fb);
              br = 2;
            }
            fast = (l1 == 0);
          }
        } else {
          // the uniform-motion delay (with the learned proposal scaled by the network's factor for the
          // block's target group and this source, staged in s_q2)
          const int lraw = WIN ? g_cur : guess_of(jj);
          // predicted out of history: the oldest-slot bound (kChordMargin) from the present separation and
          // the staged chord; where it holds, slot k0's node test is true without its record
          if (lraw < 0 && !r.exact_only) {
            const float4 ck = s_ck[jj];
            const float3 dn = separation(r, s_q0[jj], s_q1[jj]);
            const float dd = dn.x * dn.x + dn.y * dn.y + dn.z * dn.z;
            const float dc = dn.x * ck.x + dn.y * ck.y + dn.z * ck.z;
            if (fmaf(2.f, dc, dd * kChordLo) > ck.w) {
              n_tests += 1;
              brc += 1u;
              if (DUMP) a.dump[(size_t)i * N + j] = 0;
              heaviside(make_float2(dn.x, dn.y), dn.z, s_k0[jj], s_x[jj].w, win.phys(0));
              continue;
            }
          }
          const int lg = max(lraw, 0);
          pA = win.phys(lg);
          // records of the guessed bracket: from the staged window when both lie in it
          const float4* ra = src32 + 3 * pA;
          const bool inw = WIN && (unsigned)(lraw - w_lo) < (unsigned)(w_n - 1);
          if (WIN) {
            if (inw) ra = s_win + ((size_t)(threadIdx.x >> 5) * 2 + sb) * kWin * 3 + 3 * (lraw - w_lo);
            A.q0 = ra[0];
            A.q1 = ra[1];
            A.q2 = ra[2];
          } else {
            A = load_rec(src32, pA);
          }
          dA = separation(r, A.q0, A.q1);
          tabA = __ldg(a.tab32 + pA);
          if (lraw < 0) {
            // predicted out of history: the only record needed is the oldest slot's
            n_tests += 1;
            if (node_test_d<kShared>(r, dA, tabA, src64, pA, a, n_fb)) {
              l1 = 0;
              br = 0;
            } else {
              // guess wrong: gallop up from lo = 0 (P false)
              int lo = 0, hi, st = 1;
              for (;;) {
                hi = lo + st;
                if (hi >= win.nw - 1) {
                  hi = win.nw - 1;
                  break;
                }
                n_tests += 1;
                if (node_test<kShared>(r, src32, src64, win.phys(hi), a, n_fb)) break;
                lo = hi;
                st <<= 1;
              }
              l1 = bisect<kShared>(r, src32, src64, win, lo, hi, a, n_tests, n_fb);
              br = (l1 == win.nw - 2) ? 1 : 2;
              fast = (l1 == 0);
            }
          } else {
            // predicted bracket [lg, lg + 1]: both records are loaded at once
            const int pg1 = pA + 1 == D ? 0 : pA + 1;  // slot of offset lg + 1
            Rec Bn;
            if (WIN) {
              const float4* rb = inw ? ra + 3 : src32 + 3 * pg1;
              Bn.q0 = rb[0];
              Bn.q1 = rb[1];
              Bn.q2 = rb[2];
            } else {
              Bn = load_rec(src32, pg1);
            }
            n_tests += 1;
            const bool tA = node_test_d<kShared>(r, dA, tabA, src64, pA, a, n_fb);
            if (!tA) {
              bool tB = true;  // P(n) is always true
              if (lg + 1 < win.nw - 1) {
                n_tests += 1;
                tB = node_test_d<kShared>(r, separation(r, Bn.q0, Bn.q1), __ldg(a.tab32 + pg1), src64, pg1, a, n_fb);
              }
              if (tB) {
                l1 = lg;
                br = (l1 == win.nw - 2) ? 1 : 2;
                q2b = Bn.q2;
                have_b = true;
              } else {
                // gallop up from lo = lg + 1 (P false)
                int lo = lg + 1, hi, st = 1;
                for (;;) {
                  hi = lo + st;
                  if (hi >= win.nw - 1) {
                    hi = win.nw - 1;
                    break;
                  }
                  n_tests += 1;
                  if (node_test<kShared>(r, src32, src64, win.phys(hi), a, n_fb)) break;
                  lo = hi;
                  st <<= 1;
                }
                l1 = bisect<kShared>(r, src32, src64, win, lo, hi, a, n_tests, n_fb);
                br = (l1 == win.nw - 2) ? 1 : 2;
                fast = false;
              }
            } else if (lg == 0) {
              l1 = 0;
              br = 0;
            } else {
              // gallop down from hi = lg (P true)
              int hi = lg, lo = lg, st = 1;
              bool ooh = false;
              for (;;) {
                if (hi == 0) {
                  ooh = true;
                  break;
                }
                lo = max(hi - st, 0);
                n_tests += 1;
                if (!node_test<kShared>(r, src32, src64, win.phys(lo), a, n_fb)) break;
                hi = lo;
                st <<= 1;
              }
              if (ooh) {
                l1 = 0;
                br = 0;
              } else {
                l1 = bisect<kShared>(r, src32, src64, win, lo, hi, a, n_tests, n_fb);
                br = (l1 == win.nw - 2) ? 1 : 2;
              }
              fast = false;
            }
          }
        }
        if (!fast) {
          pA = win.phys(l1);
          A = load_rec(src32, pA);
          dA = separation(r, A.q0, A.q1);
          tabA = __ldg(a.tab32 + pA);
        }
        brc += 1u << (10 * br);  // branch counts of this tile, 10 bits each
        if (DUMP) a.dump[(size_t)i * N + j] = 4 * l1 + br;

        if (br == 0) {
          const float4 g0 = s_q0[jj], g1 = s_q1[jj];
          heaviside(__fadd2_rn(sub2(r.h01, g0), sub2(r.l01, g1)), __fadd_rn(__fsub_rn(r.h2, g0.z), __fsub_rn(r.l2, g1.z)),
                    make_float4(A.q2.x, A.q2.y, A.q2.z, A.q0.w), A.q2.w, pA);
          continue;
        }
        // ---- retarded state (light units) --------------------------------------------------------
        // Written with explicit round-to-nearest intrinsics: the compiler may not fuse or regroup any
        // of it, so every search variant (whose own arithmetic shares subexpressions with this code
        // in different ways) computes the same fields from the same bracket, bit for bit. The packed
        // FP32x2 forms (x and y in one instruction) round per component like the scalar ones, but the
        // compiler fuses a packed product that feeds a packed sum; so no packed product feeds a packed
        // sum here, and every multiply-add is written as one fused operation (__ffma2_rn, __fmaf_rn).
        const float d0 = dA.x, d1 = dA.y, d2 = dA.z;
        const float L1 = tabA.z;
        const float2 b101 = __fadd2_rn(bref01, make_float2(A.q2.x, A.q2.y));
        const float b10 = b101.x, b11 = b101.y, b12 = __fadd_rn(bref2, A.q2.z);
        const float ig2 = A.q0.w, g2 = A.q2.w;
        float e0, e1, e2, qd, df;  // eta, the discriminant, and (t_r - t1) / (t2 - t1)
        if (br == 1) {
          // near-field shortcut, t_r in [t_{n-1}, t_n]: the retarded point is P - beta1 tau with P the end
          // of the segment (ext32) and tau = c (t_n - t_r) = R, the positive root of
          // (1 - beta1^2) tau^2 - 2 (p.beta1) tau - |p|^2 = 0, p = r - P (eq:dt about t_n). Formed this
          // way, eta keeps FP32 precision when R is far below c (t_n - t_{n-1}).
          const float4* e = a.ext32 + (size_t)j * kExtCount;
          const float3 dp = separation(r, __ldg(e + kExtSegHi), __ldg(e + kExtSegLo));
          const float pb = dot3(dp.x, dp.y, dp.z, b10, b11, b12);
          const float pp = dot3(dp.x, dp.y, dp.z, dp.x, dp.y, dp.z);
          qd = __fmaf_rn(pb, pb, __fmul_rn(ig2, pp));
          const float sq = __fmul_rn(qd, rsqrtf(fmaxf(qd, 1e-37f)));
          const float tau = (pb <= 0.f) ? __fdividef(pp, __fsub_rn(sq, pb)) : __fmul_rn(__fadd_rn(pb, sq), g2);
          const float2 e01 = __ffma2_rn(b101, make_float2(tau, tau), make_float2(dp.x, dp.y));
          e0 = e01.x;
          e1 = e01.y;
          e2 = __fmaf_rn(b12, tau, dp.z);
          df = __fmaf_rn(-tau, tabA.w, 1.f);
        } else {
          const float hb = __fsub_rn(dot3(d0, d1, d2, b10, b11, b12), L1);
          float C0 = __fmaf_rn(L1, L1, -dot3(d0, d1, d2, d0, d1, d2));
          qd = __fmaf_rn(hb, hb, -__fmul_rn(ig2, C0));
          float sq = __fmul_rn(qd, rsqrtf(fmaxf(qd, 1e-37f)));
          float s = (hb <= 0.f) ? __fdividef(C0, __fsub_rn(sq, hb)) : __fmul_rn(-__fadd_rn(hb, sq), g2);
          // C0 = L1^2 - |d|^2 cancels when |d| is close to L1; its FP32 rounding moves eta by about
          // u L1^2 s / C0, relative to R = L1 - s. That reaches 2e-6 only for sources moving nearly
          // towards the target at high gamma (eta moves by ~ u / (1 - beta cos psi)); for those pairs
          // C0 is formed again in FP64 from the reference quantities (c (t - t1))^2 and the FP64 positions.
          // (the shift is below u / (1 - beta) < 2 u gamma^2, so sources with gamma^2 < 16 never need it)
          if (br == 2 && ig2 < 0.0625f &&
              __fmul_rn(__fmul_rn(L1, L1), fabsf(s)) > __fmul_rn(kC0Guard, __fmul_rn(C0, __fsub_rn(L1, s)))) {
            const double* w64 = src64 + 6 * pA;
            const double* rr = a.rec64 + ((size_t)i * D + pn) * 6;
            const double x0 = __dsub_rn(__ldg(rr + 0), __ldg(w64 + 0));
            const double x1 = __dsub_rn(__ldg(rr + 1), __ldg(w64 + 1));
            const double x2 = __dsub_rn(__ldg(rr + 2), __ldg(w64 + 2));
            C0 = (float)(__ldg(a.lhs64 + pA) - (x0 * x0 + x1 * x1 + x2 * x2));
            qd = __fmaf_rn(hb, hb, -__fmul_rn(ig2, C0));
            sq = __fmul_rn(qd, rsqrtf(fmaxf(qd, 1e-37f)));
            s = (hb <= 0.f) ? __fdividef(C0, __fsub_rn(sq, hb)) : __fmul_rn(-__fadd_rn(hb, sq), g2);
            count_fallback<kShared>(n_fb);
          }
          const float2 e01 = __ffma2_rn(make_float2(-b10, -b11), make_float2(s, s), make_float2(d0, d1));
          e0 = e01.x;
          e1 = e01.y;
          e2 = __fmaf_rn(-b12, s, d2);
          df = __fmul_rn(s, tabA.w);
        }
        float be0 = b10, be1 = b11, be2 = b12, al0 = 0.f, al1 = 0.f, al2 = 0.f, ug = ig2;
        float xs0 = 0.f, xs1 = 0.f, xs2 = 0.f;  // beta(t_r) - beta1 (eq:linear)
        if (br != 0) {
          if (!have_b) q2b = __ldg(src32 + 3 * (pA + 1 == D ? 0 : pA + 1) + 2);
          const float icdt = tabA.w;
          const float2 db01 = sub2(make_float2(q2b.x, q2b.y), A.q2);
          const float db2 = __fsub_rn(q2b.z, A.q2.z);
          const float2 al01 = __fmul2_rn(db01, make_float2(icdt, icdt));
          al0 = al01.x;
          al1 = al01.y;
          al2 = __fmul_rn(db2, icdt);
          const float2 x01 = __fmul2_rn(db01, make_float2(df, df));
          const float x0 = x01.x, x1 = x01.y, x2 = __fmul_rn(db2, df);
          if (ADAPT) {
            xs0 = x0;
            xs1 = x1;
            xs2 = x2;
          }
          const float2 be01 = __ffma2_rn(db01, make_float2(df, df), b101);
          be0 = be01.x;
          be1 = be01.y;
          be2 = __fmaf_rn(db2, df, b12);
          // 1 - beta^2 = (1 - beta1^2) - x.(2 beta1 + x)
          const float2 t01 = __ffma2_rn(make_float2(2.f, 2.f), b101, x01);  // 2 beta1 + x
          ug = __fsub_rn(ig2, dot3(x0, x1, x2, t01.x, t01.y, __fmaf_rn(2.f, b12, x2)));
        }
        // ---- Lienard-Wiechert fields ---------------------------------------------------------------
        const float R2 = dot3(e0, e1, e2, e0, e1, e2);
        const float invR = rsqrtf(R2);
        const float R = __fmul_rn(R2, invR);
        // u' = eta / R - beta
        const float2 u01 = __ffma2_rn(make_float2(e0, e1), make_float2(invR, invR), make_float2(-be0, -be1));
        const float u0 = u01.x, u1 = u01.y, u2 = __fmaf_rn(e2, invR, -be2);
        const float eb = dot3(e0, e1, e2, be0, be1, be2);
        // 1 / (eta . u'): R - eta.beta directly when eta.beta <= 0, else the rationalised form
        const float xb0 = cross1(e1, e2, be1, be2), xb1 = cross1(e2, e0, be2, be0), xb2 = cross1(e0, e1, be0, be1);
        const float rat = __fmaf_rn(R2, ug, dot3(xb0, xb1, xb2, xb0, xb1, xb2));
        const bool fw = eb > 0.f;
        const float ieu = __fdividef(fw ? __fadd_rn(R, eb) : 1.f, fw ? rat : __fsub_rn(R, eb));
        const bool root_ok = (qd >= 0.f) && (ig2 > 0.f);
        if (!(root_ok && R2 > 0.f && ieu > 0.f && ieu < 3.0e38f)) {
          set_err(root_ok ? kErrCoincide : kErrDisc);
          continue;
        }
        const float pref = __fmul_rn(__fmul_rn(__fmul_rn(s_kq[jj], __fmul_rn(R, ieu)), ieu), ieu);
        float2 F01;
        float F2;
        if (br != 0) {
          // (1 - beta^2) u' + eta x (u' x alpha)
          const float c0 = cross1(u1, u2, al1, al2), c1 = cross1(u2, u0, al2, al0), c2 = cross1(u0, u1, al0, al1);
          F01 = __ffma2_rn(make_float2(ug, ug), u01, make_float2(cross1(e1, e2, c1, c2), cross1(e2, e0, c2, c0)));
          F2 = __fmaf_rn(ug, u2, cross1(e0, e1, c0, c1));
        } else {
          F01 = __fmul2_rn(make_float2(ug, ug), u01);
          F2 = __fmul_rn(ug, u2);
        }
        const float F0 = F01.x, F1 = F01.y;
        // E = pref F; c B = eta_hat x E = (pref / R) (eta x F), with 1 / c applied once per target
        if (ADAPT && R >= a.eta_allow) {
          // interaction scale of the adaptive step: |eta_ij| and |beta_i(t_n) - beta_j(t_r)|, with
          // beta_j(t_r) - beta_ref = (beta1 - beta_ref) + (beta(t_r) - beta1)
          emin = fminf(emin, R);
          const float dv0 = (bi0 - A.q2.x) - xs0, dv1 = (bi1 - A.q2.y) - xs1, dv2 = (bi2 - A.q2.z) - xs2;
          vmax2 = fmaxf(vmax2, dv0 * dv0 + dv1 * dv1 + dv2 * dv2);
        }
        const float2 p01 = __ffma2_rn(make_float2(pref, pref), F01, make_float2(P[0], P[1]));
        P[0] = p01.x;
        P[1] = p01.y;
        P[2] = __fmaf_rn(pref, F2, P[2]);
        const float pb = __fmul_rn(pref, invR);
        const float2 p34 = __ffma2_rn(make_float2(pb, pb), make_float2(cross1(e1, e2, F1, F2), cross1(e2, e0, F2, F0)),
                                      make_float2(P[3], P[4]));
        P[3] = p34.x;
        P[4] = p34.y;
        P[5] = __fmaf_rn(pb, cross1(e0, e1, F0, F1), P[5]);
      }
      // Kahan-add the partial sums of these kSub sources
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const float es = s_acc[c][threadIdx.x], ec = s_acc[3 + c][threadIdx.x];
        const float y = P[c] - ec;
        const float tt = es + y;
        s_acc[3 + c][threadIdx.x] = (tt - es) - y;
        s_acc[c][threadIdx.x] = tt;
        const float bsv = s_acc[6 + c][threadIdx.x], bcv = s_acc[9 + c][threadIdx.x];
        const float yb = P[3 + c] - bcv;
        const float tb = bsv + yb;
        s_acc[9 + c][threadIdx.x] = (tb - bsv) - yb;
        s_acc[6 + c][threadIdx.x] = tb;
      }
    }
    if (!kShared) {
      n_ooh += brc & 1023u;
      n_sc += (brc >> 10) & 1023u;
      n_bi += brc >> 20;
    } else {
      const unsigned c0 = __reduce_add_sync(0xffffffffu, brc & 1023u);
      const unsigned c1 = __reduce_add_sync(0xffffffffu, (brc >> 10) & 1023u);
      const unsigned c2 = __reduce_add_sync(0xffffffffu, brc >> 20);
      if ((threadIdx.x & 31) == 0) {
        if (c0) atomicAdd(&s_cnt[0], (unsigned long long)c0);
        if (c1) atomicAdd(&s_cnt[1], (unsigned long long)c1);
        if (c2) atomicAdd(&s_cnt[2], (unsigned long long)c2);
      }
    }
  }
  if (active) {
    double Et[3], Bt[3];
    for (int c = 0; c < 3; c++) {
      Et[c] = (double)s_acc[c][threadIdx.x] - (double)s_acc[3 + c][threadIdx.x];
      Bt[c] = ((double)s_acc[6 + c][threadIdx.x] - (double)s_acc[9 + c][threadIdx.x]) * (1.0 / kC);
    }
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
    reduce_scale(a.scale + 2 * b, (double)emin, (double)vmax2 * (kC * kC));
    emin = __int_as_float(0x7f800000);
    vmax2 = 0.f;
  }
  }  // work items
  if (WIN) {
    // a window whose wait gave up: its copy completes before the block's shared memory is released
    for (int sb = 0; sb < 2; sb++)
      if (wpend & (1u << sb))
        mbar_wait_bounded(smem_u32(&s_bar[(threadIdx.x >> 5) * 2 + sb]), (wph >> sb) & 1u, kDrainLimit);
  }
  n_tests = __reduce_add_sync(0xffffffffu, n_tests);
  if ((threadIdx.x & 31) == 0 && n_tests) atomicAdd(a.stats + kStatNodeTests, (unsigned long long)n_tests);
  if (!kShared) {
    n_ooh = __reduce_add_sync(0xffffffffu, n_ooh);
    n_sc = __reduce_add_sync(0xffffffffu, n_sc);
    n_bi = __reduce_add_sync(0xffffffffu, n_bi);
    n_fb = __reduce_add_sync(0xffffffffu, n_fb);
    errbits = __reduce_or_sync(0xffffffffu, errbits);
    if ((threadIdx.x & 31) == 0) {
      if (n_ooh) atomicAdd(&s_cnt[0], (unsigned long long)n_ooh);
      if (n_sc) atomicAdd(&s_cnt[1], (unsigned long long)n_sc);
      if (n_bi) atomicAdd(&s_cnt[2], (unsigned long long)n_bi);
      if (n_fb) atomicAdd(&s_fallbacks, (unsigned long long)n_fb);
      if (errbits) atomicOr(&s_err, errbits);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_cnt[0]) atomicAdd(a.stats + kStatOOH, s_cnt[0]);
    if (s_cnt[1]) atomicAdd(a.stats + kStatShortcut, s_cnt[1]);
    if (s_cnt[2]) atomicAdd(a.stats + kStatBisect, s_cnt[2]);
    if (s_fallbacks) atomicAdd(a.stats + kStatGuard, s_fallbacks);
    if (s_err) atomicOr(a.err, s_err);
  }
}

template <bool ADAPT, int SHAPE>
int max_blocks_mixed(int proposal) {
  int nb = 0;
  constexpr int B = shape_block(SHAPE);
  if (proposal == kPropClosedForm)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_mixed_kernel<kPropClosedForm, ADAPT, false, SHAPE>, B, 0);
  else if (proposal == kPropMlp)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_mixed_kernel<kPropMlp, ADAPT, false, SHAPE>, B, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_mixed_kernel<kPropBisect, ADAPT, false, SHAPE>, B, 0);
  return nb > 0 ? nb : 1;
}

// the adaptive-step instances and the bracket dump run the default shape only
int max_blocks_pair_mixed(int proposal, bool adapt, int shape) {
  if (adapt) return max_blocks_mixed<true, 0>(proposal);
  switch (shape) {
    case 1: return max_blocks_mixed<false, 1>(proposal);
    case 2: return max_blocks_mixed<false, 2>(proposal);
    case 3: return max_blocks_mixed<false, 3>(proposal);
    case 4: return max_blocks_mixed<false, 4>(proposal);
    case 5: return max_blocks_mixed<false, 5>(proposal);
    default: return max_blocks_mixed<false, 0>(proposal);
  }
}

template <bool ADAPT, bool DUMP, int SHAPE>
void launch_mixed(int proposal, const PairLaunch& pl, const MixedArgs& a, cudaStream_t st) {
  constexpr int B = shape_block(SHAPE);
  if (proposal == kPropClosedForm)
    pair_mixed_kernel<kPropClosedForm, ADAPT, DUMP, SHAPE><<<pl.grid, B, 0, st>>>(a);
  else if (proposal == kPropMlp)
    pair_mixed_kernel<kPropMlp, ADAPT, DUMP, SHAPE><<<pl.grid, B, 0, st>>>(a);
  else
    pair_mixed_kernel<kPropBisect, ADAPT, DUMP, SHAPE><<<pl.grid, B, 0, st>>>(a);
}

cudaError_t launch_pair_mixed(const DeviceState& s, const int* order, int proposal, const AdaptParams& ap,
                              const PairLaunch& pl, cudaStream_t st, int* dump) {
  MixedArgs a;
  a.rec32 = reinterpret_cast<const float4*>(s.rec32);
  a.rec64 = s.rec64;
  a.lhs64 = s.tab.lhs64;
  a.slot_t = s.slot_t;
  a.tab32 = s.tab.tab32;
  a.kq32 = s.kq32;
  a.order = order;
  a.state = s.state;
  a.out = s.partial;
  a.E = s.Eself;
  a.B = s.Bself;
  a.stats = s.stats;
  a.err = s.err;
  a.N = (int)s.N;
  a.D = s.D;
  a.nbunch = s.nbunch;
  a.bunches = s.bunches;
  a.sched = s.sched;
  a.nitems = pl.nitems;
  a.work = s.work;
  a.fac = s.mlp_fac;
  a.scale = s.scale;
  a.eta_allow = (float)ap.eta_allow;
  a.ext32 = s.ext32;
  a.dump = dump;
  a.wait_limit = pl.wait_limit;
  // the work counter is zeroed by the set-up launch that precedes every pair launch; the bracket dump
  // runs the instance without the adaptive step's reduction (the brackets do not depend on it)
  if (dump)
    launch_mixed<false, true, 0>(proposal, pl, a, st);
  else if (ap.on)
    launch_mixed<true, false, 0>(proposal, pl, a, st);
  else if (pl.shape == 1)
    launch_mixed<false, false, 1>(proposal, pl, a, st);
  else if (pl.shape == 2)
    launch_mixed<false, false, 2>(proposal, pl, a, st);
  else if (pl.shape == 3)
    launch_mixed<false, false, 3>(proposal, pl, a, st);
  else if (pl.shape == 4)
    launch_mixed<false, false, 4>(proposal, pl, a, st);
  else if (pl.shape == 5)
    launch_mixed<false, false, 5>(proposal, pl, a, st);
  else
    launch_mixed<false, false, 0>(proposal, pl, a, st);
  return cudaGetLastError();
}

}  // namespace emppp
