// Internal declarations of the EM-PP CUDA library (not part of the C ABI).
//
// A solver holds one or more independent bunches (particles interact only within their bunch); a
// single-bunch solver is the case nbunch = 1. Particles of all bunches are concatenated: bunch b owns
// global indices off_b .. off_b + n_b - 1. All bunches share the step, time and history depth.
//
// Device data layout (one GPU, all resident in HBM):
//   rec64  [N][D][6] double   history ring, source-major: slot p of particle j holds the position
//                             w (3) and velocity v (3) at the time slot_t[p]; slots are used
//                             modulo D, so one particle's whole history is one contiguous 48*D-byte
//                             run (pair gathers of one source stay within a few cache lines).
//   rec32  [N][D][12] float   FP32 shadow of rec64 (shadow.cuh): hi(3) 1/gamma^2 | lo(3) 0 |
//                             beta - beta_ref (3) gamma^2; 48-byte records, three 16-byte loads each;
//                             origin and beta_ref are per bunch.
//   slot_t [D]                time stamp of each physical slot.
//   slot tables [D]           per step: (c (t_n - t_k))^2 in FP64 and FP32, c (t_n - t_k),
//                             1 / (t_{k+1} - t_k) in FP64 and 1 / (c (t_{k+1} - t_k)) in FP32.
//   ext32  [N][5] float4      per step (mixed path): hi/lo of w_{n-1} + v_{n-1} (t_n - t_{n-1}) - origin,
//                             w_{k0} + v_{k0} (t_n - t_{k0}) - w_n, the chord w_n - w_{k0} with the
//                             threshold of the oldest-slot bound, and the FP32 record's beta - beta_ref,
//                             1/gamma^2 and gamma^2 of slot k0 (kExt* below).
//   u      [N][3]             present proper velocities (FP64).
//   Eself/Bself [N][3]        self fields of the current step; Bout [N][3] = Bself + B_ext.
//   ke     [N]                kinetic-energy terms of the energy monitor (small systems, formed by the push).
//   bunches [nbunch]          offsets, sizes, FP32-split origins and reference velocities.
//   sched   [nbunch]          work split of the pair kernels (target tiles, source chunks, items).
//   StepState (device)        present step n, t_n, dt and the derived window k0..n; kernels read it
//                             so that one captured step can be replayed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace emppp {

// CODATA 2018 (SI)
constexpr double kC = 299792458.0;
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.25663706212e-6;
constexpr double kPi = 3.14159265358979323846;

// device error word bits
enum : int {
  kErrDisc = 1,      // negative discriminant or C2 <= 0 in eq:dt (|v| >= c)
  kErrCoincide = 2,  // eta = 0 or eta . v' <= 0
  kErrNonFinite = 4, // non-finite field or state
  kErrTimeout = 8,   // a bounded wait of a pair kernel on its bulk copies gave up
  kErrBounds = 16,   // debug build: an index outside its range (kDebug)
};

// Debug build (-DEMPPP_DEBUG, library libemppp_debug.so): the pair kernels check every history-window
// offset they turn into a ring slot, and every source and target index, against its range. A failed
// check records kErrBounds in the device error word and goes on with a safe index instead of trapping.
// The release build compiles the checks away.
#ifdef EMPPP_DEBUG
constexpr bool kDebug = true;
#else
constexpr bool kDebug = false;
#endif

// v if lo <= v < hi; otherwise (debug build) the error bit and lo
template <typename I>
__device__ __forceinline__ I debug_index(I v, I lo, I hi, int* err) {
  if (kDebug && (v < lo || v >= hi)) {
    atomicOr(err, kErrBounds);
    return lo;
  }
  return v;
}

struct StepState {
  long long n;           // present (absolute) step index
  double t;              // t_n
  double dt;             // step of the next push
  long long hist_start;  // earliest slot stored since the history was (re)started
  long long k0;          // earliest usable slot max(hist_start, n - D + 1)
  int p0;                // physical slot of k0
  int pn;                // physical slot of n
};

// retarded-time search proposals (values of emppp_proposal)
enum { kPropBisect = 0, kPropClosedForm = 1, kPropMlp = 2 };

// counters, accumulated until reset by the host
enum { kStatOOH = 0, kStatShortcut = 1, kStatBisect = 2, kStatNodeTests = 3, kStatGuard = 4, kStatCount = 8 };

// Guard band of the FP32 node test of the mixed path. The FP32 value of |r - w|^2 formed from hi/lo
// coordinates carries a relative error below 7u (u = 2^-24; two roundings in each component of d,
// one in each square and two in the sum). With the thresholds L^2 (1 + k) / (1 - k) and
// L^2 (1 - k) / (1 + k), each rounded outward to FP32, and k = 32u, a computed |d|^2 beyond a threshold
// puts the exact margin |d|^2 - L^2 beyond about 24u (|d|^2 + L^2), far above the FP64 test's own
// rounding, so the FP32 decision is the FP64 one; between the thresholds the FP64 test decides.
constexpr double kGuardBand = 32.0 * 5.9604644775390625e-08;

// Oldest-slot bound of the mixed path. For a pair whose uniform-motion guess lies beyond the history, the
// node test of slot k0 is |r - w_k0|^2 = |d|^2 + 2 d.c + |c|^2 with d = r - w_n (formed from the staged
// present records) and the source's chord c = w_n - w_k0. In FP32, |d|^2 carries a relative error below
// 7u and d.c (with c rounded to FP32) an absolute one below 3u (|d|^2 + |c|^2). So if
//   2 d.c + |d|^2 (1 - 32u)  >  T (1 + 32u) - |c|^2 (1 - 32u),
// both sides as computed, with T the FP32 upper threshold of slot k0, then the exact |r - w_k0|^2 exceeds
// T (1 + 32u), and the FP32 value the node test forms exceeds T: the test is true by its first
// comparison, with no record of slot k0 loaded. The right-hand side is formed per source in FP64 and
// rounded up (setup_kernel); kChordLo is 1 - 32u.
constexpr double kChordMargin = 32.0 * 5.9604644775390625e-08;
constexpr float kChordLo = 1.0f - 32.0f * 5.9604644775390625e-08f;

// per-source float4s of ext32 (mixed path)
enum {
  kExtSegHi = 0,   // hi of w_{n-1} + v_{n-1} (t_n - t_{n-1}) - origin
  kExtSegLo = 1,   // lo of the same
  kExtLine = 2,    // w_{k0} + v_{k0} (t_n - t_{k0}) - w_n; w: gamma^2 of slot k0 (FP32 record)
  kExtChord = 3,   // FP32 w_n - w_{k0}; w: right-hand side of the oldest-slot bound (+inf without one)
  kExtOldest = 4,  // FP32 record of slot k0: beta - beta_ref, 1/gamma^2
  kExtCount = 5
};

struct SlotTables {
  double* lhs64;    // [D] (c (t_n - t_k))^2, formed as c*(t_n - t_k) then squared (no FMA)
  double* inv_dtk;  // [D] 1 / (t_{k+1} - t_k) for k < n
  // [D] FP32 per slot: (upper threshold of (c (t_n - t_k))^2, lower threshold, c (t_n - t_k),
  // 1 / (c (t_{k+1} - t_k)))
  float4* tab32;
};

struct BunchDesc {
  long long off;       // first particle
  int n;               // particles
  int grp_off;         // learned proposal: first target group of the bunch (groups of kFacGroup targets)
  long long fac_off;   // learned proposal: first delay factor of the bunch ([groups][n] per bunch)
  double origin[3];    // origin of the FP32 hi/lo position split
  double beta_ref[3];  // reference velocity / c of the FP32 velocities
};

// learned proposal, mixed path: targets per group that share one delay factor per source (a multiple of
// every tile shape's targets per block)
constexpr int kFacGroup = 512;

// Work split of the persistent pair kernels, per bunch: items are (source chunk, target tile of the
// tile shape's targets per block)
// pairs taken chunk-major from an atomic counter by resident blocks; per-chunk partial sums are
// reduced in a fixed order afterwards (nchunk > 1).
struct BunchSched {
  int ntb;       // target tiles
  int nchunk;    // source chunks
  int chunk;     // sources per chunk
  int item_off;  // first work item of the bunch (items of all bunches are numbered consecutively)
};

struct DeviceState {
  long long N;  // particles of all bunches
  int D;
  int nbunch;
  const BunchDesc* bunches;  // [nbunch]
  const BunchSched* sched;   // [nbunch]
  const int* bunch_of;       // [N] bunch of each particle
  double* rec64;
  float* rec32;
  double* slot_t;
  SlotTables tab;
  double* u;
  double* wts;  // [N] weights (always present; 1 by default)
  float* kq32;  // [N] -e w_j / (4 pi eps0) in FP32 (mixed path)
  double* Eself;
  double* Bself;
  double* Bout;
  double* ke;       // [N] kinetic-energy terms of the energy monitor, formed by the push (small systems)
  double* partial;  // [C][N][6] per-source-chunk partial sums
  int max_split;    // chunks the partial buffer holds
  int* work;        // work-item counter of the persistent pair kernels (zeroed by the set-up launch)
  unsigned* done;   // blocks of the post-pair launch that have finished (reset by its last block)
  StepState* state;
  unsigned long long* stats;  // [kStatCount]
  int* err;
  double* bsum;     // [nbunch][4] per-bunch reductions (weighted position sums and weight)
  const void* mlp_image;  // BF16 image of the proposal network (EMPPP_PROPOSAL_MLP), or null
  // learned proposal, mixed path: the delay factor e^z of each (target group, source) pair of each bunch,
  // [groups_b][n_b] from BunchDesc::fac_off, written by the factor kernel before each pair evaluation
  float* mlp_fac;
  int ngroups;  // target groups of all bunches
  // [N][kExtCount] FP32 hi/lo of w_{n-1} + v_{n-1} (t_n - t_{n-1}) relative to the bunch origin (the end
  // of the last history segment of eq:linear, from which the mixed path forms near-field retarded points),
  // w_{k0} + v_{k0} (t_n - t_{k0}) - w_n (where the out-of-history line of eq:linear2 is at t_n), and the
  // oldest slot's chord, bound and velocity (the out-of-history pairs' node test and line)
  float4* ext32;
  // adaptive time step (Sec. 2.4)
  unsigned long long* scale;  // [nbunch][2] bit patterns of eta_min (m, by min) and v_max^2 ((m/s)^2, by max)
  double* adapt_info;         // [3] dt, eta_min, v_max of the last adaptive step
};

// adaptive time-step rule (Sec. 2.4)
struct AdaptParams {
  int on;
  double c_dt, eta_allow, dt_min, dt_max;
};

// Warp-wide min of eta and max of dv^2, then one atomic per warp into scale. Non-negative doubles order
// like their bit patterns read as unsigned integers, so the min and max are exact and independent of
// the order of the pairs. Every lane of the warp must call it.
__device__ __forceinline__ void reduce_scale(unsigned long long* scale, double emin, double vmax2) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    emin = fmin(emin, __shfl_xor_sync(0xffffffffu, emin, o));
    vmax2 = fmax(vmax2, __shfl_xor_sync(0xffffffffu, vmax2, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (emin < __longlong_as_double(0x7ff0000000000000LL))
      atomicMin(scale, (unsigned long long)__double_as_longlong(emin));
    if (vmax2 > 0.0) atomicMax(scale + 1, (unsigned long long)__double_as_longlong(vmax2));
  }
}

// stage-switch monitor (Sec. 2.7): the criterion, and the per-bunch record the device keeps
struct EnergyParams {
  int on;
  int hold;    // consecutive steps below eps
  double eps;  // threshold on |dE/dt| (J/s per electron)
};
struct EnergyMon {
  double ebar;    // mean kinetic energy per electron at the present step (J)
  double rate;    // backward difference of ebar over the last step (J/s)
  double t_prev;  // time of ebar
  double t_sw;    // time of the switch step
  long long n_sw; // switch step, -1 before
  int armed;      // the rate has reached eps
  int run;        // consecutive steps below eps since arming
  int switched;
  int pad_;
};

struct BextParams {
  int kind;
  double b[3];
  double m0;
  double center[3];
};

// Tile shapes of the pair kernels (emppp_tuning): targets per block, which is twice the number of sources
// a mixed-path block stages per tile, the mixed path's sources per FP32 partial sum, and the slots of the
// history window each warp of a mixed-path block stages per source by bulk copy (0: none). Shape 0 is the
// default; the FP64 path runs shapes 3 to 5 as shape 0 (its sums are blocked by 64 sources).
#ifndef EMPPP_WIN_SLOTS
#define EMPPP_WIN_SLOTS 16
#endif
constexpr int kNumShapes = 6;
__host__ __device__ constexpr int shape_block(int shape) { return shape == 1 ? 64 : (shape == 2 ? 256 : 128); }
__host__ __device__ constexpr int shape_sub(int shape) { return shape == 3 ? 16 : (shape >= 4 ? 32 : 8); }
__host__ __device__ constexpr int shape_win(int shape) { return shape == 5 ? EMPPP_WIN_SLOTS : 0; }

// launch configuration of a persistent pair kernel
struct PairLaunch {
  int nitems;  // work items of all bunches
  int grid;    // blocks launched
  int shape;   // tile shape (shape_block(shape) threads per block, targets per work item)
  int wait_limit = 1 << 16;  // probes of a bounded wait on a staged history window (window shapes)
};

// item -> (bunch, chunk, target tile): bunches are searched by their first item
__device__ __forceinline__ void decode_item(const BunchSched* __restrict__ sched, int nbunch, int item, int& b,
                                            int& chunk_id, int& tb) {
  int lo = 0, hi = nbunch - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sched[mid].item_off <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  b = lo;
  const int local = item - sched[b].item_off;
  chunk_id = local / sched[b].ntb;
  tb = local - chunk_id * sched[b].ntb;
}

// ---- launchers (each in its own translation unit) ------------------------------------------
// ring.cu
cudaError_t launch_init_slot0(const DeviceState& s, const double* x, const double* u, const double* w,
                              cudaStream_t st);
cudaError_t launch_scatter_slot(const DeviceState& s, int p, const double* W, const double* V, cudaStream_t st);
cudaError_t launch_gather_slot(const DeviceState& s, int p, double* W, double* V, cudaStream_t st);
cudaError_t launch_set_state(const DeviceState& s, long long n, double t, double dt, long long hist_start,
                             const double* u, const double* w, cudaStream_t st);
cudaError_t launch_prep(const DeviceState& s, cudaStream_t st);
cudaError_t launch_setup(const DeviceState& s, bool extrap, cudaStream_t st);
cudaError_t launch_reset_scale(const DeviceState& s, cudaStream_t st);
cudaError_t launch_gather_positions(const DeviceState& s, double* x, cudaStream_t st);
// pair_fp64.cu
// kernel variant of the FP64 pair path: 0 the method, 1 with the adaptive time step's reduction, 2 the
// midpoint reconstruction eq:mid
int max_blocks_pair_fp64(int proposal, int variant, int shape);
// dump (nullptr in the step): [N][N] device array that receives the bracket of every evaluated pair,
// 4 (k1 - k0) + branch (emppp_bracket_dump)
cudaError_t launch_pair_fp64(const DeviceState& s, const int* order, int proposal, int reconstruction,
                             const AdaptParams& ap, const PairLaunch& pl, cudaStream_t st, int* dump = nullptr);
cudaError_t launch_reduce_partials(const DeviceState& s, cudaStream_t st);
cudaError_t launch_zero_self(const DeviceState& s, cudaStream_t st);
// push.cu
cudaError_t launch_step_post(const DeviceState& s, const BextParams& b, const AdaptParams& ap, bool chunked,
                             bool half, bool wide, const EnergyParams* ep, EnergyMon* mon, cudaStream_t st);
cudaError_t launch_half_slot(const DeviceState& s, cudaStream_t st);
// stage2.cu
cudaError_t launch_bunch_sums(const DeviceState& s, cudaStream_t st);
cudaError_t launch_translate(const DeviceState& s, const double* shifts, cudaStream_t st);
cudaError_t launch_transport_chunk(const DeviceState& s, const BextParams& b, double dt, int nsteps, double t_end,
                                   cudaStream_t st);
// order.cu
cudaError_t prepare_target_order();
cudaError_t launch_target_order(const DeviceState& s, unsigned* key, int* order, long long max_bunch, cudaStream_t st);
// mlp.cu
size_t mlp_image_bytes();
cudaError_t launch_build_image(const float* params, void* image, cudaStream_t st);
cudaError_t launch_sample(const DeviceState& s, const int* pairs, long long m, float* feat, double* delay, float* zt,
                          cudaStream_t st);
cudaError_t launch_mlp_forward(const void* image, const float* X, long long m, float* z, int mode, cudaStream_t st);
// delay factors of the learned proposal (mixed path) for the present state, targets in `order` (or index order)
cudaError_t launch_mlp_factors(const DeviceState& s, const int* order, cudaStream_t st);
cudaError_t launch_mlp_train_pass(const void* image, const float* X, const float* T, long long row0, long long rows,
                                  float norm, float* grad, float* loss, int num_sms, cudaStream_t st);
cudaError_t launch_adam(float* p, const float* grad, float* m1, float* m2, float lr, float b1, float b2, float eps,
                        int step, cudaStream_t st);
// energy.cu
cudaError_t launch_energy(const DeviceState& s, const EnergyParams& ep, EnergyMon* mon, bool reset, cudaStream_t st);
constexpr int kEnergyThreads = 256;  // block size of the energy monitor (and of the post-pair launch)
// pair_mixed.cu
int max_blocks_pair_mixed(int proposal, bool adapt, int shape);
cudaError_t launch_pair_mixed(const DeviceState& s, const int* order, int proposal, const AdaptParams& ap,
                              const PairLaunch& pl, cudaStream_t st, int* dump = nullptr);

}  // namespace emppp
