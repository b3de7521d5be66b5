// C ABI of the EM-PP library: handle lifetime, state transfer, the step driver, the stage-2 handoff
// and transport. Every entry point validates its arguments, enqueues work on the handle's stream and
// returns a status; nothing here aborts or prints.
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/emppp.h"
#include "emppp_internal.cuh"

using namespace emppp;

namespace {

thread_local std::string g_last_error;

emppp_status fail(emppp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

#define CU(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(EMPPP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

namespace emppp {
// lets other translation units of the library report an error text through emppp_last_error
void set_error_text(const char* msg) { g_last_error = msg ? msg : ""; }
}  // namespace emppp

namespace {
// NVTX range over a scope of the host code (tracing: the ranges name each step's launches in a timeline
// tool; without one attached they cost a few nanoseconds)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

struct emppp_ctx {
  DeviceState ds{};
  int64_t N = 0;
  int32_t D = 0;
  double dt = 0.0;
  emppp_options opt{};
  cudaStream_t stream = nullptr;
  cudaStream_t aux = nullptr;      // second stream: the target order runs on it beside the set-up launch
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int device = 0;
  int num_sms = 0;
  bool has_state = false;
  int64_t n = 0;           // host mirror of the present step
  double t = 0.0;          // host mirror of t_n
  int64_t hist_start = 0;  // host mirror of the earliest stored slot
  double* staging = nullptr;  // [7N] doubles for host transfers
  std::vector<void*> allocs;
  // bunches
  int nbunch = 1;
  std::vector<BunchDesc> hb;
  std::vector<BunchSched> hs;
  BunchDesc* d_bunches = nullptr;
  BunchSched* d_sched = nullptr;
  int* d_bunch_of = nullptr;
  PairLaunch launch{};
  long long sched_key = -1;  // configuration the uploaded schedule belongs to
  int items_per_block = 16;  // work items per resident block of the pair kernel
  int target_order = 1;      // spatial target order of the pair kernels
  // proposal network image (EMPPP_PROPOSAL_MLP)
  void* mlp_image = nullptr;
  bool has_mlp = false;
  long long fac_count = 0;  // delay factors of the learned proposal (mixed path), all bunches
  // spatial target order of the mixed path
  unsigned* ord_key = nullptr;
  int* order = nullptr;
  // resident blocks per SM of the pair kernels (queried on first use), per proposal
  int blocks_fp64[3][3][kNumShapes] = {};  // [kernel variant][proposal][tile shape]
  int blocks_mixed[2][3][kNumShapes] = {};
  int shape = 0;          // tile shape of the fixed-step pair kernels (emppp_tuning)
  bool dumping = false;   // the bracket dump runs the default shape
  // adaptive time step (Sec. 2.4): the rule, and whether the host mirror of t lags the device
  AdaptParams adapt{0, 0.05, 0.0, 1e-15, 1e-12};
  bool t_stale = false;
  // stage-switch monitor (Sec. 2.7): criterion and per-bunch device record
  EnergyParams energy{0, 1, 0.0};
  long long max_bunch = 0;  // particles of the largest bunch
  EnergyMon* d_mon = nullptr;
  // counters
  int64_t launches = 0;   // kernels launched (cumulative)
  int64_t steps_acc = 0;  // steps since the last stats reset
  int64_t pairs_acc = 0;
  // timing: 4 events per step (step start, pair start, pair end, step end)
  static constexpr int kTimedSteps = 1024;
  std::vector<cudaEvent_t> events;
  int ev_used = 0;
  // one step captured in two variants, replayed by emppp_step: [1] recomputes the spatial target order,
  // [0] reuses the last one
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  int graph_launches[2] = {0, 0};  // kernels per replayed step
  unsigned char graph_key[sizeof(emppp_options) + sizeof(BextParams) + sizeof(AdaptParams) +
                          sizeof(EnergyParams)];  // configuration of both variants
  bool graph_valid[2] = {false, false};
  // Steps since the target order was computed (-1: not for the present state). The order is a
  // permutation of each bunch whatever its age, and a target's sum runs over the sources in a fixed
  // order whichever thread evaluates it, so an older order changes no result; it is recomputed every
  // kOrderEvery steps, since a bunch's particles move far less than their spacing in that time.
  int order_age = -1;
};

// steps between two computations of the spatial target order
constexpr int kOrderEvery = 16;

namespace {

emppp_status check_handle(emppp_handle h) {
  if (!h) return fail(EMPPP_ERR_ARG, "null handle");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return fail(EMPPP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  return EMPPP_OK;
}

template <typename T>
emppp_status dalloc(emppp_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(EMPPP_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
  }
  c->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return EMPPP_OK;
}

// a comparison variant of the step (eq:mid or the half-step field point)
bool is_variant(const emppp_options& o) {
  return o.reconstruction != EMPPP_RECON_LINEAR || o.field_point != EMPPP_FIELD_PRESENT;
}

emppp_status validate_options(const emppp_options* o) {
  if (o->precision != EMPPP_FP64 && o->precision != EMPPP_MIXED)
    return fail(EMPPP_ERR_ARG, "unknown precision %d", o->precision);
  if (o->proposal != EMPPP_PROPOSAL_BISECT && o->proposal != EMPPP_PROPOSAL_CLOSED_FORM &&
      o->proposal != EMPPP_PROPOSAL_MLP)
    return fail(EMPPP_ERR_ARG, "unknown proposal %d", o->proposal);
  if (o->pair_fields != 0 && o->pair_fields != 1) return fail(EMPPP_ERR_ARG, "pair_fields must be 0 or 1");
  if (o->source_split < 0) return fail(EMPPP_ERR_ARG, "source_split must be >= 0");
  if (o->timing != 0 && o->timing != 1) return fail(EMPPP_ERR_ARG, "timing must be 0 or 1");
  if (o->graphs != 0 && o->graphs != 1) return fail(EMPPP_ERR_ARG, "graphs must be 0 or 1");
  if (o->reconstruction != EMPPP_RECON_LINEAR && o->reconstruction != EMPPP_RECON_MIDPOINT)
    return fail(EMPPP_ERR_ARG, "unknown reconstruction %d", o->reconstruction);
  if (o->field_point != EMPPP_FIELD_PRESENT && o->field_point != EMPPP_FIELD_HALF_STEP)
    return fail(EMPPP_ERR_ARG, "unknown field point %d", o->field_point);
  if ((o->reconstruction != EMPPP_RECON_LINEAR || o->field_point != EMPPP_FIELD_PRESENT) &&
      o->precision != EMPPP_FP64)
    return fail(EMPPP_ERR_ARG, "the midpoint reconstruction and the half-step field point run on the FP64 path");
  return EMPPP_OK;
}

void invalidate_graph(emppp_handle h) {
  for (int v = 0; v < 2; v++) {
    if (h->graph_exec[v]) cudaGraphExecDestroy(h->graph_exec[v]);
    if (h->graph[v]) cudaGraphDestroy(h->graph[v]);
    h->graph_exec[v] = nullptr;
    h->graph[v] = nullptr;
    h->graph_valid[v] = false;
  }
  h->order_age = -1;  // every change of state or configuration recomputes the order at the next step
}

// Work split of the persistent pair kernel, per bunch: one block per resident slot of the kernel that
// is launched (occupancy query) and about 16 work items per block over all bunches, so that the uneven
// cost of the items (the branch mix differs across a bunch) evens out; systems too small for that get
// one round of items with short chunks instead. At most max_split chunks per bunch. Uploaded when the
// configuration changes.
constexpr long long kMinChunk = 4;  // fewest sources per chunk

emppp_status update_schedule(emppp_handle c) {
  const bool mixed = c->opt.precision == EMPPP_MIXED;
  const int ad = c->adapt.on ? 1 : 0;
  // FP64 kernel variant: the method (0), with the adaptive step's reduction (1), eq:mid (2)
  const int var64 = c->opt.reconstruction == EMPPP_RECON_MIDPOINT ? 2 : ad;
  // tile shape: the tuned one for the fixed-step kernels; the adaptive-step and eq:mid variants and the
  // bracket dump run the default shape, and the FP64 path runs shape 3 as the default
  int shp = (ad || var64 != 0 || c->dumping) ? 0 : c->shape;
  if (!mixed && shp >= 3) shp = 0;
  const long long TB = shape_block(shp);  // targets per work item (mixed path: twice the sources per staged tile)
  const long long key = (mixed ? 1 : 0) | ((long long)(c->opt.proposal & 3) << 1) |
                        ((long long)c->items_per_block << 3) | ((long long)c->opt.source_split << 13) |
                        ((long long)ad << 40) | ((long long)var64 << 41) | ((long long)shp << 44);
  if (key == c->sched_key) return EMPPP_OK;
  int& nb = mixed ? c->blocks_mixed[ad][c->opt.proposal % 3][shp] : c->blocks_fp64[var64][c->opt.proposal % 3][shp];
  if (nb <= 0)
    nb = mixed ? max_blocks_pair_mixed(c->opt.proposal, ad, shp) : max_blocks_pair_fp64(c->opt.proposal, var64, shp);
  // The source chunking (and with it the order of every target's sum) follows the closed-form
  // variant's residency whatever the proposal, so that all proposals give identical fields; only the
  // number of persistent blocks follows the variant that runs.
  // The history-window shape splits the work like the same shape without the window, so that their fields
  // are identical.
  const int shp_ref = shape_win(shp) > 0 ? 4 : shp;
  int& nref = mixed ? c->blocks_mixed[ad][EMPPP_PROPOSAL_CLOSED_FORM][shp_ref]
                    : c->blocks_fp64[ad][EMPPP_PROPOSAL_CLOSED_FORM][shp_ref];
  if (nref <= 0)
    nref = mixed ? max_blocks_pair_mixed(EMPPP_PROPOSAL_CLOSED_FORM, ad, shp_ref)
                 : max_blocks_pair_fp64(EMPPP_PROPOSAL_CLOSED_FORM, ad, shp_ref);
  // resident blocks in units of 128 threads, so that the item count per SM does not depend on the shape
  const long long R = (long long)nb * c->num_sms;
  const long long Rsched = (long long)nref * c->num_sms * TB / 128;
  const long long Rreal = (long long)nref * c->num_sms;  // resident blocks of the shape
  long long total_tiles = 0;
  for (int b = 0; b < c->nbunch; b++) total_tiles += (c->hb[b].n + TB - 1) / TB;
  const long long tiles128 = [&] {
    long long t = 0;
    for (int b = 0; b < c->nbunch; b++) t += (c->hb[b].n + 127) / 128;
    return t;
  }();
  // chunking of one bunch: about items_per_block items per resident block over all bunches (counted in
  // 128-target tiles), in whole tiles of TB sources and at least 256 sources (small == false); or, for a
  // system too small to fill the resident blocks that way, one round of items with chunks of 4k sources
  // (small == true), since then each block's time is its own chunk length
  auto chunks = [&](long long n, bool small) -> long long {
    long long nchunk;
    if (c->opt.source_split > 0) {
      nchunk = c->opt.source_split;
    } else if (!small) {
      // the FP64 path gathers both rings, so its chunks are cut 4x shorter to keep a chunk's window in L2
      const long long ipb = mixed ? 2LL * c->items_per_block : 4LL * c->items_per_block;
      nchunk = (ipb * Rsched + tiles128 - 1) / tiles128;
      const long long by_size = (n + 255) / 256;
      if (nchunk > by_size) nchunk = by_size;
    } else {
      nchunk = Rreal / total_tiles > 1 ? Rreal / total_tiles : 1;
      const long long by_size = (n + kMinChunk - 1) / kMinChunk;
      if (nchunk > by_size) nchunk = by_size;
    }
    if (nchunk > c->ds.max_split) nchunk = c->ds.max_split;
    if (nchunk < 1) nchunk = 1;
    long long chunk = (n + nchunk - 1) / nchunk;
    return chunk >= TB ? (chunk + TB - 1) / TB * TB : (chunk + kMinChunk - 1) / kMinChunk * kMinChunk;
  };
  long long items_large = 0;
  for (int b = 0; b < c->nbunch; b++) {
    const long long n = c->hb[b].n;
    const long long chunk = chunks(n, false);
    items_large += ((n + TB - 1) / TB) * ((n + chunk - 1) / chunk);
  }
  const bool small = items_large < Rreal;
  int item = 0;
  for (int b = 0; b < c->nbunch; b++) {
    BunchSched& s = c->hs[b];
    const long long n = c->hb[b].n;
    s.ntb = (int)((n + TB - 1) / TB);
    const long long chunk = chunks(n, small);
    s.chunk = (int)chunk;
    s.nchunk = (int)((n + chunk - 1) / chunk);
    s.item_off = item;
    item += s.ntb * s.nchunk;
  }
  c->launch.nitems = item;
  c->launch.grid = (int)(R < item ? R : item);
  c->launch.shape = shp;
  CU(cudaMemcpyAsync(c->d_sched, c->hs.data(), sizeof(BunchSched) * c->nbunch, cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  c->sched_key = key;
  invalidate_graph(c);
  return EMPPP_OK;
}

bool any_chunked(const emppp_ctx* c) {
  for (int b = 0; b < c->nbunch; b++)
    if (c->hs[b].nchunk > 1) return true;
  return false;
}

// the post-pair launch reads the per-chunk partial sums with a warp per particle when a small system is
// split into many chunks (a thread per particle would read them one after another)
bool wide_reduction(const emppp_ctx* c) {
  if (c->N > 16384) return false;
  for (int b = 0; b < c->nbunch; b++)
    if (c->hs[b].nchunk >= 8) return true;
  return false;
}

emppp_status read_err(emppp_handle h) {
  int herr = 0;
  CU(cudaMemcpyAsync(&herr, h->ds.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  if (herr == kErrTimeout) {
    CU(cudaMemsetAsync(h->ds.err, 0, sizeof(int), h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return fail(EMPPP_ERR_TIMEOUT, "a warp's wait on its staged history window gave up (the records were "
                "gathered from the ring instead; the fields are exact)");
  }
  if (herr) {
    return fail(EMPPP_ERR_NUMERIC,
                "device numeric fault (bits 0x%x: 1 = negative discriminant or |v| >= c, 2 = coincident pair, "
                "4 = non-finite state, 8 = wait limit, 16 = index outside its range in the debug build)",
                herr);
  }
  return EMPPP_OK;
}

// with the adaptive time step the device chooses each step's size: refresh the host mirror of t_n
emppp_status sync_time(emppp_handle h) {
  if (!h->t_stale) return EMPPP_OK;
  StepState hs;
  CU(cudaMemcpyAsync(&hs, h->ds.state, sizeof(StepState), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->t = hs.t;
  h->t_stale = false;
  return EMPPP_OK;
}

// copy n doubles from caller memory (host or device) into device memory
emppp_status to_device(emppp_handle h, double* dst, const double* src, size_t n, int is_dev) {
  CU(cudaMemcpyAsync(dst, src, n * sizeof(double), is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     h->stream));
  return EMPPP_OK;
}

emppp_status from_device(emppp_handle h, double* dst, const double* src, size_t n, int is_dev) {
  CU(cudaMemcpyAsync(dst, src, n * sizeof(double), is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     h->stream));
  return EMPPP_OK;
}

// reads 3 doubles at element 3*i of a caller array (host or device)
emppp_status read3(emppp_handle h, const double* a, long long i, int is_dev, double out[3]) {
  if (is_dev) {
    CU(cudaMemcpyAsync(out, a + 3 * i, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  } else {
    memcpy(out, a + 3 * i, 3 * sizeof(double));
  }
  return EMPPP_OK;
}

// Origin of each bunch's FP32 position split and reference velocity of its FP32 velocities: those of
// the bunch's first particle when the state is set. x and v_or_u index the present positions and
// velocities (or proper velocities).
emppp_status set_bunch_frames(emppp_handle h, const double* x, const double* v_or_u, bool is_u, int is_dev) {
  for (int b = 0; b < h->nbunch; b++) {
    double x0[3], v0[3];
    emppp_status st = read3(h, x, h->hb[b].off, is_dev, x0);
    if (st != EMPPP_OK) return st;
    st = read3(h, v_or_u, h->hb[b].off, is_dev, v0);
    if (st != EMPPP_OK) return st;
    double g = 1.0;
    if (is_u) g = sqrt(1.0 + (v0[0] * v0[0] + v0[1] * v0[1] + v0[2] * v0[2]) / (kC * kC));
    for (int c = 0; c < 3; c++) {
      h->hb[b].origin[c] = x0[c];
      h->hb[b].beta_ref[c] = v0[c] / g / kC;
    }
  }
  CU(cudaMemcpyAsync(h->d_bunches, h->hb.data(), sizeof(BunchDesc) * h->nbunch, cudaMemcpyHostToDevice, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return EMPPP_OK;
}

emppp_status ensure_events(emppp_handle h) {
  if (!h->opt.timing || !h->events.empty()) return EMPPP_OK;
  h->events.resize(4 * emppp_ctx::kTimedSteps, nullptr);
  for (auto& e : h->events) CU(cudaEventCreate(&e));
  return EMPPP_OK;
}

emppp_status reset_counters(emppp_handle h) {
  CU(cudaMemsetAsync(h->ds.stats, 0, sizeof(unsigned long long) * kStatCount, h->stream));
  h->steps_acc = 0;
  h->pairs_acc = 0;
  h->ev_used = 0;
  return EMPPP_OK;
}

emppp_status convert_bext(const emppp_bext* bext, BextParams* bp) {
  memset(bp, 0, sizeof(*bp));
  if (!bext) return EMPPP_OK;
  if (bext->kind < EMPPP_BEXT_NONE || bext->kind > EMPPP_BEXT_DIPOLE)
    return fail(EMPPP_ERR_ARG, "unknown background field kind %d", bext->kind);
  bp->kind = bext->kind;
  for (int c = 0; c < 3; c++) {
    bp->b[c] = bext->b[c];
    bp->center[c] = bext->center[c];
  }
  bp->m0 = bext->m0;
  return EMPPP_OK;
}

// enqueues the kernels of one step and reports how many kernels it launched; refresh_order recomputes the
// spatial target order first (else the last one is used)
emppp_status enqueue_step(emppp_handle h, const BextParams& bp, cudaEvent_t* ev, int* nkernels, bool refresh_order) {
  int k = 0;
  if (ev) CU(cudaEventRecord(ev[0], h->stream));
  const bool half = h->opt.pair_fields && h->opt.field_point == EMPPP_FIELD_HALF_STEP;
  if (half) {
    // provisional slot n+1 at t_n + dt/2 holding the half-drifted positions; the clock moves there
    CU(launch_half_slot(h->ds, h->stream));
    k += 1;
  }
  // window, slot tables, work counter and (mixed path) per-source segment vectors; beside it, on the
  // second stream, the spatial order of the targets (it reads only the present positions). Small systems
  // on the mixed path skip the order: a few target tiles gain less from it than its launch costs (the
  // FP64 path keeps it, since it keeps out-of-history and bracketed pairs in separate warps).
  const bool mixed_pairs = h->opt.pair_fields && h->opt.precision == EMPPP_MIXED;
  const bool ordered = h->opt.pair_fields && h->target_order && !(mixed_pairs && h->N <= 2048);
  {
    NvtxRange r("emppp:setup");
    if (ordered && refresh_order) {
      CU(cudaEventRecord(h->ev_fork, h->stream));
      CU(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
      CU(launch_target_order(h->ds, h->ord_key, h->order, h->max_bunch, h->aux));
      CU(cudaEventRecord(h->ev_join, h->aux));
      k += 1;
    }
    CU(launch_setup(h->ds, mixed_pairs, h->stream));
    k += 1;
  }
  if (ordered && refresh_order) CU(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  if (ev) CU(cudaEventRecord(ev[1], h->stream));
  if (h->opt.pair_fields) {
    NvtxRange r("emppp:pair_fields");
    if (h->opt.precision == EMPPP_MIXED && h->opt.proposal == EMPPP_PROPOSAL_MLP) {
      // the learned proposal's delay factors of every (target group, source) pair
      CU(launch_mlp_factors(h->ds, ordered ? h->order : nullptr, h->stream));
      k += 1;
    }
    if (h->opt.precision == EMPPP_MIXED)
      CU(launch_pair_mixed(h->ds, ordered ? h->order : nullptr, h->opt.proposal, h->adapt, h->launch, h->stream));
    else
      CU(launch_pair_fp64(h->ds, ordered ? h->order : nullptr, h->opt.proposal, h->opt.reconstruction, h->adapt,
                          h->launch, h->stream));
    k += 1;
  } else {
    CU(launch_zero_self(h->ds, h->stream));
    k += 1;
  }
  if (ev) CU(cudaEventRecord(ev[2], h->stream));
  // partial sums, step size (Sec. 2.4), push and append (Sec. 2.3), clock advance: one launch
  const bool chunked = h->opt.pair_fields && any_chunked(h);
  // small systems of few bunches: the energy monitor runs in the post-pair launch's last block (its own
  // launch evaluates the bunches in parallel, one block each)
  const bool fused_energy = h->energy.on && h->N <= 16384 && h->nbunch <= 8;
  NvtxRange r_post("emppp:push_append");
  CU(launch_step_post(h->ds, bp, h->adapt, chunked, half, chunked && wide_reduction(h),
                      fused_energy ? &h->energy : nullptr, h->d_mon, h->stream));
  k += 1;
  if (h->energy.on && !fused_energy) {
    // mean energy of the new state and the switch criterion (Sec. 2.7)
    CU(launch_energy(h->ds, h->energy, h->d_mon, false, h->stream));
    k += 1;
  }
  if (ev) CU(cudaEventRecord(ev[3], h->stream));
  *nkernels = k;
  return EMPPP_OK;
}

// captures one step into a CUDA graph for the current configuration (options and background field), in the
// variant that recomputes the target order (refresh_order) or the one that reuses it
emppp_status capture_step(emppp_handle h, const BextParams& bp, bool refresh_order) {
  const int v = refresh_order ? 1 : 0;
  unsigned char key[sizeof(emppp_options) + sizeof(BextParams) + sizeof(AdaptParams) + sizeof(EnergyParams)];
  memset(key, 0, sizeof(key));
  memcpy(key, &h->opt, sizeof(emppp_options));
  memcpy(key + sizeof(emppp_options), &bp, sizeof(BextParams));
  memcpy(key + sizeof(emppp_options) + sizeof(BextParams), &h->adapt, sizeof(AdaptParams));
  memcpy(key + sizeof(emppp_options) + sizeof(BextParams) + sizeof(AdaptParams), &h->energy, sizeof(EnergyParams));
  if (memcmp(key, h->graph_key, sizeof(key)) != 0) {
    const int age = h->order_age;
    invalidate_graph(h);
    h->order_age = age;  // a new field or option does not move the particles
    memcpy(h->graph_key, key, sizeof(key));
  }
  if (h->graph_valid[v]) return EMPPP_OK;
  CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  int k = 0;
  emppp_status st = enqueue_step(h, bp, nullptr, &k, refresh_order);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (st != EMPPP_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(EMPPP_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->graph_exec[v], g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(EMPPP_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(e));
  }
  h->graph[v] = g;
  h->graph_launches[v] = k;
  h->graph_valid[v] = true;
  return EMPPP_OK;
}

emppp_status create_impl(int32_t nbunch, const int64_t* nper, int32_t history_depth, double dt,
                         const emppp_options* opt, void* cuda_stream, emppp_handle* out) {
  if (!out) return fail(EMPPP_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (nbunch < 1 || !nper) return fail(EMPPP_ERR_ARG, "nbunch must be >= 1 with n_per_bunch given");
  long long n = 0;
  for (int b = 0; b < nbunch; b++) {
    if (nper[b] < 1) return fail(EMPPP_ERR_ARG, "every bunch needs n >= 1 (bunch %d has %lld)", b, (long long)nper[b]);
    n += nper[b];
  }
  if (history_depth < 2) return fail(EMPPP_ERR_ARG, "history_depth must be >= 2 (got %d)", history_depth);
  if (!(dt > 0.0) || !(dt < 1e300)) return fail(EMPPP_ERR_ARG, "dt must be positive and finite");
  if ((double)n * (double)history_depth > 4e10) return fail(EMPPP_ERR_ARG, "n * history_depth too large");
  if (n > 2147483647LL) return fail(EMPPP_ERR_ARG, "the total particle count must be below 2^31");
  emppp_options o;
  emppp_default_options(&o);
  if (opt) o = *opt;
  emppp_status st = validate_options(&o);
  if (st != EMPPP_OK) return st;

  emppp_ctx* c = new (std::nothrow) emppp_ctx();
  if (!c) return fail(EMPPP_ERR_OOM, "host allocation failed");
  c->N = n;
  c->D = history_depth;
  c->dt = dt;
  c->opt = o;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->nbunch = nbunch;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = prepare_target_order();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->aux) cudaStreamDestroy(c->aux);
    delete c;
    return fail(EMPPP_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
  }
  c->hb.resize(nbunch);
  c->hs.resize(nbunch);
  std::vector<int> bunch_of((size_t)n);
  long long off = 0, fac_off = 0;
  int grp_off = 0;
  for (int b = 0; b < nbunch; b++) {
    memset(&c->hb[b], 0, sizeof(BunchDesc));
    c->hb[b].off = off;
    c->hb[b].n = (int)nper[b];
    // learned proposal: target groups of the bunch and its delay factors [groups][n]
    const int groups = (int)((nper[b] + kFacGroup - 1) / kFacGroup);
    c->hb[b].grp_off = grp_off;
    c->hb[b].fac_off = fac_off;
    grp_off += groups;
    fac_off += (long long)groups * nper[b];
    if (nper[b] > c->max_bunch) c->max_bunch = nper[b];
    for (long long k = 0; k < nper[b]; k++) bunch_of[(size_t)(off + k)] = b;
    off += nper[b];
  }
  DeviceState& s = c->ds;
  s.N = n;
  s.D = history_depth;
  s.nbunch = nbunch;
  s.ngroups = grp_off;
  s.mlp_fac = nullptr;  // allocated by the first emppp_set_proposal
  c->fac_count = fac_off;
  const size_t N = (size_t)n, D = (size_t)history_depth;
  {
    // partial sums of up to 64 source chunks within 1 GiB, or up to 256 chunks for small systems, whose
    // few target tiles need many chunks to fill the GPU (within 256 MiB)
    const long long by_mem = (1LL << 30) / ((long long)n * 48);
    const long long small = (256LL << 20) / ((long long)n * 48);
    long long ms = by_mem > 64 ? 64 : by_mem;
    if (small > ms) ms = small > 256 ? 256 : small;
    s.max_split = (int)(ms < 1 ? 1 : ms);
  }
#define ALLOC(p, cnt)            \
  do {                           \
    st = dalloc(c, &(p), (cnt)); \
    if (st != EMPPP_OK) {        \
      emppp_destroy(c);          \
      return st;                 \
    }                            \
  } while (0)
  ALLOC(s.rec64, N * D * 6);
  ALLOC(s.rec32, N * D * 12);
  ALLOC(s.slot_t, D);
  ALLOC(s.tab.lhs64, D);
  ALLOC(s.tab.inv_dtk, D);
  ALLOC(s.tab.tab32, D);
  ALLOC(s.u, N * 3);
  ALLOC(s.wts, N);
  ALLOC(s.kq32, N);
  ALLOC(s.Eself, N * 3);
  ALLOC(s.Bself, N * 3);
  ALLOC(s.Bout, N * 3);
  ALLOC(s.ke, N);
  ALLOC(s.partial, (size_t)s.max_split * N * 6);
  ALLOC(s.state, 1);
  ALLOC(s.work, 1);
  ALLOC(s.done, 1);
  if (cudaMemset(s.done, 0, sizeof(unsigned)) != cudaSuccess || cudaMemset(s.work, 0, sizeof(int)) != cudaSuccess) {
    emppp_destroy(c);
    return fail(EMPPP_ERR_CUDA, "zeroing the launch counters failed");
  }
  ALLOC(s.stats, kStatCount);
  ALLOC(s.err, 1);
  ALLOC(s.bsum, (size_t)nbunch * 4);
  ALLOC(s.scale, (size_t)nbunch * 2);
  ALLOC(s.adapt_info, 3);
  ALLOC(s.ext32, N * kExtCount);
  ALLOC(c->d_mon, (size_t)nbunch);
  ALLOC(c->staging, N * 7);
  ALLOC(c->ord_key, N);
  ALLOC(c->order, N);
  ALLOC(c->d_bunches, (size_t)nbunch);
  ALLOC(c->d_sched, (size_t)nbunch);
  ALLOC(c->d_bunch_of, N);
  {
    unsigned char* img = nullptr;
    ALLOC(img, mlp_image_bytes());
    c->mlp_image = img;
  }
#undef ALLOC
  s.bunches = c->d_bunches;
  s.sched = c->d_sched;
  s.bunch_of = c->d_bunch_of;
  s.mlp_image = c->mlp_image;
  e = cudaMemcpyAsync(c->d_bunch_of, bunch_of.data(), sizeof(int) * N, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_bunches, c->hb.data(), sizeof(BunchDesc) * nbunch, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.err, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.stats, 0, sizeof(unsigned long long) * kStatCount, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.Eself, 0, sizeof(double) * N * 3, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.Bout, 0, sizeof(double) * N * 3, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    emppp_destroy(c);
    return fail(EMPPP_ERR_CUDA, "initialisation: %s", cudaGetErrorString(e));
  }
  if ((st = ensure_events(c)) != EMPPP_OK || (st = update_schedule(c)) != EMPPP_OK) {
    emppp_destroy(c);
    return st;
  }
  *out = c;
  return EMPPP_OK;
}

}  // namespace

extern "C" {

EMPPP_API const char* emppp_version(void) { return "emppp 0.2 (sm_103a)"; }

EMPPP_API const char* emppp_last_error(void) { return g_last_error.c_str(); }

EMPPP_API void emppp_default_options(emppp_options* out) {
  if (!out) return;
  memset(out, 0, sizeof(*out));
  out->precision = EMPPP_FP64;
  out->proposal = EMPPP_PROPOSAL_BISECT;
  out->pair_fields = 1;
  out->source_split = 0;
  out->timing = 0;
  out->graphs = 1;
}

EMPPP_API emppp_status emppp_create(int64_t n, int32_t history_depth, double dt, const emppp_options* opt,
                                    void* cuda_stream, emppp_handle* out) {
  if (n < 1) {
    if (out) *out = nullptr;
    return fail(EMPPP_ERR_ARG, "n must be >= 1 (got %lld)", (long long)n);
  }
  return create_impl(1, &n, history_depth, dt, opt, cuda_stream, out);
}

EMPPP_API emppp_status emppp_create_batch(int32_t nbunch, const int64_t* n_per_bunch, int32_t history_depth,
                                          double dt, const emppp_options* opt, void* cuda_stream,
                                          emppp_handle* out) {
  return create_impl(nbunch, n_per_bunch, history_depth, dt, opt, cuda_stream, out);
}

EMPPP_API void emppp_destroy(emppp_handle h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream)
    cudaStreamSynchronize(h->stream);
  else
    cudaDeviceSynchronize();
  invalidate_graph(h);
  for (cudaEvent_t e : h->events)
    if (e) cudaEventDestroy(e);
  if (h->aux) {
    cudaStreamSynchronize(h->aux);
    cudaStreamDestroy(h->aux);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (void* p : h->allocs) cudaFree(p);
  delete h;
}

EMPPP_API emppp_status emppp_set_particles(emppp_handle h, const double* x, const double* u, const double* w,
                                           int32_t is_device_ptr) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!x || !u) return fail(EMPPP_ERR_ARG, "x and u must not be NULL");
  const size_t N = (size_t)h->N;
  const double* dx = x;
  const double* du = u;
  const double* dw = w;
  if (!is_device_ptr) {
    double* sx = h->staging;
    double* su = h->staging + 3 * N;
    double* sw = h->staging + 6 * N;
    if ((st = to_device(h, sx, x, 3 * N, 0)) != EMPPP_OK) return st;
    if ((st = to_device(h, su, u, 3 * N, 0)) != EMPPP_OK) return st;
    if (w && (st = to_device(h, sw, w, N, 0)) != EMPPP_OK) return st;
    dx = sx;
    du = su;
    dw = w ? sw : nullptr;
  }
  if ((st = set_bunch_frames(h, x, u, true, is_device_ptr)) != EMPPP_OK) return st;
  CU(launch_set_state(h->ds, 0, 0.0, h->dt, 0, du, dw, h->stream));
  CU(launch_init_slot0(h->ds, dx, du, dw, h->stream));
  CU(launch_reset_scale(h->ds, h->stream));
  h->launches += 3;
  if (h->energy.on) {
    CU(launch_energy(h->ds, h->energy, h->d_mon, true, h->stream));
    h->launches += 1;
  }
  h->t_stale = false;
  if ((st = reset_counters(h)) != EMPPP_OK) return st;
  CU(cudaMemsetAsync(h->ds.Eself, 0, sizeof(double) * N * 3, h->stream));
  CU(cudaMemsetAsync(h->ds.Bout, 0, sizeof(double) * N * 3, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->n = 0;
  h->t = 0.0;
  h->hist_start = 0;
  h->has_state = true;
  h->order_age = -1;  // a new state: the next step recomputes the target order
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_set_history(emppp_handle h, int64_t n, int32_t nslots, const double* T,
                                         const double* W, const double* V, const double* u, const double* w,
                                         int32_t is_device_ptr) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!T || !W || !V || !u) return fail(EMPPP_ERR_ARG, "T, W, V and u must not be NULL");
  if (n < 0) return fail(EMPPP_ERR_ARG, "n must be >= 0");
  const int64_t want = n + 1 < h->D ? n + 1 : h->D;
  if (nslots != want)
    return fail(EMPPP_ERR_ARG, "nslots must be min(n + 1, depth) = %lld (got %d)", (long long)want, nslots);
  const size_t N = (size_t)h->N;
  std::vector<double> hT(nslots);
  if (is_device_ptr) {
    CU(cudaMemcpyAsync(hT.data(), T, sizeof(double) * nslots, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  } else {
    memcpy(hT.data(), T, sizeof(double) * nslots);
  }
  for (int s = 0; s < nslots; s++) {
    if (!(hT[s] == hT[s]) || (s > 0 && !(hT[s] > hT[s - 1])))
      return fail(EMPPP_ERR_ARG, "time stamps must be finite and strictly increasing (slot %d)", s);
  }
  // FP32 frames: the present position and velocity of each bunch's first particle
  const double* Wlast = W + (size_t)(nslots - 1) * N * 3;
  const double* Vlast = V + (size_t)(nslots - 1) * N * 3;
  if ((st = set_bunch_frames(h, Wlast, Vlast, false, is_device_ptr)) != EMPPP_OK) return st;
  std::vector<double> ht((size_t)h->D, 0.0);
  for (int s = 0; s < nslots; s++) {
    const int64_t k = n - nslots + 1 + s;
    const int p = (int)(k % h->D);
    ht[p] = hT[s];
    const double* Ws = W + (size_t)s * N * 3;
    const double* Vs = V + (size_t)s * N * 3;
    if (!is_device_ptr) {
      if ((st = to_device(h, h->staging, Ws, 3 * N, 0)) != EMPPP_OK) return st;
      if ((st = to_device(h, h->staging + 3 * N, Vs, 3 * N, 0)) != EMPPP_OK) return st;
      Ws = h->staging;
      Vs = h->staging + 3 * N;
    }
    CU(launch_scatter_slot(h->ds, p, Ws, Vs, h->stream));
    h->launches += 1;
    if (!is_device_ptr) CU(cudaStreamSynchronize(h->stream));  // staging is reused by the next slot
  }
  CU(cudaMemcpyAsync(h->ds.slot_t, ht.data(), sizeof(double) * h->D, cudaMemcpyHostToDevice, h->stream));
  const double* du = u;
  const double* dw = w;
  if (!is_device_ptr) {
    if ((st = to_device(h, h->staging, u, 3 * N, 0)) != EMPPP_OK) return st;
    if (w && (st = to_device(h, h->staging + 6 * N, w, N, 0)) != EMPPP_OK) return st;
    du = h->staging;
    dw = w ? h->staging + 6 * N : nullptr;
  }
  const int64_t hs = n - nslots + 1;
  CU(launch_set_state(h->ds, n, hT[nslots - 1], h->dt, hs, du, dw, h->stream));
  CU(launch_reset_scale(h->ds, h->stream));
  h->launches += 2;
  if (h->energy.on) {
    CU(launch_energy(h->ds, h->energy, h->d_mon, true, h->stream));
    h->launches += 1;
  }
  h->t_stale = false;
  if ((st = reset_counters(h)) != EMPPP_OK) return st;
  CU(cudaMemsetAsync(h->ds.Eself, 0, sizeof(double) * N * 3, h->stream));
  CU(cudaMemsetAsync(h->ds.Bout, 0, sizeof(double) * N * 3, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->n = n;
  h->t = hT[nslots - 1];
  h->hist_start = hs;
  h->has_state = true;
  h->order_age = -1;  // a new state: the next step recomputes the target order
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_get_history(emppp_handle h, int64_t* n_now, int32_t* nslots, double* T, double* W,
                                         double* V, double* u, int32_t is_device_ptr) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!h->has_state) return fail(EMPPP_ERR_STATE, "no state: call emppp_set_particles first");
  if ((st = read_err(h)) != EMPPP_OK) return st;
  const size_t N = (size_t)h->N;
  const int64_t stored = h->n - h->hist_start + 1;
  const int32_t ns = (int32_t)(stored < h->D ? stored : h->D);
  std::vector<double> ht((size_t)h->D);
  CU(cudaMemcpyAsync(ht.data(), h->ds.slot_t, sizeof(double) * h->D, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  std::vector<double> hTs(ns);
  for (int s = 0; s < ns; s++) {
    const int64_t k = h->n - ns + 1 + s;
    const int p = (int)(k % h->D);
    hTs[s] = ht[p];
    double* Ws = W ? W + (size_t)s * N * 3 : nullptr;
    double* Vs = V ? V + (size_t)s * N * 3 : nullptr;
    if (is_device_ptr) {
      CU(launch_gather_slot(h->ds, p, Ws, Vs, h->stream));
      h->launches += 1;
    } else {
      CU(launch_gather_slot(h->ds, p, h->staging, h->staging + 3 * N, h->stream));
      h->launches += 1;
      if (Ws && (st = from_device(h, Ws, h->staging, 3 * N, 0)) != EMPPP_OK) return st;
      if (Vs && (st = from_device(h, Vs, h->staging + 3 * N, 3 * N, 0)) != EMPPP_OK) return st;
      CU(cudaStreamSynchronize(h->stream));
    }
  }
  if (T) {
    if (is_device_ptr)
      CU(cudaMemcpyAsync(T, hTs.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, h->stream));
    else
      memcpy(T, hTs.data(), sizeof(double) * ns);
  }
  if (u && (st = from_device(h, u, h->ds.u, 3 * N, is_device_ptr)) != EMPPP_OK) return st;
  CU(cudaStreamSynchronize(h->stream));
  if (n_now) *n_now = h->n;
  if (nslots) *nslots = ns;
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_step(emppp_handle h, int64_t nsteps, const emppp_bext* bext) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!h->has_state) return fail(EMPPP_ERR_STATE, "no state: call emppp_set_particles first");
  if (nsteps < 0) return fail(EMPPP_ERR_ARG, "nsteps must be >= 0");
  BextParams bp;
  if ((st = convert_bext(bext, &bp)) != EMPPP_OK) return st;
  if (h->opt.proposal == EMPPP_PROPOSAL_MLP && h->opt.pair_fields && !h->has_mlp)
    return fail(EMPPP_ERR_STATE, "the MLP proposal needs a network: call emppp_set_proposal first");
  if ((st = update_schedule(h)) != EMPPP_OK) return st;
  const bool use_graph = h->opt.graphs && !h->opt.timing && h->stream != nullptr && nsteps > 1;
  NvtxRange r_step(use_graph ? "emppp_step (graph replay)" : "emppp_step");
  long long pairs_per_step = 0;
  if (h->opt.pair_fields)
    for (int b = 0; b < h->nbunch; b++) pairs_per_step += (long long)h->hb[b].n * (h->hb[b].n - 1);
  for (int64_t k = 0; k < nsteps; k++) {
    int nk = 0;
    const bool refresh = h->order_age < 0 || h->order_age >= kOrderEvery - 1;
    if (use_graph) {
      if ((st = capture_step(h, bp, refresh)) != EMPPP_OK) return st;
      const int v = refresh ? 1 : 0;
      CU(cudaGraphLaunch(h->graph_exec[v], h->stream));
      nk = h->graph_launches[v];
    } else {
      cudaEvent_t* ev = nullptr;
      if (h->opt.timing && h->ev_used < emppp_ctx::kTimedSteps) ev = &h->events[4 * h->ev_used++];
      if ((st = enqueue_step(h, bp, ev, &nk, refresh)) != EMPPP_OK) return st;
    }
    h->order_age = refresh ? 0 : h->order_age + 1;
    h->launches += nk;
    h->pairs_acc += pairs_per_step;
    h->steps_acc += 1;
    h->n += 1;
    if (h->adapt.on)
      h->t_stale = true;  // each step's size is chosen on the device
    else
      h->t = h->t + h->dt;
  }
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_handoff(emppp_handle h, const double* center) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!h->has_state) return fail(EMPPP_ERR_STATE, "no state: call emppp_set_particles first");
  if (!center) return fail(EMPPP_ERR_ARG, "center is NULL");
  if ((st = read_err(h)) != EMPPP_OK) return st;
  CU(launch_bunch_sums(h->ds, h->stream));
  std::vector<double> sums((size_t)h->nbunch * 4);
  CU(cudaMemcpyAsync(sums.data(), h->ds.bsum, sizeof(double) * sums.size(), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  std::vector<double> shifts((size_t)h->nbunch * 3);
  for (int b = 0; b < h->nbunch; b++) {
    const double wsum = sums[4 * b + 3];
    if (!(wsum != 0.0)) return fail(EMPPP_ERR_NUMERIC, "bunch %d has zero total weight", b);
    for (int c = 0; c < 3; c++) {
      shifts[3 * b + c] = center[c] - sums[4 * b + c] / wsum;
      h->hb[b].origin[c] += shifts[3 * b + c];  // keeps x - origin unchanged
    }
  }
  CU(cudaMemcpyAsync(h->d_bunches, h->hb.data(), sizeof(BunchDesc) * h->nbunch, cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemcpyAsync(h->ds.bsum, shifts.data(), sizeof(double) * shifts.size(), cudaMemcpyHostToDevice, h->stream));
  CU(launch_translate(h->ds, h->ds.bsum, h->stream));
  h->launches += 2;
  CU(cudaStreamSynchronize(h->stream));
  h->hist_start = h->n;
  invalidate_graph(h);
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_transport(emppp_handle h, int64_t nsteps, double dt, const emppp_bext* bext) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!h->has_state) return fail(EMPPP_ERR_STATE, "no state: call emppp_set_particles first");
  if (nsteps < 0) return fail(EMPPP_ERR_ARG, "nsteps must be >= 0");
  if (!(dt > 0.0) || !(dt < 1e300)) return fail(EMPPP_ERR_ARG, "dt must be positive and finite");
  BextParams bp;
  if ((st = convert_bext(bext, &bp)) != EMPPP_OK) return st;
  if ((st = sync_time(h)) != EMPPP_OK) return st;
  const int64_t kChunk = 4096;
  for (int64_t done = 0; done < nsteps;) {
    const int k = (int)(nsteps - done < kChunk ? nsteps - done : kChunk);
    double t = h->t;
    for (int s = 0; s < k; s++) t = t + dt;
    CU(launch_transport_chunk(h->ds, bp, dt, k, t, h->stream));
    h->launches += 2;
    h->n += k;
    h->t = t;
    h->hist_start = h->n;
    done += k;
  }
  invalidate_graph(h);
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_get_state(emppp_handle h, double* x, double* u, double* t_now, int64_t* n_now,
                                       int32_t is_device_ptr) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!h->has_state) return fail(EMPPP_ERR_STATE, "no state: call emppp_set_particles first");
  if ((st = read_err(h)) != EMPPP_OK) return st;
  const size_t N = (size_t)h->N;
  if (x) {
    h->launches += 1;
    if (is_device_ptr) {
      CU(launch_gather_positions(h->ds, x, h->stream));
    } else {
      CU(launch_gather_positions(h->ds, h->staging, h->stream));
      if ((st = from_device(h, x, h->staging, 3 * N, 0)) != EMPPP_OK) return st;
    }
  }
  if (u && (st = from_device(h, u, h->ds.u, 3 * N, is_device_ptr)) != EMPPP_OK) return st;
  CU(cudaStreamSynchronize(h->stream));
  if ((st = sync_time(h)) != EMPPP_OK) return st;
  if (t_now) *t_now = h->t;
  if (n_now) *n_now = h->n;
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_get_fields(emppp_handle h, double* E, double* B, int32_t is_device_ptr) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!h->has_state) return fail(EMPPP_ERR_STATE, "no state: call emppp_set_particles first");
  if ((st = read_err(h)) != EMPPP_OK) return st;
  const size_t N = (size_t)h->N;
  if (E && (st = from_device(h, E, h->ds.Eself, 3 * N, is_device_ptr)) != EMPPP_OK) return st;
  if (B && (st = from_device(h, B, h->ds.Bout, 3 * N, is_device_ptr)) != EMPPP_OK) return st;
  CU(cudaStreamSynchronize(h->stream));
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_get_stats(emppp_handle h, emppp_stats* out) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!out) return fail(EMPPP_ERR_ARG, "out is NULL");
  unsigned long long hs[kStatCount];
  CU(cudaMemcpyAsync(hs, h->ds.stats, sizeof(hs), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  memset(out, 0, sizeof(*out));
  out->steps = h->steps_acc;
  out->pairs = h->pairs_acc;
  out->out_of_history = (int64_t)hs[kStatOOH];
  out->shortcut = (int64_t)hs[kStatShortcut];
  out->bisection = (int64_t)hs[kStatBisect];
  out->node_tests = (int64_t)hs[kStatNodeTests];
  out->guard_fallbacks = (int64_t)hs[kStatGuard];
  out->kernel_launches = h->launches;
  double pair_ms = 0.0, step_ms = 0.0;
  for (int k = 0; k < h->ev_used; k++) {
    float a = 0.f, b = 0.f;
    CU(cudaEventElapsedTime(&a, h->events[4 * k + 1], h->events[4 * k + 2]));
    CU(cudaEventElapsedTime(&b, h->events[4 * k + 0], h->events[4 * k + 3]));
    pair_ms += a;
    step_ms += b;
  }
  out->pair_ms = pair_ms;
  out->step_ms = step_ms;
  out->timed_steps = h->ev_used;
  double ai[3] = {h->dt, 0.0, 0.0};
  if (h->has_state) {
    CU(cudaMemcpyAsync(ai, h->ds.adapt_info, sizeof(ai), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  out->dt_last = ai[0];
  out->eta_min = ai[1];
  out->v_max = ai[2];
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_reset_stats(emppp_handle h) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  return reset_counters(h);
}

// one evaluation of the self fields of the present state: slot tables, target order, pair kernel,
// reduction (no push: the state does not change)
emppp_status enqueue_fields(emppp_handle h, int* dump = nullptr) {
  CU(launch_setup(h->ds, h->opt.precision == EMPPP_MIXED, h->stream));
  const bool ordered = h->target_order != 0;
  if (ordered) CU(launch_target_order(h->ds, h->ord_key, h->order, h->max_bunch, h->stream));
  if (h->opt.precision == EMPPP_MIXED) {
    if (h->opt.proposal == EMPPP_PROPOSAL_MLP) {
      CU(launch_mlp_factors(h->ds, ordered ? h->order : nullptr, h->stream));
      h->launches += 1;
    }
    CU(launch_pair_mixed(h->ds, ordered ? h->order : nullptr, h->opt.proposal, h->adapt, h->launch, h->stream,
                         dump));
  } else {
    CU(launch_pair_fp64(h->ds, ordered ? h->order : nullptr, h->opt.proposal, h->opt.reconstruction, h->adapt,
                        h->launch, h->stream, dump));
  }
  if (any_chunked(h)) CU(launch_reduce_partials(h->ds, h->stream));
  h->launches += 2 + (ordered ? 1 : 0) + (any_chunked(h) ? 1 : 0);
  return EMPPP_OK;
}

// tile shape of (targets per block, sources per partial sum, history window on), -1 if it is none
static int shape_of(int targets_per_block, int sources_per_sum, int history_window) {
  const int tb = targets_per_block == 0 ? 128 : targets_per_block;
  const int ss = sources_per_sum == 0 ? 8 : sources_per_sum;
  for (int k = 0; k < kNumShapes; k++)
    if (shape_block(k) == tb && shape_sub(k) == ss && (shape_win(k) > 0) == (history_window != 0)) return k;
  return -1;
}

EMPPP_API emppp_status emppp_autotune(emppp_handle h, emppp_tuning_report* report) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!h->has_state) return fail(EMPPP_ERR_STATE, "no state: call emppp_set_particles first");
  if (!h->opt.pair_fields) return fail(EMPPP_ERR_STATE, "pair fields are off: nothing to tune");
  if (h->opt.proposal == EMPPP_PROPOSAL_MLP && !h->has_mlp)
    return fail(EMPPP_ERR_STATE, "the MLP proposal needs a network: call emppp_set_proposal first");
  if ((st = read_err(h)) != EMPPP_OK) return st;
  const int ipb[5] = {4, 8, 16, 32, 64};
  emppp_tuning_report rep;
  memset(&rep, 0, sizeof(rep));
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  double best_ms = 1e300;
  // one candidate: warm-up, then the best of two timed evaluations
  auto time_candidate = [&](int items, int order, int shape) -> emppp_status {
    h->items_per_block = items;
    h->target_order = order;
    h->shape = shape;
    emppp_status s2 = update_schedule(h);
    if (s2 == EMPPP_OK) s2 = enqueue_fields(h);
    float best = 3.4e38f;
    for (int rpt = 0; rpt < 2 && s2 == EMPPP_OK; rpt++) {
      cudaEventRecord(e0, h->stream);
      s2 = enqueue_fields(h);
      cudaEventRecord(e1, h->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    if (s2 != EMPPP_OK) return s2;
    emppp_tuning& c = rep.cand[rep.ncand];
    c.items_per_block = items;
    c.target_order = order;
    c.targets_per_block = shape_block(shape);
    c.sources_per_sum = shape_sub(shape);
    c.history_window = shape_win(shape);
    c.ms = best;
    if (best < best_ms) {
      best_ms = best;
      rep.best = rep.ncand;
    }
    rep.ncand++;
    return EMPPP_OK;
  };
  // work split and target order at the default shape
  for (int o = 0; o < 2 && st == EMPPP_OK; o++)
    for (int k = 0; k < 5 && st == EMPPP_OK; k++) st = time_candidate(ipb[k], 1 - o, 0);
  // the other tile shapes with the fastest split and order (the adaptive step runs the default shape)
  if (st == EMPPP_OK && !h->adapt.on) {
    const int items = rep.cand[rep.best].items_per_block, order = rep.cand[rep.best].target_order;
    const int nshapes = h->opt.precision == EMPPP_MIXED ? kNumShapes : 3;
    for (int shp = 1; shp < nshapes && st == EMPPP_OK; shp++) st = time_candidate(items, order, shp);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != EMPPP_OK) return st;
  const emppp_tuning& b = rep.cand[rep.best];
  h->items_per_block = b.items_per_block;
  h->target_order = b.target_order;
  h->shape = shape_of(b.targets_per_block, b.sources_per_sum, b.history_window);
  invalidate_graph(h);
  if ((st = update_schedule(h)) != EMPPP_OK) return st;
  if ((st = reset_counters(h)) != EMPPP_OK) return st;
  CU(cudaStreamSynchronize(h->stream));
  if ((st = read_err(h)) != EMPPP_OK) return st;
  if (report) *report = rep;
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_bracket_dump(emppp_handle h, int32_t* brackets, int64_t* k0) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!brackets) return fail(EMPPP_ERR_ARG, "brackets is NULL");
  if (h->N > 65536) return fail(EMPPP_ERR_ARG, "the bracket dump is for systems of at most 65536 particles");
  if (!h->has_state) return fail(EMPPP_ERR_STATE, "no state: call emppp_set_particles first");
  if (!h->opt.pair_fields) return fail(EMPPP_ERR_STATE, "pair fields are off: there are no brackets");
  if (h->opt.field_point != EMPPP_FIELD_PRESENT)
    return fail(EMPPP_ERR_STATE, "the bracket dump evaluates the present field point only");
  if (h->opt.proposal == EMPPP_PROPOSAL_MLP && !h->has_mlp)
    return fail(EMPPP_ERR_STATE, "the MLP proposal needs a network: call emppp_set_proposal first");
  if ((st = read_err(h)) != EMPPP_OK) return st;
  h->dumping = true;  // the dump instances run the default tile shape
  st = update_schedule(h);
  if (st == EMPPP_OK) {
    cudaError_t e = cudaMemsetAsync(brackets, 0xff, sizeof(int32_t) * (size_t)h->N * (size_t)h->N, h->stream);
    st = e == cudaSuccess ? enqueue_fields(h, brackets) : fail(EMPPP_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
  }
  h->dumping = false;
  if (st != EMPPP_OK) return st;
  CU(cudaStreamSynchronize(h->stream));
  if ((st = read_err(h)) != EMPPP_OK) return st;
  if ((st = reset_counters(h)) != EMPPP_OK) return st;
  if (k0) {
    StepState ss;
    CU(cudaMemcpy(&ss, h->ds.state, sizeof(StepState), cudaMemcpyDeviceToHost));
    *k0 = ss.k0;
  }
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_set_tuning(emppp_handle h, const emppp_tuning* tuning) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!tuning || tuning->items_per_block < 1 || tuning->items_per_block > 256 ||
      (tuning->target_order != 0 && tuning->target_order != 1))
    return fail(EMPPP_ERR_ARG, "items_per_block must be in 1..256 and target_order 0 or 1");
  const int shp = shape_of(tuning->targets_per_block, tuning->sources_per_sum, tuning->history_window);
  if (shp < 0)
    return fail(EMPPP_ERR_ARG, "tile shape (%d targets per block, %d sources per sum, history window %d) is not one "
                "of (128, 8), (64, 8), (256, 8), (128, 16), (128, 32) or (128, 32) with the window",
                tuning->targets_per_block, tuning->sources_per_sum, tuning->history_window);
  h->items_per_block = tuning->items_per_block;
  h->target_order = tuning->target_order;
  h->shape = shp;
  invalidate_graph(h);
  return update_schedule(h);
}

EMPPP_API emppp_status emppp_set_wait_limit(emppp_handle h, int32_t probes) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (probes < 0) return fail(EMPPP_ERR_ARG, "probes must be >= 0");
  h->launch.wait_limit = probes;
  invalidate_graph(h);
  return EMPPP_OK;
}

// ---- learned proposal ------------------------------------------------------------------------
EMPPP_API emppp_status emppp_sample_delays(emppp_handle h, const int32_t* pairs, int64_t m, float* features,
                                           double* delays, float* targets, int32_t is_device_ptr) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!h->has_state) return fail(EMPPP_ERR_STATE, "no state: call emppp_set_particles first");
  if (m < 0 || (m > 0 && (!pairs || !features || !delays || !targets))) return fail(EMPPP_ERR_ARG, "bad arguments");
  if (m == 0) return EMPPP_OK;
  std::vector<int32_t> hp;
  const int32_t* pp = pairs;
  if (!is_device_ptr) {
    hp.assign(pairs, pairs + 2 * m);
  } else {
    hp.resize((size_t)(2 * m));
    CU(cudaMemcpyAsync(hp.data(), pairs, sizeof(int32_t) * 2 * m, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  for (int64_t k = 0; k < m; k++) {
    const int32_t i = hp[2 * k], j = hp[2 * k + 1];
    if (i < 0 || j < 0 || i >= h->N || j >= h->N || i == j)
      return fail(EMPPP_ERR_ARG, "pair %lld = (%d, %d) is not two different particles", (long long)k, i, j);
  }
  // device buffers for this call (one-off training-data generation, not the step path)
  void *dp = nullptr, *df = nullptr, *dd = nullptr, *dz = nullptr;
  auto cleanup = [&]() {
    if (!is_device_ptr) {
      cudaFree(dp);
      cudaFree(df);
      cudaFree(dd);
      cudaFree(dz);
    }
  };
  if (!is_device_ptr) {
    if (cudaMalloc(&dp, sizeof(int32_t) * 2 * m) != cudaSuccess || cudaMalloc(&df, sizeof(float) * 10 * m) != cudaSuccess ||
        cudaMalloc(&dd, sizeof(double) * m) != cudaSuccess || cudaMalloc(&dz, sizeof(float) * m) != cudaSuccess) {
      cudaGetLastError();
      cleanup();
      return fail(EMPPP_ERR_OOM, "device buffers for %lld samples", (long long)m);
    }
    cudaMemcpyAsync(dp, hp.data(), sizeof(int32_t) * 2 * m, cudaMemcpyHostToDevice, h->stream);
    pp = static_cast<int32_t*>(dp);
  } else {
    df = features;
    dd = delays;
    dz = targets;
  }
  cudaError_t e = launch_prep(h->ds, h->stream);
  if (e == cudaSuccess)
    e = launch_sample(h->ds, pp, m, static_cast<float*>(df), static_cast<double*>(dd), static_cast<float*>(dz),
                      h->stream);
  if (e == cudaSuccess && !is_device_ptr) {
    e = cudaMemcpyAsync(features, df, sizeof(float) * 10 * m, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(delays, dd, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(targets, dz, sizeof(float) * m, cudaMemcpyDeviceToHost, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cleanup();
  h->launches += 2;
  if (e != cudaSuccess) return fail(EMPPP_ERR_CUDA, "sampling: %s", cudaGetErrorString(e));
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_set_proposal(emppp_handle h, const float* params, int32_t is_device_ptr) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!params) return fail(EMPPP_ERR_ARG, "params is NULL");
  if (h->fac_count > 2147483647LL)
    return fail(EMPPP_ERR_ARG, "the learned proposal's table of delay factors would hold %lld entries, more than "
                "2^31 - 1 (bunches of more than about a million particles)", h->fac_count);
  if (!h->ds.mlp_fac && h->fac_count > 0) {
    // the delay factors of the mixed path's learned proposal: one per (target group, source) pair
    if ((st = dalloc(h, &h->ds.mlp_fac, (size_t)h->fac_count)) != EMPPP_OK) return st;
    invalidate_graph(h);
  }
  float* dparams = nullptr;
  if (cudaMalloc(&dparams, sizeof(float) * EMPPP_MLP_NUM_PARAMS) != cudaSuccess) {
    cudaGetLastError();
    return fail(EMPPP_ERR_OOM, "parameter buffer");
  }
  cudaError_t e = cudaMemcpyAsync(dparams, params, sizeof(float) * EMPPP_MLP_NUM_PARAMS,
                                  is_device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = launch_build_image(dparams, h->mlp_image, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(dparams);
  if (e != cudaSuccess) return fail(EMPPP_ERR_CUDA, "set_proposal: %s", cudaGetErrorString(e));
  h->has_mlp = true;
  h->launches += 1;
  return EMPPP_OK;
}

}  // extern "C"

namespace {

// temporary device buffers of the handle-free network calls
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  bool alloc(size_t n) {
    if (cudaMalloc(&p, n) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return false;
    }
    return true;
  }
};

int device_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

extern "C" {

EMPPP_API emppp_status emppp_mlp_forward(const float* params, const float* features, int64_t m, float* z,
                                         int32_t mode, void* cuda_stream) {
  if (!params || !features || !z || m < 0 || mode < 0 || mode > 1) return fail(EMPPP_ERR_ARG, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  DevBuf img;
  if (!img.alloc(mlp_image_bytes())) return fail(EMPPP_ERR_OOM, "network image");
  CU(launch_build_image(params, img.p, s));
  CU(launch_mlp_forward(img.p, features, m, z, mode, s));
  CU(cudaStreamSynchronize(s));
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_mlp_gradient(const float* params, const float* features, const float* targets,
                                          int64_t m, float* grad, double* loss, void* cuda_stream) {
  if (!params || !features || !targets || !grad || m < 1) return fail(EMPPP_ERR_ARG, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  DevBuf img, dl;
  if (!img.alloc(mlp_image_bytes()) || !dl.alloc(sizeof(float))) return fail(EMPPP_ERR_OOM, "network buffers");
  CU(launch_build_image(params, img.p, s));
  CU(cudaMemsetAsync(grad, 0, sizeof(float) * EMPPP_MLP_NUM_PARAMS, s));
  CU(cudaMemsetAsync(dl.p, 0, sizeof(float), s));
  CU(launch_mlp_train_pass(img.p, features, targets, 0, m, (float)m, grad, static_cast<float*>(dl.p), device_sms(), s));
  float hl = 0.f;
  CU(cudaMemcpyAsync(&hl, dl.p, sizeof(float), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (loss) *loss = (double)hl / (double)m;
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_mlp_train(float* params, const float* features, const float* targets, int64_t m,
                                       const emppp_mlp_config* cfg, float* loss_per_epoch, void* cuda_stream) {
  if (!params || !features || !targets || !cfg || m < 1) return fail(EMPPP_ERR_ARG, "bad arguments");
  if (cfg->epochs < 0 || cfg->batch < 16 || !(cfg->lr > 0.f)) return fail(EMPPP_ERR_ARG, "bad training config");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  DevBuf img, grad, m1, m2, dl;
  const size_t P = sizeof(float) * EMPPP_MLP_NUM_PARAMS;
  if (!img.alloc(mlp_image_bytes()) || !grad.alloc(P) || !m1.alloc(P) || !m2.alloc(P) || !dl.alloc(sizeof(float)))
    return fail(EMPPP_ERR_OOM, "training buffers");
  CU(cudaMemsetAsync(m1.p, 0, P, s));
  CU(cudaMemsetAsync(m2.p, 0, P, s));
  const int sms = device_sms();
  int step = 0;
  const long long batches = (m + cfg->batch - 1) / cfg->batch;
  const long long total = batches * cfg->epochs;
  const bool decay = cfg->lr_final > 0.f && cfg->lr_final < cfg->lr && total > 1;
  for (int ep = 0; ep < cfg->epochs; ep++) {
    CU(cudaMemsetAsync(dl.p, 0, sizeof(float), s));
    for (int64_t r0 = 0; r0 < m; r0 += cfg->batch) {
      const int64_t rows = (m - r0 < cfg->batch) ? m - r0 : cfg->batch;
      CU(launch_build_image(params, img.p, s));
      CU(cudaMemsetAsync(grad.p, 0, P, s));
      CU(launch_mlp_train_pass(img.p, features, targets, r0, rows, (float)rows, static_cast<float*>(grad.p),
                               static_cast<float*>(dl.p), sms, s));
      // cosine schedule from lr (first step) to lr_final (last step)
      const double frac = decay ? (double)step / (double)(total - 1) : 0.0;
      const float lr = decay ? (float)(cfg->lr_final + 0.5 * (cfg->lr - cfg->lr_final) * (1.0 + cos(3.14159265358979323846 * frac)))
                             : cfg->lr;
      CU(launch_adam(params, static_cast<float*>(grad.p), static_cast<float*>(m1.p), static_cast<float*>(m2.p), lr,
                     cfg->beta1, cfg->beta2, cfg->eps, ++step, s));
    }
    float hl = 0.f;
    CU(cudaMemcpyAsync(&hl, dl.p, sizeof(float), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (loss_per_epoch) loss_per_epoch[ep] = hl / (float)m;
  }
  CU(cudaStreamSynchronize(s));
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_set_adaptive_dt(emppp_handle h, const emppp_adaptive_dt* cfg) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  AdaptParams ap;
  memset(&ap, 0, sizeof(ap));
  ap.c_dt = 0.05;
  ap.dt_min = 1e-15;
  ap.dt_max = 1e-12;
  if (cfg && cfg->enable && is_variant(h->opt))
    return fail(EMPPP_ERR_STATE, "the midpoint reconstruction and the half-step field point run with a fixed dt");
  if (cfg && cfg->enable) {
    const bool ok = cfg->c_dt > 0.0 && cfg->c_dt < 1e300 && cfg->eta_allow >= 0.0 && cfg->eta_allow < 1e300 &&
                    cfg->dt_min > 0.0 && cfg->dt_max >= cfg->dt_min && cfg->dt_max < 1e300;
    if (!ok) return fail(EMPPP_ERR_ARG, "adaptive step: need c_dt > 0, eta_allow >= 0, 0 < dt_min <= dt_max, all finite");
    ap.on = 1;
    ap.c_dt = cfg->c_dt;
    ap.eta_allow = cfg->eta_allow;
    ap.dt_min = cfg->dt_min;
    ap.dt_max = cfg->dt_max;
  }
  if ((st = sync_time(h)) != EMPPP_OK) return st;
  const bool was_on = h->adapt.on != 0;
  h->adapt = ap;
  if (was_on && !ap.on && h->has_state) {
    // back to the fixed step of emppp_create
    CU(cudaMemcpyAsync(reinterpret_cast<char*>(h->ds.state) + offsetof(StepState, dt), &h->dt, sizeof(double),
                       cudaMemcpyHostToDevice, h->stream));
    CU(launch_reset_scale(h->ds, h->stream));  // the reported step size becomes the fixed one
    h->launches += 1;
    CU(cudaStreamSynchronize(h->stream));
  }
  invalidate_graph(h);
  return update_schedule(h);
}

EMPPP_API emppp_status emppp_set_energy_monitor(emppp_handle h, const emppp_energy_monitor* cfg) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  EnergyParams ep{0, 1, 0.0};
  if (cfg && cfg->enable) {
    if (!(cfg->eps_E > 0.0 && cfg->eps_E < 1e300) || cfg->hold < 1)
      return fail(EMPPP_ERR_ARG, "energy monitor: need eps_E > 0 (finite) and hold >= 1");
    ep.on = 1;
    ep.hold = cfg->hold;
    ep.eps = cfg->eps_E;
  }
  h->energy = ep;
  invalidate_graph(h);
  if (ep.on && h->has_state) {
    // the record starts at the present state
    CU(launch_energy(h->ds, h->energy, h->d_mon, true, h->stream));
    h->launches += 1;
    CU(cudaStreamSynchronize(h->stream));
  }
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_get_energy(emppp_handle h, emppp_energy_state* out) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!out) return fail(EMPPP_ERR_ARG, "out is NULL");
  if (!h->energy.on || !h->has_state) return fail(EMPPP_ERR_STATE, "energy monitor off or no state");
  if ((st = read_err(h)) != EMPPP_OK) return st;
  std::vector<EnergyMon> m((size_t)h->nbunch);
  CU(cudaMemcpyAsync(m.data(), h->d_mon, sizeof(EnergyMon) * m.size(), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  for (int b = 0; b < h->nbunch; b++) {
    out[b].ebar = m[b].ebar;
    out[b].rate = m[b].rate;
    out[b].t_sw = m[b].t_sw;
    out[b].n_sw = m[b].n_sw;
    out[b].armed = m[b].armed;
    out[b].switched = m[b].switched;
  }
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_two_stage(emppp_handle h, const double* x0, const double* u0, const double* w0,
                                       int32_t is_device_ptr, const emppp_two_stage_config* cfg,
                                       emppp_two_stage_report* rep) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!cfg || !rep || !x0 || !u0) return fail(EMPPP_ERR_ARG, "x0, u0, cfg and rep must not be NULL");
  if (cfg->max_stage1_steps < 1 || cfg->check_every < 1 || cfg->steps2 < 0 || !(cfg->dt2 > 0.0) ||
      !(cfg->t_after >= 0.0 && cfg->t_after < 1e300))
    return fail(EMPPP_ERR_ARG,
                "two-stage: need max_stage1_steps >= 1, check_every >= 1, steps2 >= 0, dt2 > 0, t_after >= 0");
  memset(rep, 0, sizeof(*rep));
  emppp_energy_monitor mon;
  memset(&mon, 0, sizeof(mon));
  mon.enable = 1;
  mon.hold = cfg->hold;
  mon.eps_E = cfg->eps_E;
  if ((st = emppp_set_energy_monitor(h, &mon)) != EMPPP_OK) return st;
  // 1. full EM-PP from the initial state until every bunch has met the criterion (or the cap)
  if ((st = emppp_set_particles(h, x0, u0, w0, is_device_ptr)) != EMPPP_OK) return st;
  std::vector<emppp_energy_state> es((size_t)h->nbunch);
  int64_t done = 0;
  bool all = false;
  while (done < cfg->max_stage1_steps && !all) {
    const int64_t k = cfg->max_stage1_steps - done < cfg->check_every ? cfg->max_stage1_steps - done : cfg->check_every;
    if ((st = emppp_step(h, k, &cfg->bext1)) != EMPPP_OK) return st;
    done += k;
    if ((st = emppp_get_energy(h, es.data())) != EMPPP_OK) return st;
    all = true;
    for (int b = 0; b < h->nbunch; b++) all = all && es[b].switched;
  }
  int64_t n_th = 0;
  double t_th = 0.0;
  for (int b = 0; b < h->nbunch; b++) {
    if (es[b].switched && es[b].n_sw > n_th) {
      n_th = es[b].n_sw;
      t_th = es[b].t_sw;
    }
  }
  if (!all) {  // the cap ends the search
    n_th = done;
    if ((st = emppp_get_state(h, nullptr, nullptr, &t_th, nullptr, 0)) != EMPPP_OK) return st;
  }
  rep->switched = all ? 1 : 0;
  rep->n_th = n_th;
  rep->t_th = t_th;
  rep->stage1_steps_first_run = done;
  // 2. the re-run from the same initial state: full EM-PP through the threshold, then on to t_th + t_after
  if ((st = emppp_set_particles(h, x0, u0, w0, is_device_ptr)) != EMPPP_OK) return st;
  if ((st = emppp_step(h, n_th, &cfg->bext1)) != EMPPP_OK) return st;
  const double t_target = t_th + cfg->t_after;
  int64_t n_sw = n_th;
  double t_sw = t_th;
  while (t_sw < t_target) {  // one step at a time: with the adaptive step only the device knows dt
    if ((st = emppp_step(h, 1, &cfg->bext1)) != EMPPP_OK) return st;
    if ((st = emppp_get_state(h, nullptr, nullptr, &t_sw, &n_sw, 0)) != EMPPP_OK) return st;
  }
  rep->n_sw = n_sw;
  rep->t_sw = t_sw;
  // 3. stage 2: pair fields off, background field only, larger step
  if (cfg->do_handoff && (st = emppp_handoff(h, cfg->center)) != EMPPP_OK) return st;
  if ((st = emppp_transport(h, cfg->steps2, cfg->dt2, &cfg->bext2)) != EMPPP_OK) return st;
  return emppp_synchronize(h);
}

EMPPP_API emppp_status emppp_set_options(emppp_handle h, const emppp_options* opt) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  if (!opt) return fail(EMPPP_ERR_ARG, "opt is NULL");
  if ((st = validate_options(opt)) != EMPPP_OK) return st;
  if (h->adapt.on && is_variant(*opt))
    return fail(EMPPP_ERR_STATE, "the midpoint reconstruction and the half-step field point run with a fixed dt");
  h->opt = *opt;
  if ((st = ensure_events(h)) != EMPPP_OK) return st;
  return update_schedule(h);
}

EMPPP_API emppp_status emppp_set_stream(emppp_handle h, void* cuda_stream) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  CU(cudaStreamSynchronize(h->stream));
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  invalidate_graph(h);
  return EMPPP_OK;
}

EMPPP_API emppp_status emppp_synchronize(emppp_handle h) {
  emppp_status st = check_handle(h);
  if (st != EMPPP_OK) return st;
  CU(cudaStreamSynchronize(h->stream));
  CU(cudaGetLastError());
  return read_err(h);
}

}  // extern "C"
