// Host runtime of polyrx: the C ABI of include/polyrx.h.
//
// A system owns its device buffers (layout in prx_internal.cuh), a private
// capture stream and three CUDA graphs built once per reaction scheme:
//   step   : one step kernel followed by an IF node whose body rebuilds the
//            cell list; the step kernel's last block sets the condition from
//            the device flag, so a rebuild runs exactly when some particle
//            left its extended cell, with no host round trip;
//   chunk  : Theta copies of `step` followed by the reaction kernels (or ten
//            steps when no reaction is set);
//   react  : the reaction kernels alone.
// prx_run replays `chunk` for whole reaction intervals and `step`/`react`
// for the remainder.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "prx_internal.cuh"

using namespace prx;

namespace {
constexpr double kDefaultSkin = 0.3;
constexpr uint32_t kHistCap = 8192;
constexpr uint64_t kCkptMagic = 0x31305850594C4F50ull;  // "POLYRX01"
constexpr int kNoRxChunk = 10;

struct ProfEvent {
  std::string name;
  cudaEvent_t a, b;
};
}  // namespace

struct prx_system {
  prx_system_desc d{};
  int has_rx = 0;
  prx_reaction_desc rxd{};  // reaction 0 of the scheme (its Theta is the scheme's)
  prx_reaction_desc rxs[PRX_MAX_REACTIONS]{};
  uint32_t nrx = 0;         // reactions in the scheme
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t cap = nullptr;
  Sys S{};
  Ctl* ctl_host = nullptr;  // pinned mirror for read-back
  struct ObsHost {          // pinned read-back of the observables
    double sums[4];         // kinetic energy / 2, momentum
    HistRec rec;            // populations
    Ctl ctl;                // step, bonds, status
  }* obs_host = nullptr;    // PRX_OBS_SLOTS pipelined slots + one for the synchronous call
  cudaEvent_t obs_ev[PRX_OBS_SLOTS] = {};
  bool obs_pending[PRX_OBS_SLOTS] = {};
  std::vector<void*> dev_allocs;
  std::vector<void*> grid_allocs;
  double grid_rcut = 0.0;
  double skin_used = 0.0;
  uint64_t host_step = 0;
  uint64_t step_launches = 0;      // step kernels (graphs and direct)
  uint64_t graph_rx_launches = 0;  // reaction sequences replayed inside graphs
  uint64_t other_launches = 0;     // other kernels launched directly (reaction, forces, observables)
  cudaGraphExec_t g_step = nullptr, g_chunk = nullptr, g_react = nullptr;
  cudaGraphExec_t g_chunk1 = nullptr;  // one interval, when g_chunk holds several
  uint32_t chunk_m = 1;                // reaction intervals per g_chunk replay
  // device graphs of device-driven runs (dg.cu): one step (+ k_dg_next), the
  // rebuild, the reaction; dg_ok when all three instantiated
  cudaGraphExec_t dg_step = nullptr, dg_rebuild = nullptr, dg_react = nullptr;
  bool dg_ok = false;
  bool graphs_valid = false;
  bool profiling = false;
  std::vector<ProfEvent> prof;
  std::string err;
  prx_batch* batch = nullptr;      // batch this system belongs to, if any
  cudaStream_t solo_stream = nullptr;  // the system's own stream while in a batch
  prx_batch* slot_batch = nullptr; // batch holding this system's admission slot
  int32_t slot = -1;               // its slot there (admitted until polled)
  cudaEvent_t join_ev = nullptr;   // orders the system's queued work before a batch's
};

// A batch: systems advanced together, one launch per kernel for all members.
struct prx_batch {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t cap = nullptr;
  std::vector<prx_system*> members;
  uint64_t theta = 0;  // reaction interval shared by the reacting members (0: none)
  uint64_t phase = 0;  // steps run mod theta
  uint64_t steps = 0, kernel_steps = 0, graph_launches = 0, rx_runs = 0;
  // device tables (valid while `valid`)
  BatchCtl* bctl = nullptr;
  BatchCtl* bctl_host = nullptr;
  Sys* T = nullptr;
  size_t T_cap = 0;
  BlkMap* maps = nullptr;    // the block maps, then as many entries for their compaction
  size_t maps_cap = 0;
  uint32_t* act_n = nullptr;  // compacted counts of the rebuild plan
  int n_step_variants = 0;     // step-kernel launches per batch step
  BatchLaunch L{};
  uint32_t n_active = 0;
  bool any_rx = false;
  cudaGraphExec_t g_step = nullptr, g_chunk = nullptr, g_react = nullptr;
  // device graphs of device-driven batch runs (dg.cu); dg_ok when all built
  cudaGraphExec_t dg_step = nullptr, dg_rebuild = nullptr, dg_react = nullptr;
  bool dg_ok = false;
  bool valid = false;
  std::string err;
  // admission (prx_batch_admit / step_epoch / poll)
  uint32_t max_slots = 0;     // 0: no limit
  uint64_t mem_budget = 0;    // 0: no limit
  uint64_t bytes_in_use = 0;  // estimates of the members and the unreported admitted systems
  uint64_t epochs = 0;
  struct Slot {
    prx_system* sys = nullptr;  // nullptr: free
    uint64_t left = 0;          // steps still to run (targeted members)
    uint64_t bytes = 0;
    bool targeted = false;      // admitted with a step target
    bool finishing = false;     // left the batch; done when `done` has completed
    cudaEvent_t done = nullptr;
  };
  std::vector<Slot> slots;
  std::vector<cudaEvent_t> inflight;  // ends of the epochs still queued (oldest first)
  std::vector<cudaEvent_t> ev_pool;   // spare epoch events
  // pinned staging of the member table and block maps (a ring, so that an
  // upload still queued is never overwritten)
  struct Stage {
    char* host = nullptr;
    size_t cap = 0;
    cudaEvent_t used = nullptr;  // recorded after the copies from this buffer
  } stage[4];
  int stage_next = 0;
};

namespace {

thread_local std::string g_create_error;

int fail(prx_system* s, int code, const std::string& msg) {
  if (s) s->err = msg;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(sys, PRX_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
  } while (0)

// The fixed per-system arrays, carved out of one device allocation (each
// part aligned to 256 bytes like a cudaMalloc of its own): creation and
// destruction then cost one allocation call each.
struct DevArena {
  struct Req {
    void** p;
    size_t bytes;
  };
  std::vector<Req> reqs;
  template <class T>
  void add(T** p, size_t count) {
    reqs.push_back(Req{(void**)p, sizeof(T) * (count ? count : 1)});
  }
  int commit(prx_system* sys, std::vector<void*>& list) {
    size_t total = 0;
    for (const Req& r : reqs) total += (r.bytes + 255) & ~(size_t)255;
    void* base = nullptr;
    if (cudaMalloc(&base, total) != cudaSuccess) {
      cudaGetLastError();
      return fail(sys, PRX_ENOMEM, "cudaMalloc of " + std::to_string(total) + " bytes failed");
    }
    list.push_back(base);
    char* c = (char*)base;
    for (const Req& r : reqs) {
      *r.p = c;
      c += (r.bytes + 255) & ~(size_t)255;
    }
    return PRX_OK;
  }
};

double wca_rc(const prx_system_desc& d) { return std::pow(2.0, 1.0 / 6.0) * d.wca_sigma; }

int validate_desc(prx_system* sys, const prx_system_desc* d) {
  if (!d) return fail(sys, PRX_EINVAL, "descriptor is NULL");
  if (d->adj_cap < 1 || d->adj_cap > PRX_MAX_ADJ) return fail(sys, PRX_EINVAL, "adj_cap must be 1..8");
  for (int k = 0; k < 3; ++k)
    if (!(d->box[k] > 0.0 && d->box[k] < 1e8)) return fail(sys, PRX_EINVAL, "box edges must be in (0, 1e8)");
  if (!(d->dt > 0.0) || !(d->mass > 0.0) || !(d->kT >= 0.0) || !(d->gamma >= 0.0))
    return fail(sys, PRX_EINVAL, "dt, mass must be > 0; kT, gamma >= 0");
  if (!(d->wca_sigma > 0.0) || !(d->wca_eps >= 0.0) || !(d->fene_r0 > 0.0) || !(d->fene_k >= 0.0))
    return fail(sys, PRX_EINVAL, "bad potential parameters");
  if (!(d->force_cap >= 0.0)) return fail(sys, PRX_EINVAL, "force_cap must be >= 0");
  if (d->force_precision != PRX_FORCE_FP32 && d->force_precision != PRX_FORCE_FP64)
    return fail(sys, PRX_EINVAL, "unknown force precision");
  if (d->reserved != 0) return fail(sys, PRX_EINVAL, "reserved field must be 0");
  if (d->n > 0x7FFFFFF0u) return fail(sys, PRX_EINVAL, "too many particles");
  return PRX_OK;
}

int validate_rx(prx_system* sys, const prx_reaction_desc* r) {
  if (r->a_lo > r->a_hi || r->t_lo > r->t_hi) return fail(sys, PRX_EINVAL, "empty state window");
  if (r->theta < 1 || !(r->k >= 0.0) || !(r->r_react > 0.0))
    return fail(sys, PRX_EINVAL, "theta >= 1, k >= 0, r_react > 0 required");
  if (r->bond_style != PRX_BOND_FENE && r->bond_style != PRX_BOND_MIRROR_LJ)
    return fail(sys, PRX_EINVAL, "unknown bond style");
  if (r->selection != PRX_SELECT_RANDOM && r->selection != PRX_SELECT_NEAREST)
    return fail(sys, PRX_EINVAL, "unknown selection rule");
  if ((r->type_mask_A | r->type_mask_T) >> PRX_MAX_TYPES) return fail(sys, PRX_EINVAL, "type mask beyond 8 types");
  if ((r->type_mask_A & r->type_mask_T) && !(r->a_hi < r->t_lo || r->t_hi < r->a_lo))
    return fail(sys, PRX_EINVAL, "A and T state windows overlap for a type in both masks");
  return PRX_OK;
}

// A set of concurrent reactions: each valid alone, one Theta, the random
// selection rule when there are several, and no (type, state) that is an A
// of one reaction and a T of another.
int validate_rxs(prx_system* sys, const prx_reaction_desc* r, uint32_t n) {
  if (n < 1 || n > PRX_MAX_REACTIONS) return fail(sys, PRX_EINVAL, "1 to 4 reactions");
  for (uint32_t q = 0; q < n; ++q) {
    int rc = validate_rx(sys, &r[q]);
    if (rc) return rc;
    if (r[q].theta != r[0].theta) return fail(sys, PRX_EINVAL, "concurrent reactions need one Theta");
    if (n > 1 && r[q].selection != PRX_SELECT_RANDOM)
      return fail(sys, PRX_EINVAL, "concurrent reactions use the random selection rule");
  }
  for (uint32_t q = 0; q < n; ++q)
    for (uint32_t w = 0; w < n; ++w)
      if ((r[q].type_mask_A & r[w].type_mask_T) && !(r[q].a_hi < r[w].t_lo || r[w].t_hi < r[q].a_lo))
        return fail(sys, PRX_EINVAL, "a (type, state) is an A of one reaction and a T of another");
  return PRX_OK;
}

double max_r_react(const prx_system* sys) {
  double r = 0.0;
  for (uint32_t q = 0; q < sys->nrx; ++q) r = std::max(r, sys->rxs[q].r_react);
  return r;
}

void destroy_graphs(prx_system* s) {
  // a device-driven run in flight launches these graphs from the device:
  // it must have finished before they go
  if ((s->dg_step || s->dg_rebuild || s->dg_react) && s->stream) cudaStreamSynchronize(s->stream);
  if (s->g_step) cudaGraphExecDestroy(s->g_step);
  if (s->g_chunk) cudaGraphExecDestroy(s->g_chunk);
  if (s->g_chunk1) cudaGraphExecDestroy(s->g_chunk1);
  if (s->g_react) cudaGraphExecDestroy(s->g_react);
  s->g_step = s->g_chunk = s->g_chunk1 = s->g_react = nullptr;
  if (s->dg_step) cudaGraphExecDestroy(s->dg_step);
  if (s->dg_rebuild) cudaGraphExecDestroy(s->dg_rebuild);
  if (s->dg_react) cudaGraphExecDestroy(s->dg_react);
  s->dg_step = s->dg_rebuild = s->dg_react = nullptr;
  s->dg_ok = false;
  s->graphs_valid = false;
}

void free_list(std::vector<void*>& l) {
  for (void* p : l) cudaFree(p);
  l.clear();
}

// Grid, fixed-point constants and Verlet-list layout for list cutoff rc
// (the larger of the WCA and reaction cutoffs):
//   list radius r_v = rc + skin; cells of edge >= r_v (only used to build the
//   lists); a rebuild is triggered when some particle moved more than skin/2
//   since the last build; X = floor(x / L 2^32) mod 2^32 per axis.
int setup_grid(prx_system* sys, double rc) {
  Sys& S = sys->S;
  double skin = sys->d.skin < 0.0 ? kDefaultSkin : sys->d.skin;
  if (!(skin > 0.0)) return fail(sys, PRX_EINVAL, "skin must be positive");
  // small boxes: shrink the skin until three list radii fit along every edge
  const double Lmin = std::min(sys->d.box[0], std::min(sys->d.box[1], sys->d.box[2]));
  if (Lmin / (rc + skin) < 3.0 * (1.0 + 1e-9)) skin = Lmin / (3.0 * (1.0 + 2e-9)) - rc;
  if (!(skin >= 0.02)) return fail(sys, PRX_EINVAL, "box edge below three interaction cutoffs plus skin");
  sys->skin_used = skin;
  const double rv = rc + skin;
  long long ncell = 1;
  for (int k = 0; k < 3; ++k) {
    const double L = sys->d.box[k];
    int nc = (int)std::floor(L / (rv * (1.0 + 1e-9)));
    if (nc < 3) return fail(sys, PRX_EINVAL, "box edge below three list radii (cutoff + skin)");
    if (nc > 1023) nc = 1023;
    S.nc[k] = nc;
    S.Lfx[k] = (long long)std::llround(L * 4294967296.0);
    S.M64[k] = (unsigned long long)(std::ldexp((long double)1.0, 64) / (long double)L + 0.5L);
    S.scale[k] = (float)(L / 4294967296.0);
    int sh = 0;
    while (sh < 22 && std::ldexp(1.0, sh + 9) * (L / 4294967296.0) < skin) ++sh;
    S.wshift[k] = sh;
    S.wunit[k] = (float)(std::ldexp(1.0, sh) * (L / 4294967296.0));
    ncell *= nc;
  }
  S.cubic = S.scale[0] == S.scale[1] && S.scale[1] == S.scale[2] ? 1 : 0;
  S.s2f = S.scale[0] * S.scale[0];
  S.rc2u = (float)(S.rc2 / ((double)S.scale[0] * (double)S.scale[0]));
  const double wmax = std::max((double)S.wunit[0], std::max((double)S.wunit[1], (double)S.wunit[2]));
  const double dmax = 0.5 * skin - 2.0 * std::sqrt(3.0) * wmax - 1e-6;
  if (!(dmax > 0.0)) return fail(sys, PRX_EINVAL, "skin too small for the displacement trigger");
  S.disp2_max = (float)(dmax * dmax);
  // the list build compares FP32 tile-frame coordinates (~2e-7 L of rounding
  // per coordinate): its radius is widened by more than that error
  {
    const double Lmax = std::max(sys->d.box[0], std::max(sys->d.box[1], sys->d.box[2]));
    const double rvb = rv * (1.0 + 1e-5) + 1e-6 * Lmax;
    S.rv2_build = (float)(rvb * rvb);
  }
  S.ncell = (int)ncell;
  sys->grid_rcut = rc;
  free_list(sys->grid_allocs);
  int rc2;
  DevArena A;
  A.add(&S.cell_start, (size_t)ncell + 1), A.add(&S.count, (size_t)ncell), A.add(&S.fill, (size_t)ncell);
  const size_t nblk = std::max<size_t>((S.n + RX_THREADS - 1) / RX_THREADS,
                                       ((size_t)ncell + SCAN_TILE - 1) / SCAN_TILE) + 1;
  A.add(&S.blk_count, nblk), A.add(&S.blk_off, nblk);
  // Verlet list: capacity from the mean count at this density; entries are
  // the neighbours' slots, 16-bit up to 65,535 particles
  const double V = sys->d.box[0] * sys->d.box[1] * sys->d.box[2];
  const double rho = (double)S.n / V;
  const double mean_nb = rho * 4.0 / 3.0 * M_PI * rv * rv * rv;
  // (a multiple of 4: the build pads each list to whole stages of four)
  S.list_cap = (std::max(32, std::min(252, (int)std::ceil(2.5 * mean_nb + 16.0))) + 3) & ~3;
  S.nl16 = S.n <= 65535 ? 1 : 0;
  A.add((uint8_t**)&S.nl, (size_t)S.list_cap * S.n * (S.nl16 ? 2 : 4));
  A.add(&S.nn, (size_t)S.n);
  if ((rc2 = A.commit(sys, sys->grid_allocs))) return rc2;
  {
    // list-build tiling: the largest tile of 1..4 cell rows whose particles
    // fit about two passes of 256 threads (fewer restaged neighbour rows per
    // particle); staging buffer sized for all neighbour rows at once
    const double per_row = (double)S.n / ((double)S.nc[1] * S.nc[2]);
    const double per_cell = (double)S.n / (double)ncell;
    int ty = 1;
    for (int c = 2; c <= 4; ++c)
      if (c * per_row + 3.0 * std::sqrt(c * per_row) + 16.0 <= 640.0) ty = c;
    ty = std::max(1, std::min(ty, S.nc[1]));
    S.tile_y = ty;
    S.tiles_y = (S.nc[1] + ty - 1) / ty;
    const double mean_tile = ty * per_row;
    int t = (int)std::ceil((mean_tile + 3.0 * std::sqrt(mean_tile) + 16.0) / 32.0) * 32;
    S.tile_threads = std::max(64, std::min(256, t));
    const double mean_tot = 3.0 * (ty + 2) * (per_row + 2.0 * per_cell);
    int cap = (int)std::ceil((mean_tot + 4.0 * std::sqrt(mean_tot) + 64.0) / 32.0) * 32;
    S.tile_cap = 0;
    const size_t fixed = build_tile_smem(S);
    const size_t budget = 160 * 1024;
    if (fixed + 16 * (size_t)cap > budget) cap = (int)((budget - fixed) / 16);
    S.tile_cap = std::max(64, std::min(cap, 65535));
    if (configure_build_kernel(build_tile_smem(S)))
      return fail(sys, PRX_ECUDA, "cannot set the list-build kernel's shared-memory size");
  }
  return PRX_OK;
}

int read_ctl(prx_system* sys) {
  CK(cudaMemcpyAsync(sys->ctl_host, sys->S.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, sys->stream));
  CK(cudaStreamSynchronize(sys->stream));
  return PRX_OK;
}

int sync_status(prx_system* sys) {
  int rc = read_ctl(sys);
  if (rc) return rc;
  const int st = sys->ctl_host->status;
  if (st) return fail(sys, st, std::string("device reported ") + prx_status_string(st));
  return PRX_OK;
}

// Event hook used while profiling: records an event before and after each launch.
void prof_hook(void* ctx, const char* name, int phase) {
  prx_system* s = (prx_system*)ctx;
  if (phase == 0) {
    ProfEvent e;
    e.name = name;
    cudaEventCreate(&e.a);
    cudaEventCreate(&e.b);
    cudaEventRecord(e.a, s->stream);
    s->prof.push_back(e);
  } else {
    cudaEventRecord(s->prof.back().b, s->stream);
  }
}

int full_rebin(prx_system* sys, int mode) {
  launch_rebin(sys->S, sys->stream, mode, nullptr, nullptr);
  CK(cudaGetLastError());
  return PRX_OK;
}

#define CE(call)                       \
  do {                                 \
    cudaError_t e_ = (call);           \
    if (e_ != cudaSuccess) return e_;  \
  } while (0)

// Captures `nsteps` x (step, IF(rebuild)) followed optionally by the
// reaction kernels into one executable graph.  `step(h)` launches the step
// kernel(s) that set the conditional handle h; `rebuild()` and `rx()` the
// rebuild and reaction sequences; all on the capture stream.
// With reps > 1 the (steps, reaction) sequence is captured reps times.
template <class StepF, class RebuildF, class RxF>
cudaError_t capture_graph(cudaStream_t cap, int nsteps, bool with_rx, StepF step, RebuildF rebuild,
                          RxF rx, cudaGraphExec_t* out, int reps = 1) {
  cudaGraph_t g;
  CE(cudaGraphCreate(&g, 0));
  std::vector<cudaGraph_t> bodies;
  CE(cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  for (int rep = 0; rep < reps; ++rep) {
  for (int s = 0; s < nsteps; ++s) {
    cudaGraphConditionalHandle h;
    CE(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    step(h);
    cudaStreamCaptureStatus cs;
    cudaGraph_t gcap;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    CE(cudaStreamGetCaptureInfo(cap, &cs, nullptr, &gcap, &deps, nullptr, &ndeps));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t cn;
    CE(cudaGraphAddNode(&cn, gcap, deps, nullptr, ndeps, &np));
    bodies.push_back(np.conditional.phGraph_out[0]);
    CE(cudaStreamUpdateCaptureDependencies(cap, &cn, nullptr, 1, cudaStreamSetCaptureDependencies));
  }
  if (with_rx) rx();
  }
  CE(cudaStreamEndCapture(cap, &g));
  for (cudaGraph_t body : bodies) {
    CE(cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    rebuild();
    cudaGraph_t tmp;
    CE(cudaStreamEndCapture(cap, &tmp));
  }
  CE(cudaGraphInstantiate(out, g, 0));
  CE(cudaGraphDestroy(g));
  return cudaSuccess;
}

int build_graph(prx_system* sys, int nsteps, bool with_rx, cudaGraphExec_t* out, int reps = 1) {
  const bool fp64 = sys->d.force_precision == PRX_FORCE_FP64;
  CK(capture_graph(
      sys->cap, nsteps, with_rx,
      [&](cudaGraphConditionalHandle h) { launch_step(sys->S, sys->cap, fp64, 0, h, 1); },
      [&] { launch_rebin(sys->S, sys->cap, 0, nullptr, nullptr); },
      [&] { launch_rx(sys->S, sys->cap, -1, nullptr, nullptr); }, out, reps));
  return PRX_OK;
}

// One device-launchable graph of whatever `body()` launches on the capture
// stream, uploaded to the device.
template <class F>
cudaError_t capture_device_graph(cudaStream_t cap, F body, cudaGraphExec_t* out) {
  cudaGraph_t g;
  CE(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  body();
  CE(cudaStreamEndCapture(cap, &g));
  const cudaError_t e = cudaGraphInstantiateWithFlags(out, g, cudaGraphInstantiateFlagDeviceLaunch);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return e;
  }
  return cudaGraphUpload(*out, cap);
}

// The device graphs of device-driven runs; on any failure the system keeps
// the host-replayed graphs (the same kernels).
void build_device_graphs(prx_system* sys) {
  const bool fp64 = sys->d.force_precision == PRX_FORCE_FP64;
  const unsigned theta = sys->has_rx ? (unsigned)sys->rxd.theta : 1u;
  cudaError_t e = capture_device_graph(sys->cap, [&] {
    launch_step(sys->S, sys->cap, fp64, 0, 0, 0);
    launch_dg_next(sys->S, sys->cap, theta);
  }, &sys->dg_step);
  if (e == cudaSuccess)
    e = capture_device_graph(sys->cap, [&] { launch_rebin(sys->S, sys->cap, 0, nullptr, nullptr); },
                             &sys->dg_rebuild);
  if (e == cudaSuccess && sys->has_rx)
    e = capture_device_graph(sys->cap, [&] { launch_rx(sys->S, sys->cap, -1, nullptr, nullptr); },
                             &sys->dg_react);
  if (e == cudaSuccess) e = cudaStreamSynchronize(sys->cap);
  sys->dg_ok = e == cudaSuccess;
  if (!sys->dg_ok) {
    cudaGetLastError();
    if (sys->dg_step) cudaGraphExecDestroy(sys->dg_step);
    if (sys->dg_rebuild) cudaGraphExecDestroy(sys->dg_rebuild);
    if (sys->dg_react) cudaGraphExecDestroy(sys->dg_react);
    sys->dg_step = sys->dg_rebuild = sys->dg_react = nullptr;
  }
}

int ensure_graphs(prx_system* sys) {
  if (sys->graphs_valid) return PRX_OK;
  destroy_graphs(sys);
  build_device_graphs(sys);
  if (sys->dg_ok) {
    sys->graphs_valid = true;
    return PRX_OK;
  }
  int rc;
  if ((rc = build_graph(sys, 1, false, &sys->g_step))) return rc;
  const int m = (int)sys->chunk_m;
  if (sys->has_rx) {
    if ((rc = build_graph(sys, (int)sys->rxd.theta, true, &sys->g_chunk, m))) return rc;
    if (m > 1 && (rc = build_graph(sys, (int)sys->rxd.theta, true, &sys->g_chunk1))) return rc;
    if ((rc = build_graph(sys, 0, true, &sys->g_react))) return rc;
  } else {
    if ((rc = build_graph(sys, kNoRxChunk, false, &sys->g_chunk, m))) return rc;
    if (m > 1 && (rc = build_graph(sys, kNoRxChunk, false, &sys->g_chunk1))) return rc;
  }
  sys->graphs_valid = true;
  return PRX_OK;
}

// One step launched directly (profiling): the flag is read back after the
// step to decide on the rebuild.
int direct_step(prx_system* sys) {
  prof_hook(sys, "step", 0);
  launch_step(sys->S, sys->stream, sys->d.force_precision == PRX_FORCE_FP64, 0, 0, 0);
  prof_hook(sys, "step", 1);
  sys->step_launches++;
  CK(cudaGetLastError());
  int rc = read_ctl(sys);
  if (rc) return rc;
  if (sys->ctl_host->rebin_flag) launch_rebin(sys->S, sys->stream, 0, prof_hook, sys);
  sys->host_step++;
  if (sys->has_rx && sys->host_step % sys->rxd.theta == 0) {
    launch_rx(sys->S, sys->stream, -1, prof_hook, sys);
    sys->other_launches += rx_kernel_count(sys->S.R.rule);
  }
  CK(cudaGetLastError());
  return PRX_OK;
}

// Host copies of the current per-slot arrays.
struct HostSlots {
  std::vector<double> x, y, z, vx, vy, vz;
  std::vector<uint32_t> id, adj;
  std::vector<uint8_t> type, nadj;
  std::vector<int8_t> state;
  std::vector<uint4> P;
};

// What fetch_slots copies besides the ids (bit mask).
enum : unsigned { FS_POS = 1u, FS_VEL = 2u, FS_TYPE = 4u, FS_STATE = 8u, FS_TOPO = 16u };

int fetch_slots(prx_system* sys, HostSlots& h, unsigned what) {
  const bool pos = what & FS_POS, vel = what & FS_VEL, topo = what & FS_TOPO;
  int rc = read_ctl(sys);
  if (rc) return rc;
  const size_t n = sys->S.n;
  const SoA& B = sys->ctl_host->set ? sys->S.s1 : sys->S.s0;
  h.id.resize(n);
  if (n) CK(cudaMemcpyAsync(h.id.data(), B.id, 4 * n, cudaMemcpyDeviceToHost, sys->stream));
  if (pos && n) {
    h.x.resize(n); h.y.resize(n); h.z.resize(n);
    CK(cudaMemcpyAsync(h.x.data(), B.x, 8 * n, cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaMemcpyAsync(h.y.data(), B.y, 8 * n, cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaMemcpyAsync(h.z.data(), B.z, 8 * n, cudaMemcpyDeviceToHost, sys->stream));
  }
  if (vel && n) {
    h.vx.resize(n); h.vy.resize(n); h.vz.resize(n);
    CK(cudaMemcpyAsync(h.vx.data(), B.vx, 8 * n, cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaMemcpyAsync(h.vy.data(), B.vy, 8 * n, cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaMemcpyAsync(h.vz.data(), B.vz, 8 * n, cudaMemcpyDeviceToHost, sys->stream));
  }
  if ((what & FS_TYPE) && n) {
    h.type.resize(n);
    CK(cudaMemcpyAsync(h.type.data(), B.type, n, cudaMemcpyDeviceToHost, sys->stream));
  }
  if ((what & FS_STATE) && n) {
    h.state.resize(n);
    CK(cudaMemcpyAsync(h.state.data(), B.state, n, cudaMemcpyDeviceToHost, sys->stream));
  }
  if (topo && n) {
    h.nadj.resize(n); h.adj.resize(n * sys->S.cap);
    h.P.resize(n);
    const uint4* Pd = sys->ctl_host->phase ? sys->S.P1 : sys->S.P0;
    CK(cudaMemcpyAsync(h.nadj.data(), B.nadj, n, cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaMemcpyAsync(h.adj.data(), B.adj, 4 * n * sys->S.cap, cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaMemcpyAsync(h.P.data(), Pd, sizeof(uint4) * n, cudaMemcpyDeviceToHost, sys->stream));
  }
  CK(cudaStreamSynchronize(sys->stream));
  return PRX_OK;
}

double wrap_host(double v, double L) {
  if (v >= L) v -= L;
  if (v < 0.0) v += L;
  return v;
}

// Creates the device system from per-slot arrays.  `cells` (optional) gives
// each slot's cell; without it the slots are binned from their positions.
int create_impl(const prx_system_desc* desc, const double* pos, const double* vel,
                const uint8_t* type, const int8_t* state, const prx_bond* bonds, uint64_t n_bonds,
                void* stream, const uint32_t* slot_ids, const uint32_t* slot_cells,
                const uint32_t* slot_adj_ids, const uint8_t* slot_nadj, uint64_t step0,
                double grid_rc, const uint32_t* slot_w, const uint8_t* slot_nn,
                const int32_t* slot_nl, int nl_cap_saved, prx_system** out) {
  prx_system* sys = nullptr;
  if (!out) return PRX_EINVAL;
  *out = nullptr;
  sys = new (std::nothrow) prx_system();
  if (!sys) return PRX_ENOMEM;
  auto bail = [&](int rc) {
    if (rc) {
      g_create_error = sys->err;
      prx_destroy(sys);
    }
    return rc;
  };
  int rc = validate_desc(sys, desc);
  if (rc) return bail(rc);
  const uint32_t n = desc->n;
  if (n && (!pos || !type || !state)) return bail(fail(sys, PRX_EINVAL, "pos, type and state are required"));
  if (n_bonds && !bonds) return bail(fail(sys, PRX_EINVAL, "bonds is NULL"));
  sys->d = *desc;
  Sys& S = sys->S;
  S.n = n;
  S.cap = desc->adj_cap;
  for (int k = 0; k < 3; ++k) {
    S.L[k] = desc->box[k];
    S.halfL[k] = 0.5 * desc->box[k];
  }
  const double rc_w = wca_rc(*desc);
  S.rc = rc_w;
  S.rc2 = rc_w * rc_w;
  S.rcf = (float)rc_w;
  S.rc2f = (float)S.rc2;
  S.sig = desc->wca_sigma;
  S.sigf = (float)S.sig;
  S.sig2 = desc->wca_sigma * desc->wca_sigma;
  S.sig2f = (float)S.sig2;
  S.eps24 = 24.0 * desc->wca_eps;
  S.eps24f = (float)S.eps24;
  S.eps4 = 4.0 * desc->wca_eps;
  S.eps4f = (float)S.eps4;
  S.fcap = desc->force_cap;
  S.fcapf = (float)desc->force_cap;
  S.fk = desc->fene_k;
  S.fkf = (float)desc->fene_k;
  S.fr02 = desc->fene_r0 * desc->fene_r0;
  S.fr02f = (float)S.fr02;
  S.fr02if = (float)(1.0 / S.fr02);
  S.dt = desc->dt;
  S.mass = desc->mass;
  S.b_kick = desc->dt / desc->mass;
  S.b_kickf = (float)S.b_kick;
  S.gm = desc->gamma * desc->mass;
  S.a_fric = 1.0 - S.b_kick * S.gm;
  S.cR = std::sqrt(24.0 * desc->gamma * desc->kT * desc->mass / desc->dt);
  S.cRf = (float)S.cR;
  S.thermo = desc->gamma > 0.0 ? 1 : 0;
  S.seed = desc->seed;
  S.hist_cap = kHistCap;
  S.step_bt = 256;
  S.step_bpsm = 0;
  S.step_lanes = 1;
  S.bond_cap = std::max<unsigned long long>(1ull, ((unsigned long long)n * S.cap) / 2ull);

  if (stream) {
    sys->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&sys->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(sys, PRX_ECUDA, "stream creation failed"));
    sys->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&sys->cap, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(sys, PRX_ECUDA, "capture stream creation failed"));
  if (cudaMallocHost(&sys->ctl_host, sizeof(Ctl)) != cudaSuccess)
    return bail(fail(sys, PRX_ENOMEM, "pinned control block"));
  if (cudaMallocHost(&sys->obs_host, sizeof(*sys->obs_host) * (PRX_OBS_SLOTS + 1)) != cudaSuccess)
    return bail(fail(sys, PRX_ENOMEM, "pinned observables block"));
  memset(sys->ctl_host, 0, sizeof(Ctl));

  DevArena A;
  SoA* sets[2] = {&S.s0, &S.s1};
  for (SoA* B : sets) {
    A.add(&B->x, n), A.add(&B->y, n), A.add(&B->z, n);
    A.add(&B->vx, n), A.add(&B->vy, n), A.add(&B->vz, n);
    A.add(&B->id, n), A.add(&B->type, n), A.add(&B->state, n), A.add(&B->nadj, n);
    A.add(&B->adj, (size_t)n * S.cap);
  }
  A.add(&S.P0, n), A.add(&S.P1, n), A.add(&S.key, n), A.add(&S.tmp, n), A.add(&S.new_of_old, n);
  A.add(&S.win, n), A.add(&S.wch, n), A.add(&S.bonds, (size_t)S.bond_cap);
  A.add(&S.hist, (size_t)S.hist_cap + 2), A.add(&S.ctl, 1);
  A.add(&S.pop, (size_t)POP_REPLICAS * PRX_MAX_TYPES * PRX_MAX_STATES);
  A.add(&S.red, 4 * ((size_t)(n + RX_THREADS - 1) / RX_THREADS + 1));
  A.add(&S.fout, 3 * (size_t)n), A.add(&S.eout, (size_t)n);
  if ((rc = A.commit(sys, sys->dev_allocs))) return bail(rc);
  if ((rc = setup_grid(sys, grid_rc > rc_w ? grid_rc : rc_w))) return bail(rc);

  const SoA& B = S.s0;
  auto up = [&](void* dst, const void* src, size_t bytes) -> int {
    if (!bytes) return PRX_OK;
    if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, sys->stream) != cudaSuccess)
      return fail(sys, PRX_ECUDA, "upload failed");
    return PRX_OK;
  };
  // a plain creation (particle p in slot p) stages positions, velocities and
  // ids on the device; a restore (saved slot order) goes through the host
  const bool plain = !slot_ids && !slot_cells && !slot_adj_ids;
  if (plain) {
    std::vector<uint8_t> hn;
    std::vector<uint32_t> hadj;
    if (n_bonds) {
      hn.assign(n, 0);
      hadj.assign((size_t)n * S.cap, 0u);
      for (uint64_t b = 0; b < n_bonds; ++b) {
        const prx_bond& bd = bonds[b];
        if (bd.a >= n || bd.t >= n || bd.a == bd.t || bd.style > 1u)
          return bail(fail(sys, PRX_EINVAL, "bad initial bond"));
        if (hn[bd.a] >= S.cap || hn[bd.t] >= S.cap)
          return bail(fail(sys, PRX_ECAPACITY, "initial bonds exceed adj_cap"));
        hadj[(size_t)bd.a * S.cap + hn[bd.a]++] = bd.t | (bd.style << 31);
        hadj[(size_t)bd.t * S.cap + hn[bd.t]++] = bd.a | (bd.style << 31);
      }
    }
    if (n_bonds > S.bond_cap) return bail(fail(sys, PRX_ECAPACITY, "more bonds than the bond list holds"));
    Ctl z;
    memset(&z, 0, sizeof(z));
    if ((rc = up(S.ctl, &z, sizeof(Ctl))) || (rc = up(B.type, type, n)) || (rc = up(B.state, state, n)))
      return bail(rc);
    if ((rc = up(S.fout, pos, 24ull * n))) return bail(rc);
    launch_stage_input(S, sys->stream, S.fout, 0);
    if (vel) {
      if ((rc = up(S.fout, vel, 24ull * n))) return bail(rc);
      launch_stage_input(S, sys->stream, S.fout, 1);
    } else if (n && (cudaMemsetAsync(B.vx, 0, 8ull * n, sys->stream) != cudaSuccess ||
                     cudaMemsetAsync(B.vy, 0, 8ull * n, sys->stream) != cudaSuccess ||
                     cudaMemsetAsync(B.vz, 0, 8ull * n, sys->stream) != cudaSuccess)) {
      return bail(fail(sys, PRX_ECUDA, "memset failed"));
    }
    if (n_bonds) {
      if ((rc = up(B.nadj, hn.data(), n)) || (rc = up(B.adj, hadj.data(), 4ull * n * S.cap))) return bail(rc);
    } else if (n && (cudaMemsetAsync(B.nadj, 0, n, sys->stream) != cudaSuccess ||
                     cudaMemsetAsync(B.adj, 0, 4ull * n * S.cap, sys->stream) != cudaSuccess)) {
      return bail(fail(sys, PRX_ECUDA, "memset failed"));
    }
    if (cudaGetLastError() != cudaSuccess) return bail(fail(sys, PRX_ECUDA, "input staging launch failed"));
    if ((rc = read_ctl(sys))) return bail(rc);
    switch (sys->ctl_host->input_err) {
      case 0: break;
      case 1: return bail(fail(sys, PRX_EINVAL, "non-finite position"));
      case 2: return bail(fail(sys, PRX_EINVAL, "position more than one box edge outside the box"));
      default: return bail(fail(sys, PRX_EINVAL, "type >= 8"));
    }
  } else {
    // host staging in slot order
    std::vector<uint32_t> ids(n);
    for (uint32_t s = 0; s < n; ++s) ids[s] = slot_ids ? slot_ids[s] : s;
    std::vector<uint32_t> slot_of(n, 0xFFFFFFFFu);
    for (uint32_t s = 0; s < n; ++s) {
      if (ids[s] >= n || slot_of[ids[s]] != 0xFFFFFFFFu) return bail(fail(sys, PRX_EINVAL, "bad slot order"));
      slot_of[ids[s]] = s;
    }
    std::vector<double> hx(n), hy(n), hz(n), hvx(n, 0.0), hvy(n, 0.0), hvz(n, 0.0);
    std::vector<uint8_t> ht(n), hn(n, 0);
    std::vector<int8_t> hs(n);
    std::vector<uint32_t> hadj((size_t)n * S.cap, 0u);
    for (uint32_t s = 0; s < n; ++s) {
      const uint32_t p = ids[s];
      double c[3];
      for (int k = 0; k < 3; ++k) {
        const double v = pos[3 * (size_t)p + k];
        if (!std::isfinite(v)) return bail(fail(sys, PRX_EINVAL, "non-finite position"));
        c[k] = slot_cells ? v : wrap_host(v, desc->box[k]);
        if (!slot_cells && !(c[k] >= 0.0 && c[k] < desc->box[k]))
          return bail(fail(sys, PRX_EINVAL, "position more than one box edge outside the box"));
      }
      hx[s] = c[0];
      hy[s] = c[1];
      hz[s] = c[2];
      if (vel) {
        hvx[s] = vel[3 * (size_t)p];
        hvy[s] = vel[3 * (size_t)p + 1];
        hvz[s] = vel[3 * (size_t)p + 2];
      }
      if (type[p] >= PRX_MAX_TYPES) return bail(fail(sys, PRX_EINVAL, "type >= 8"));
      ht[s] = type[p];
      hs[s] = state[p];
    }
    if (slot_adj_ids) {
      for (uint32_t s = 0; s < n; ++s) {
        if (slot_nadj[s] > S.cap) return bail(fail(sys, PRX_ECAPACITY, "adjacency row beyond capacity"));
        hn[s] = slot_nadj[s];
        for (uint32_t b = 0; b < slot_nadj[s]; ++b) {
          const uint32_t e = slot_adj_ids[(size_t)s * S.cap + b];
          if ((e & SLOT_MASK) >= n) return bail(fail(sys, PRX_EINVAL, "bad adjacency entry"));
          hadj[(size_t)s * S.cap + b] = slot_of[e & SLOT_MASK] | (e & ~SLOT_MASK);
        }
      }
    } else {
      for (uint64_t b = 0; b < n_bonds; ++b) {
        const prx_bond& bd = bonds[b];
        if (bd.a >= n || bd.t >= n || bd.a == bd.t || bd.style > 1u)
          return bail(fail(sys, PRX_EINVAL, "bad initial bond"));
        const uint32_t pa = slot_of[bd.a], pt = slot_of[bd.t];
        if (hn[pa] >= S.cap || hn[pt] >= S.cap) return bail(fail(sys, PRX_ECAPACITY, "initial bonds exceed adj_cap"));
        hadj[(size_t)pa * S.cap + hn[pa]++] = pt | (bd.style << 31);
        hadj[(size_t)pt * S.cap + hn[pt]++] = pa | (bd.style << 31);
      }
    }
    if (n_bonds > S.bond_cap) return bail(fail(sys, PRX_ECAPACITY, "more bonds than the bond list holds"));

    if ((rc = up(B.x, hx.data(), 8ull * n)) || (rc = up(B.y, hy.data(), 8ull * n)) || (rc = up(B.z, hz.data(), 8ull * n)) ||
        (rc = up(B.vx, hvx.data(), 8ull * n)) || (rc = up(B.vy, hvy.data(), 8ull * n)) ||
        (rc = up(B.vz, hvz.data(), 8ull * n)) || (rc = up(B.id, ids.data(), 4ull * n)) ||
        (rc = up(B.type, ht.data(), n)) || (rc = up(B.state, hs.data(), n)) || (rc = up(B.nadj, hn.data(), n)) ||
        (rc = up(B.adj, hadj.data(), 4ull * n * S.cap)))
      return bail(rc);
  }
  if (n_bonds) {
    if ((rc = up(S.bonds, bonds, sizeof(prx_bond) * n_bonds))) return bail(rc);
  }
  Ctl c0;
  memset(&c0, 0, sizeof(c0));
  c0.nbonds = n_bonds;
  c0.step = step0;
  if ((rc = up(S.ctl, &c0, sizeof(Ctl)))) return bail(rc);
  sys->host_step = step0;
  if (cudaMemsetAsync(S.hist, 0, sizeof(HistRec) * (S.hist_cap + 2), sys->stream) != cudaSuccess)
    return bail(fail(sys, PRX_ECUDA, "memset failed"));

  if (slot_cells) {
    // restore the saved cell of every slot: with the keys given, the counting
    // sort keeps the slot order because the saved order is sorted by cell
    for (uint32_t s = 0; s < n; ++s)
      if (slot_cells[s] >= (uint32_t)S.ncell || (s && slot_cells[s] < slot_cells[s - 1]))
        return bail(fail(sys, PRX_EINVAL, "checkpoint cells out of order"));
    if ((rc = up(S.key, slot_cells, 4ull * n))) return bail(rc);
  }
  // bin into set 1 (full keys from positions, or the restored cells)
  if ((rc = full_rebin(sys, slot_cells ? 2 : 1))) return bail(rc);
  launch_pop_init(S, sys->stream);  // the running populations of the reaction records
  if ((rc = sync_status(sys))) return bail(rc);
  if (slot_cells && slot_w && slot_nn && slot_nl) {
    // a checkpoint also restores the displacement references and the exact
    // Verlet lists, so the rebuilds happen at the same steps as before
    if (nl_cap_saved != S.list_cap) return bail(fail(sys, PRX_EIO, "checkpoint list capacity differs"));
    std::vector<uint4> Ph(n);
    uint4* Pd = sys->ctl_host->phase ? S.P1 : S.P0;
    if (n) {
      if (cudaMemcpy(Ph.data(), Pd, sizeof(uint4) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return bail(fail(sys, PRX_ECUDA, "download failed"));
      for (uint32_t q = 0; q < n; ++q) Ph[q].w = slot_w[q];
      if ((rc = up(Pd, Ph.data(), sizeof(uint4) * n))) return bail(rc);
      if ((rc = up(S.nn, slot_nn, n))) return bail(rc);
      const size_t ne = (size_t)S.list_cap * n;
      if (S.nl16) {
        std::vector<uint16_t> v(ne);
        for (size_t q = 0; q < ne; ++q) v[q] = (uint16_t)slot_nl[q];
        if ((rc = up(S.nl, v.data(), 2 * ne))) return bail(rc);
      } else {
        if ((rc = up(S.nl, slot_nl, 4 * ne))) return bail(rc);
      }
    }
    if ((rc = sync_status(sys))) return bail(rc);
  }
  *out = sys;
  return PRX_OK;
}

int bfail(prx_batch* b, int code, const std::string& msg) {
  b->err = msg;
  return code;
}

#define CKB(call)                                                                      \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return bfail(b, PRX_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
  } while (0)

void batch_destroy_graphs(prx_batch* b) {
  // a device-driven run in flight launches its graphs from the device
  if ((b->dg_step || b->dg_rebuild || b->dg_react) && b->stream) cudaStreamSynchronize(b->stream);
  if (b->g_step) cudaGraphExecDestroy(b->g_step);
  if (b->g_chunk) cudaGraphExecDestroy(b->g_chunk);
  if (b->g_react) cudaGraphExecDestroy(b->g_react);
  b->g_step = b->g_chunk = b->g_react = nullptr;
  if (b->dg_step) cudaGraphExecDestroy(b->dg_step);
  if (b->dg_rebuild) cudaGraphExecDestroy(b->dg_rebuild);
  if (b->dg_react) cudaGraphExecDestroy(b->dg_react);
  b->dg_step = b->dg_rebuild = b->dg_react = nullptr;
  b->dg_ok = false;
}

// Member table, block maps and graphs of a batch after its membership
// changed.  Each active member (n > 0) gets a copy of its Sys marked as a
// batch member; every kernel family gets a block map listing, per block,
// the member and the block's index within that member's own grid (the grid
// the member would be launched with alone).
//
// Everything is ordered on the batch's stream, with no host wait: the tables
// are uploaded by copies queued behind the work already queued (pageable
// sources are staged by the copy call itself), grown tables are allocated and
// the old ones freed in stream order, and graph executables still running
// are released by CUDA when they complete.  The batch control block needs no
// reset: its member counter and rebuild flag return to zero at the end of
// every batch step, and its rebuild count is cumulative.
int batch_prepare(prx_batch* b) {
  if (b->valid) return PRX_OK;
  batch_destroy_graphs(b);
  std::vector<Sys> table;
  b->any_rx = false;
  for (prx_system* m : b->members) {
    if (!m->S.n) continue;
    table.push_back(m->S);
    b->any_rx = b->any_rx || m->has_rx;
  }
  b->n_active = (uint32_t)table.size();
  if (!b->n_active) {
    b->valid = true;
    return PRX_OK;
  }
  std::vector<BlkMap> part, cell, tile, one, build;
  auto add = [](std::vector<BlkMap>& v, uint32_t sys, uint64_t nb) {
    if (nb == 0) nb = 1;
    for (uint64_t q = 0; q < nb; ++q) v.push_back(BlkMap{sys, (uint32_t)q, (uint32_t)nb, 0u});
  };
  int build_threads = 32;
  size_t build_smem = 0;
  // the part map ordered by step-kernel variant (list width, cubic box)
  unsigned step_off[4] = {0, 0, 0, 0}, step_n[4] = {0, 0, 0, 0};
  b->n_step_variants = 0;
  for (int v = 0; v < 4; ++v) {
    step_off[v] = (unsigned)part.size();
    for (uint32_t q = 0; q < b->n_active; ++q)
      if ((table[q].nl16 ? 2 : 0) + (table[q].cubic ? 1 : 0) == v) add(part, q, (table[q].n + 255) / 256);
    step_n[v] = (unsigned)part.size() - step_off[v];
    if (step_n[v]) b->n_step_variants += 1;
  }
  for (uint32_t q = 0; q < b->n_active; ++q) {
    Sys& S = table[q];
    S.in_batch = 1;
    S.batch = b->bctl;
    S.n_members = b->n_active;
    add(cell, q, ((uint64_t)S.ncell + 255) / 256);
    add(tile, q, ((uint64_t)S.ncell + SCAN_TILE - 1) / SCAN_TILE);
    add(one, q, 1);
    add(build, q, (uint64_t)S.tiles_y * S.nc[2]);
    build_threads = std::max(build_threads, S.tile_threads);
    build_smem = std::max(build_smem, build_tile_smem(S));
  }
  const size_t nmaps = part.size() + cell.size() + tile.size() + one.size() + build.size();
  if (b->n_active > b->T_cap) {
    if (b->T) CKB(cudaFreeAsync(b->T, b->stream));
    b->T = nullptr;
    b->T_cap = 0;
    const size_t cap = std::max<size_t>(b->n_active, 2 * b->members.size());
    CKB(cudaMallocAsync((void**)&b->T, sizeof(Sys) * cap, b->stream));
    b->T_cap = cap;
  }
  if (2 * nmaps > b->maps_cap) {
    if (b->maps) CKB(cudaFreeAsync(b->maps, b->stream));
    b->maps = nullptr;
    b->maps_cap = 0;
    CKB(cudaMallocAsync((void**)&b->maps, sizeof(BlkMap) * 4 * nmaps, b->stream));
    b->maps_cap = 4 * nmaps;
  }
  if (!b->act_n) CKB(cudaMallocAsync((void**)&b->act_n, sizeof(uint32_t) * 8, b->stream));
  CKB(cudaMemsetAsync(b->act_n, 0, sizeof(uint32_t) * 8, b->stream));
  std::vector<BlkMap> all;
  all.reserve(nmaps);
  BatchLaunch& L = b->L;
  L.T = b->T;
  auto place = [&](std::vector<BlkMap>& v, const BlkMap** ptr, unsigned* cnt) {
    *ptr = b->maps + all.size();
    *cnt = (unsigned)v.size();
    all.insert(all.end(), v.begin(), v.end());
  };
  place(part, &L.part, &L.n_part);
  place(cell, &L.cell, &L.n_cell);
  place(tile, &L.tile, &L.n_tile);
  place(one, &L.one, &L.n_one);
  place(build, &L.build, &L.n_build);
  L.build_threads = build_threads;
  L.build_smem = build_smem;
  L.act = b->maps + nmaps;
  L.act_n = b->act_n;
  for (int v = 0; v < 4; ++v) {
    L.step_off[v] = step_off[v];
    L.step_n[v] = step_n[v];
  }
  {
    const size_t tb = sizeof(Sys) * table.size(), mb = sizeof(BlkMap) * all.size();
    prx_batch::Stage& sg = b->stage[b->stage_next];
    b->stage_next = (b->stage_next + 1) % 4;
    if (sg.used) CKB(cudaEventSynchronize(sg.used));  // normally long complete
    else CKB(cudaEventCreateWithFlags(&sg.used, cudaEventDisableTiming));
    if (sg.cap < tb + mb) {
      if (sg.host) CKB(cudaFreeHost(sg.host));
      sg.host = nullptr;
      sg.cap = 0;
      const size_t cap = 2 * (tb + mb) + 4096;
      CKB(cudaMallocHost((void**)&sg.host, cap));
      sg.cap = cap;
    }
    memcpy(sg.host, table.data(), tb);
    memcpy(sg.host + tb, all.data(), mb);
    CKB(cudaMemcpyAsync(b->T, sg.host, tb, cudaMemcpyHostToDevice, b->stream));
    CKB(cudaMemcpyAsync(b->maps, sg.host + tb, mb, cudaMemcpyHostToDevice, b->stream));
    CKB(cudaEventRecord(sg.used, b->stream));
  }
  if (configure_batch_build_kernel(build_smem))
    return bfail(b, PRX_ECUDA, "list-build shared memory of " + std::to_string(build_smem) + " bytes refused");
  const int chunk = b->any_rx ? (int)b->theta : kNoRxChunk;
  auto step = [&](cudaGraphConditionalHandle h) { launch_batch_step(L, b->cap, h, 1); };
  auto rebuild = [&] { launch_batch_rebuild(L, b->cap); };
  auto rx = [&] { launch_batch_rx(L, b->cap); };
  // device-driven runs first; the host-replayed graphs only if those fail
  {
    cudaError_t e = capture_device_graph(b->cap, [&] {
      launch_batch_step(L, b->cap, 0, 0);
      launch_dgb_next(b->bctl, b->cap);
    }, &b->dg_step);
    if (e == cudaSuccess) e = capture_device_graph(b->cap, rebuild, &b->dg_rebuild);
    if (e == cudaSuccess && b->any_rx) e = capture_device_graph(b->cap, rx, &b->dg_react);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap);
    b->dg_ok = e == cudaSuccess;
    if (!b->dg_ok) {
      cudaGetLastError();
      if (b->dg_step) cudaGraphExecDestroy(b->dg_step);
      if (b->dg_rebuild) cudaGraphExecDestroy(b->dg_rebuild);
      if (b->dg_react) cudaGraphExecDestroy(b->dg_react);
      b->dg_step = b->dg_rebuild = b->dg_react = nullptr;
    }
  }
  if (!b->dg_ok) {
    CKB(capture_graph(b->cap, 1, false, step, rebuild, rx, &b->g_step));
    CKB(capture_graph(b->cap, chunk, b->any_rx, step, rebuild, rx, &b->g_chunk));
    if (b->any_rx) CKB(capture_graph(b->cap, 0, true, step, rebuild, rx, &b->g_react));
  }
  b->valid = true;
  return PRX_OK;
}

// Device bytes of a system of descriptor d whose list cutoff includes
// r_react (0: the WCA cutoff alone).
uint64_t estimate_bytes(const prx_system_desc& d, double r_react) {
  // mirrors the allocations of prx_create and of the cell grid / Verlet
  // list set up for the larger of the WCA and reaction cutoffs
  const prx_system_desc* desc = &d;
  const uint64_t n = desc->n, cap = desc->adj_cap ? desc->adj_cap : 1;
  const double rc = std::max(std::pow(2.0, 1.0 / 6.0) * desc->wca_sigma, r_react);
  double skin = desc->skin < 0.0 ? kDefaultSkin : desc->skin;
  const double Lmin = std::min(desc->box[0], std::min(desc->box[1], desc->box[2]));
  if (Lmin / (rc + skin) < 3.0) skin = std::max(0.02, Lmin / 3.0 - rc);
  const double rv = rc + skin;
  uint64_t ncell = 1;
  int nc[3];
  for (int k = 0; k < 3; ++k) {
    nc[k] = std::max(3, std::min(1023, (int)std::floor(desc->box[k] / rv)));
    ncell *= (uint64_t)nc[k];
  }
  const double V = desc->box[0] * desc->box[1] * desc->box[2];
  const double mean_nb = (double)n / V * 4.0 / 3.0 * M_PI * rv * rv * rv;
  const uint64_t list_cap =
      (uint64_t)((std::max(32, std::min(252, (int)std::ceil(2.5 * mean_nb + 16.0))) + 3) & ~3);
  const uint64_t nl_bytes = n <= 65535 ? 2 : 4;  // as setup_grid
  const uint64_t per_set = n * (6 * 8 + 4 + 3 + 4 * cap);
  const uint64_t nblk = std::max<uint64_t>(n / RX_THREADS + 1, ncell / SCAN_TILE + 1) + 1;
  const uint64_t allocs = 40;  // separate cudaMalloc calls, each rounded up
  return 2 * per_set + n * (2 * 16 + 4 * 4) + (n * cap / 2 + 1) * sizeof(prx_bond) +
           (kHistCap + 2ull) * sizeof(prx_history_record) + sizeof(Ctl) + 32 * (n / RX_THREADS + 2) +
           32 * n + ncell * 12 + 8 * nblk + list_cap * n * nl_bytes + 2 * n + 16384 + allocs * 4096;
}


void free_slot(prx_batch* b, prx_system* sys);  // (defined with the batch entry points)

// Calls that would change a batch member on its own are refused.
int refuse_member(prx_system* sys) {
  return fail(sys, PRX_EINVAL, "not allowed while the system is a member of a batch");
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* prx_status_string(int st) {
  switch (st) {
    case PRX_OK: return "ok";
    case PRX_EINVAL: return "invalid argument";
    case PRX_ENOMEM: return "out of memory";
    case PRX_ECAPACITY: return "capacity exceeded";
    case PRX_EOVERSTRETCH: return "FENE bond overstretched";
    case PRX_ENONFINITE: return "non-finite value or particle jump";
    case PRX_ETIMEOUT: return "device wait timed out";
    case PRX_ECUDA: return "CUDA error";
    case PRX_EIO: return "I/O error";
    default: return "unknown status";
  }
}

// With sys == NULL: the message of the last failed prx_create / prx_load on this thread.
const char* prx_last_error(const prx_system* sys) { return sys ? sys->err.c_str() : g_create_error.c_str(); }

int prx_estimate_bytes(const prx_system_desc* desc, const prx_reaction_desc* rx, uint64_t* bytes) {
  if (!desc || !bytes) return PRX_EINVAL;
  *bytes = estimate_bytes(*desc, rx ? rx->r_react : 0.0);
  return PRX_OK;
}

int prx_create(const prx_system_desc* desc, const double* pos, const double* vel, const uint8_t* type,
               const int8_t* state, const prx_bond* bonds, uint64_t n_bonds, void* cuda_stream,
               prx_system** out) {
  return create_impl(desc, pos, vel, type, state, bonds, n_bonds, cuda_stream, nullptr, nullptr, nullptr,
                     nullptr, 0, 0.0, nullptr, nullptr, nullptr, 0, out);
}

void prx_destroy(prx_system* sys) {
  if (!sys) return;
  if (sys->batch) prx_batch_remove(sys->batch, sys);
  if (sys->stream) cudaStreamSynchronize(sys->stream);
  if (sys->slot_batch) free_slot(sys->slot_batch, sys);  // admitted, finished, not yet polled
  if (sys->join_ev) cudaEventDestroy(sys->join_ev);
  destroy_graphs(sys);
  for (auto& e : sys->prof) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  free_list(sys->grid_allocs);
  free_list(sys->dev_allocs);
  if (sys->ctl_host) cudaFreeHost(sys->ctl_host);
  if (sys->obs_host) cudaFreeHost(sys->obs_host);
  for (cudaEvent_t& e : sys->obs_ev)
    if (e) cudaEventDestroy(e);
  if (sys->cap) cudaStreamDestroy(sys->cap);
  if (sys->own_stream && sys->stream) cudaStreamDestroy(sys->stream);
  delete sys;
}

int prx_set_reaction(prx_system* sys, const prx_reaction_desc* rx) {
  return prx_set_reactions(sys, rx, rx ? 1u : 0u);
}

int prx_set_reactions(prx_system* sys, const prx_reaction_desc* rx, uint32_t n_rx) {
  if (!sys) return PRX_EINVAL;
  if (sys->batch) return refuse_member(sys);
  if (!rx || n_rx == 0) {
    sys->has_rx = 0;
    sys->S.has_rx = 0;
    sys->nrx = 0;
    destroy_graphs(sys);
    return PRX_OK;
  }
  int rc = validate_rxs(sys, rx, n_rx);
  if (rc) return rc;
  CK(cudaStreamSynchronize(sys->stream));
  sys->rxd = rx[0];
  sys->nrx = n_rx;
  for (uint32_t q = 0; q < n_rx; ++q) sys->rxs[q] = rx[q];
  RxParams& R = sys->S.R;
  R = RxParams{};
  R.mask_A = rx->type_mask_A;
  R.mask_T = rx->type_mask_T;
  R.a_lo = rx->a_lo;
  R.a_hi = rx->a_hi;
  R.t_lo = rx->t_lo;
  R.t_hi = rx->t_hi;
  R.dA = rx->dA;
  R.dT = rx->dT;
  R.p = rx->k * sys->d.dt * (double)rx->theta;
  R.p53 = p53_of(R.p);
  R.rr2 = rx->r_react * rx->r_react;
  const double rmax = max_r_react(sys);
  R.rr2_pre = (float)((rmax + 1e-3) * (rmax + 1e-3));
  {
    // bound on |r^2(FP32, fixed point) - r^2(FP64)| near the cutoff: the
    // fixed-point positions are within 3 units of L / 2^32, the conversion
    // and FP32 arithmetic within 2e-7 (relative), for |d| ~ r_react <= 2
    const double u = std::max(sys->d.box[0], std::max(sys->d.box[1], sys->d.box[2])) / 4294967296.0;
    const double margin = 2.0 * std::sqrt(3.0) * rx->r_react * (6.0 * u + 2e-7 * rx->r_react) +
                          4e-7 * R.rr2 + 1e-9;
    R.rr2_in = std::nextafter((float)std::max(0.0, R.rr2 - 2.0 * margin), 0.0f);
  }
  R.style = (uint32_t)rx->bond_style;
  R.rule = rx->selection;
  for (int t = 0; t < PRX_MAX_TYPES; ++t) R.maxval[t] = rx->max_valence[t];
  // concurrent reactions: per-reaction parameters and, for every candidate
  // set m (bit q: reaction q), the cumulative acceptance bounds of its
  // members in the scheme's order, P_j summed in FP64
  R.nr = (int32_t)n_rx;
  double p_r[PRX_MAX_REACTIONS];
  for (uint32_t q = 0; q < n_rx; ++q) {
    const prx_reaction_desc& x = rx[q];
    R.mA[q] = x.type_mask_A;
    R.mT[q] = x.type_mask_T;
    R.alo[q] = x.a_lo;
    R.ahi[q] = x.a_hi;
    R.tlo[q] = x.t_lo;
    R.thi[q] = x.t_hi;
    R.dAr[q] = x.dA;
    R.dTr[q] = x.dT;
    R.styler[q] = (uint32_t)x.bond_style;
    for (int t = 0; t < PRX_MAX_TYPES; ++t) R.maxvalr[q][t] = x.max_valence[t];
    R.rr2r[q] = x.r_react * x.r_react;
    p_r[q] = x.k * sys->d.dt * (double)x.theta;
  }
  for (uint32_t m = 1; m < (1u << n_rx); ++m) {
    double P = 0.0;
    int j = 0;
    for (uint32_t q = 0; q < n_rx; ++q) {
      if (!((m >> q) & 1u)) continue;
      P = P + p_r[q];
      R.p53c[m][j++] = p53_of(P);
    }
  }
  sys->has_rx = 1;
  sys->S.has_rx = 1;
  destroy_graphs(sys);
  const double need = std::max(wca_rc(sys->d), rmax);
  if (need > sys->grid_rcut) {
    if ((rc = setup_grid(sys, need))) return rc;
    if ((rc = full_rebin(sys, 1))) return rc;
    if ((rc = sync_status(sys))) return rc;
  }
  return PRX_OK;
}

int prx_run(prx_system* sys, uint64_t nsteps) {
  if (!sys) return PRX_EINVAL;
  if (sys->batch) return refuse_member(sys);
  if (sys->S.n == 0) {
    sys->host_step += nsteps;
    return PRX_OK;
  }
  if (sys->profiling) {
    for (uint64_t q = 0; q < nsteps; ++q) {
      int rc = direct_step(sys);
      if (rc) return rc;
    }
    return PRX_OK;
  }
  int rc = ensure_graphs(sys);
  if (rc) return rc;
  if (sys->dg_ok) {
    // one device-driven chain of nsteps steps (with the rebuilds and the
    // reaction steps it decides on) behind one host launch
    if (nsteps == 0) return PRX_OK;
    launch_dg_arm(sys->S, sys->stream, nsteps, (unsigned long long)sys->dg_rebuild,
                  (unsigned long long)sys->dg_react);
    CK(cudaGraphLaunch(sys->dg_step, sys->stream));
    if (sys->has_rx) {
      const uint64_t th = sys->rxd.theta;
      sys->graph_rx_launches += (sys->host_step + nsteps) / th - sys->host_step / th;
    }
    sys->host_step += nsteps;
    sys->step_launches += nsteps;
    sys->other_launches += 1 + nsteps;  // the arm kernel, one k_dg_next per step
    return PRX_OK;
  }
  const uint64_t theta = sys->has_rx ? sys->rxd.theta : (uint64_t)kNoRxChunk;
  const uint64_t m = sys->chunk_m;
  while (nsteps > 0) {
    if (sys->host_step % theta == 0 && nsteps >= theta) {
      const bool many = m > 1 && nsteps >= m * theta;
      const uint64_t k = many || m == 1 ? m : 1;  // intervals in this replay
      CK(cudaGraphLaunch(many || m == 1 ? sys->g_chunk : sys->g_chunk1, sys->stream));
      sys->host_step += k * theta;
      sys->step_launches += k * theta;
      if (sys->has_rx) sys->graph_rx_launches += k;
      nsteps -= k * theta;
    } else {
      CK(cudaGraphLaunch(sys->g_step, sys->stream));
      sys->host_step++;
      sys->step_launches++;
      nsteps--;
      if (sys->has_rx && sys->host_step % theta == 0) {
        CK(cudaGraphLaunch(sys->g_react, sys->stream));
        sys->graph_rx_launches++;
      }
    }
  }
  return PRX_OK;
}

int prx_sync(prx_system* sys) {
  if (!sys) return PRX_EINVAL;
  return sync_status(sys);
}

int prx_react_once(prx_system* sys, uint64_t step, prx_rx_trace* trace) {
  if (!sys) return PRX_EINVAL;
  if (sys->batch) return refuse_member(sys);
  if (!sys->has_rx) return fail(sys, PRX_EINVAL, "no reaction scheme set");
  if (sys->S.n) {
    launch_rx(sys->S, sys->stream, (long long)step, sys->profiling ? prof_hook : nullptr, sys);
    sys->other_launches += rx_kernel_count(sys->S.R.rule);
    CK(cudaGetLastError());
  }
  int rc = sync_status(sys);
  if (trace) {
    trace->candidates = sys->ctl_host->trace[0];
    trace->retained = sys->ctl_host->trace[1];
    trace->a_winners = sys->ctl_host->trace[2];
    trace->formed = sys->ctl_host->trace[3];
    if (!sys->S.n) memset(trace, 0, sizeof(*trace));
  }
  return rc;
}

int prx_compute_forces(prx_system* sys, double* f_out, double* epot_out) {
  if (!sys || (!f_out && sys->S.n)) return PRX_EINVAL;
  if (sys->batch) return refuse_member(sys);
  const size_t n = sys->S.n;
  if (!n) {
    if (epot_out) *epot_out = 0.0;
    return PRX_OK;
  }
  launch_step(sys->S, sys->stream, sys->d.force_precision == PRX_FORCE_FP64, 1, 0, 0);
  sys->other_launches++;
  CK(cudaGetLastError());
  std::vector<double> f(3 * n), e(n);
  CK(cudaMemcpyAsync(f.data(), sys->S.fout, 24 * n, cudaMemcpyDeviceToHost, sys->stream));
  CK(cudaMemcpyAsync(e.data(), sys->S.eout, 8 * n, cudaMemcpyDeviceToHost, sys->stream));
  HostSlots h;
  int rc = fetch_slots(sys, h, 0u);
  if (rc) return rc;
  std::vector<double> e_by_id(n);
  for (size_t s = 0; s < n; ++s) {
    const uint32_t p = h.id[s];
    for (int k = 0; k < 3; ++k) f_out[3 * (size_t)p + k] = f[3 * s + k];
    e_by_id[p] = e[s];
  }
  if (epot_out) {
    double t = 0.0;
    for (size_t p = 0; p < n; ++p) t += e_by_id[p];
    *epot_out = t;
  }
  return sync_status(sys);
}

int prx_get_step(prx_system* sys, uint64_t* step) {
  if (!sys || !step) return PRX_EINVAL;
  int rc = sync_status(sys);
  *step = sys->S.n ? sys->ctl_host->step : sys->host_step;  // an empty system launches nothing
  return rc;
}

// Per-particle read-back: arranged in particle order on the device (into
// the force scratch buffer), then one copy into the caller's buffer.
int readback_by_id(prx_system* sys, int what, void* out, size_t bytes) {
  if (!sys || (!out && sys->S.n)) return PRX_EINVAL;
  if (sys->S.n) {
    launch_gather_by_id(sys->S, sys->stream, what, sys->S.fout);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, sys->S.fout, bytes, cudaMemcpyDeviceToHost, sys->stream));
  }
  return sync_status(sys);
}

int prx_get_positions(prx_system* sys, double* out) {
  return readback_by_id(sys, 2, out, sys ? 24ull * sys->S.n : 0);
}

int prx_get_velocities(prx_system* sys, double* out) {
  return readback_by_id(sys, 3, out, sys ? 24ull * sys->S.n : 0);
}

int prx_get_states(prx_system* sys, int8_t* out) {
  return readback_by_id(sys, 0, out, sys ? (size_t)sys->S.n : 0);
}

int prx_get_types(prx_system* sys, uint8_t* out) {
  return readback_by_id(sys, 1, out, sys ? (size_t)sys->S.n : 0);
}

int prx_get_bonds(prx_system* sys, prx_bond* out, uint64_t cap, uint64_t* n_out) {
  if (!sys || !n_out) return PRX_EINVAL;
  int rc = read_ctl(sys);
  if (rc) return rc;
  // (a failed reaction step can leave the counter past the list's capacity)
  const uint64_t nb = std::min<uint64_t>(sys->ctl_host->nbonds, sys->S.bond_cap);
  *n_out = nb;
  const uint64_t m = std::min(cap, nb);
  if (!m || !out) {  // the count alone
    rc = sync_status(sys);
    if (rc) return rc;
    return cap < nb ? fail(sys, PRX_ECAPACITY, "bond buffer too small") : PRX_OK;
  }
  std::vector<prx_bond> b(nb);
  if (nb) {
    CK(cudaMemcpyAsync(b.data(), sys->S.bonds, sizeof(prx_bond) * nb, cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
  }
  std::stable_sort(b.begin(), b.end(), [](const prx_bond& x, const prx_bond& y) {
    if (x.step != y.step) return x.step < y.step;
    if (x.a != y.a) return x.a < y.a;
    return x.t < y.t;
  });
  memcpy(out, b.data(), sizeof(prx_bond) * m);
  rc = sync_status(sys);
  if (rc) return rc;
  return cap < nb ? fail(sys, PRX_ECAPACITY, "bond buffer too small") : PRX_OK;
}

// Enqueues the observables and their copy into pinned slot q (no wait).
int enqueue_observables(prx_system* sys, int q) {
  const uint32_t n = sys->S.n;
  const int nblk = (int)((n + RX_THREADS - 1) / RX_THREADS);
  auto* oh = sys->obs_host + q;
  if (n) {
    launch_observables(sys->S, sys->stream, nblk);
    sys->other_launches += 3;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(oh->sums, sys->S.red + 4 * (size_t)nblk, sizeof(oh->sums), cudaMemcpyDeviceToHost,
                       sys->stream));
    CK(cudaMemcpyAsync(&oh->rec, &sys->S.hist[sys->S.hist_cap], sizeof(HistRec), cudaMemcpyDeviceToHost,
                       sys->stream));
  }
  CK(cudaMemcpyAsync(&oh->ctl, sys->S.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, sys->stream));
  return PRX_OK;
}

// Fills *out from pinned slot q (its copies complete).
int fill_observables(prx_system* sys, int q, prx_observables* out) {
  const auto* oh = sys->obs_host + q;
  memset(out, 0, sizeof(*out));
  if (sys->S.n) {
    out->ke_half = oh->sums[0];
    for (int k = 0; k < 3; ++k) out->momentum[k] = oh->sums[1 + k];
    for (int t = 0; t < PRX_MAX_TYPES; ++t)
      for (int s = 0; s < PRX_MAX_STATES; ++s) out->counts[t][s] = oh->rec.counts[t][s];
  }
  out->step = (int64_t)oh->ctl.step;
  out->bonds = (int64_t)oh->ctl.nbonds;
  *sys->ctl_host = oh->ctl;
  const int st = oh->ctl.status;
  if (st) return fail(sys, st, std::string("device reported ") + prx_status_string(st));
  return PRX_OK;
}

int prx_get_observables(prx_system* sys, prx_observables* out) {
  if (!sys || !out) return PRX_EINVAL;
  int rc = enqueue_observables(sys, PRX_OBS_SLOTS);
  if (rc) return rc;
  CK(cudaStreamSynchronize(sys->stream));  // one wait for sums, populations and control block
  return fill_observables(sys, PRX_OBS_SLOTS, out);
}

int prx_observables_begin(prx_system* sys, int slot) {
  if (!sys) return PRX_EINVAL;
  if (sys->batch) return refuse_member(sys);
  if (slot < 0 || slot >= PRX_OBS_SLOTS) return fail(sys, PRX_EINVAL, "observables slot out of range");
  if (sys->obs_pending[slot]) return fail(sys, PRX_EINVAL, "observables slot still pending");
  if (!sys->obs_ev[slot] && cudaEventCreateWithFlags(&sys->obs_ev[slot], cudaEventDisableTiming) != cudaSuccess)
    return fail(sys, PRX_ECUDA, "event creation failed");
  int rc = enqueue_observables(sys, slot);
  if (rc) return rc;
  CK(cudaEventRecord(sys->obs_ev[slot], sys->stream));
  sys->obs_pending[slot] = true;
  return PRX_OK;
}

int prx_observables_end(prx_system* sys, int slot, prx_observables* out) {
  if (!sys || !out) return PRX_EINVAL;
  if (slot < 0 || slot >= PRX_OBS_SLOTS || !sys->obs_pending[slot])
    return fail(sys, PRX_EINVAL, "no pending observables in this slot");
  sys->obs_pending[slot] = false;
  CK(cudaEventSynchronize(sys->obs_ev[slot]));
  return fill_observables(sys, slot, out);
}

int prx_history_begin(prx_system* sys, int slot) {
  if (!sys) return PRX_EINVAL;
  if (sys->batch) return refuse_member(sys);
  if (slot < 0 || slot >= PRX_OBS_SLOTS) return fail(sys, PRX_EINVAL, "slot out of range");
  if (sys->obs_pending[slot]) return fail(sys, PRX_EINVAL, "slot still pending");
  if (!sys->obs_ev[slot] && cudaEventCreateWithFlags(&sys->obs_ev[slot], cudaEventDisableTiming) != cudaSuccess)
    return fail(sys, PRX_ECUDA, "event creation failed");
  auto* oh = sys->obs_host + slot;
  if (sys->S.n) {
    CK(cudaMemcpyAsync(&oh->rec, &sys->S.hist[sys->S.hist_cap + 1], sizeof(HistRec), cudaMemcpyDeviceToHost,
                       sys->stream));
  } else {
    memset(&oh->rec, 0, sizeof(HistRec));
  }
  CK(cudaMemcpyAsync(&oh->ctl, sys->S.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, sys->stream));
  CK(cudaEventRecord(sys->obs_ev[slot], sys->stream));
  sys->obs_pending[slot] = true;
  return PRX_OK;
}

int prx_history_end(prx_system* sys, int slot, prx_history_record* out) {
  if (!sys || !out) return PRX_EINVAL;
  if (slot < 0 || slot >= PRX_OBS_SLOTS || !sys->obs_pending[slot])
    return fail(sys, PRX_EINVAL, "nothing pending in this slot");
  sys->obs_pending[slot] = false;
  CK(cudaEventSynchronize(sys->obs_ev[slot]));
  const auto* oh = sys->obs_host + slot;
  memcpy(out, &oh->rec, sizeof(*out));
  *sys->ctl_host = oh->ctl;
  const int st = oh->ctl.status;
  if (st) return fail(sys, st, std::string("device reported ") + prx_status_string(st));
  return PRX_OK;
}

int prx_get_history(prx_system* sys, prx_history_record* out, uint64_t cap, uint64_t* n_out) {
  if (!sys || !n_out) return PRX_EINVAL;
  int rc = read_ctl(sys);
  if (rc) return rc;
  const uint64_t total = sys->ctl_host->hist_count;
  const uint64_t kept = std::min<uint64_t>(total, sys->S.hist_cap);
  const uint64_t m = std::min(cap, kept);
  *n_out = m;
  if (m && out) {
    std::vector<HistRec> all(sys->S.hist_cap);
    CK(cudaMemcpyAsync(all.data(), sys->S.hist, sizeof(HistRec) * sys->S.hist_cap, cudaMemcpyDeviceToHost,
                       sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    const uint64_t first = total - m;
    for (uint64_t q = 0; q < m; ++q) memcpy(&out[q], &all[(first + q) % sys->S.hist_cap], sizeof(HistRec));
  }
  return sync_status(sys);
}

int prx_get_stats(prx_system* sys, prx_stats* out) {
  if (!sys || !out) return PRX_EINVAL;
  int rc = read_ctl(sys);
  if (rc) return rc;
  memset(out, 0, sizeof(*out));
  out->steps = sys->ctl_host->step;
  out->reactions = sys->ctl_host->reactions;
  out->rebins = sys->ctl_host->rebins;
  out->step_launches = sys->step_launches;
  // every rebuild, inside a graph's IF node or launched directly, is the same
  // sequence of kernels and increments the device counter once
  out->kernel_launches = sys->step_launches * (uint64_t)step_kernel_count(sys->d.force_precision) +
                         sys->ctl_host->rebins * (uint64_t)rebin_kernel_count(sys->S) +
                         sys->graph_rx_launches * (uint64_t)rx_kernel_count(sys->S.R.rule) + sys->other_launches;
  for (int k = 0; k < 3; ++k) {
    out->cells[k] = (uint32_t)sys->S.nc[k];
    out->cell_edge[k] = sys->d.box[k] / sys->S.nc[k];
  }
  return sync_status(sys);
}

int prx_profile_begin(prx_system* sys) {
  if (!sys) return PRX_EINVAL;
  if (sys->batch) return refuse_member(sys);
  CK(cudaStreamSynchronize(sys->stream));
  for (auto& e : sys->prof) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  sys->prof.clear();
  sys->profiling = true;
  return PRX_OK;
}

int prx_profile_end(prx_system* sys, prx_kernel_time* out, uint32_t cap, uint32_t* n_out) {
  if (!sys || !n_out) return PRX_EINVAL;
  CK(cudaStreamSynchronize(sys->stream));
  std::map<std::string, std::pair<uint64_t, double>> agg;
  std::vector<std::string> order;
  for (auto& e : sys->prof) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e.a, e.b);
    if (!agg.count(e.name)) order.push_back(e.name);
    agg[e.name].first += 1;
    agg[e.name].second += ms;
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  sys->prof.clear();
  sys->profiling = false;
  *n_out = (uint32_t)order.size();
  for (uint32_t q = 0; q < order.size() && q < cap && out; ++q) {
    memset(&out[q], 0, sizeof(prx_kernel_time));
    strncpy(out[q].name, order[q].c_str(), sizeof(out[q].name) - 1);
    out[q].launches = agg[order[q]].first;
    out[q].total_ms = agg[order[q]].second;
  }
  return sync_status(sys);
}

// Checkpoint: descriptor, reaction, step, then per-slot arrays in slot order
// (ids, cells, positions, velocities, types, states, adjacency as partner
// ids) and the bond list.  Restoring the slot order and the cell of every
// slot makes the continued run identical bit for bit.
int prx_save(prx_system* sys, const char* path) {
  if (!sys || !path) return PRX_EINVAL;
  HostSlots h;
  int rc = fetch_slots(sys, h, FS_POS | FS_VEL | FS_TYPE | FS_STATE | FS_TOPO);
  if (rc) return rc;
  rc = sync_status(sys);
  if (rc) return rc;
  const uint64_t n = sys->S.n, cap = sys->S.cap,
                 nb = std::min<uint64_t>(sys->ctl_host->nbonds, sys->S.bond_cap);
  std::vector<prx_bond> bonds(nb);
  if (nb) {
    CK(cudaMemcpy(bonds.data(), sys->S.bonds, sizeof(prx_bond) * nb, cudaMemcpyDeviceToHost));
  }
  std::vector<uint32_t> cells(n), adj_ids(n * cap, 0u), wref(n);
  std::vector<uint32_t> cs((size_t)sys->S.ncell + 1);
  std::vector<uint8_t> nn(n);
  const int lcap = sys->S.list_cap;
  std::vector<int32_t> nl((size_t)lcap * n);
  if (n) {
    CK(cudaMemcpy(cs.data(), sys->S.cell_start, 4 * cs.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(nn.data(), sys->S.nn, n, cudaMemcpyDeviceToHost));
    if (sys->S.nl16) {
      std::vector<uint16_t> v((size_t)lcap * n);
      CK(cudaMemcpy(v.data(), sys->S.nl, 2 * v.size(), cudaMemcpyDeviceToHost));
      for (size_t q = 0; q < v.size(); ++q) nl[q] = v[q];
    } else {
      CK(cudaMemcpy(nl.data(), sys->S.nl, 4 * nl.size(), cudaMemcpyDeviceToHost));
    }
  }
  uint32_t c = 0;
  for (uint64_t q = 0; q < n; ++q) {
    while (cs[c + 1] <= q) ++c;  // slot q lies in cell c of the last rebuild
    cells[q] = c;
    wref[q] = h.P[q].w;
    for (uint32_t b = 0; b < h.nadj[q]; ++b) {
      const uint32_t e = h.adj[q * cap + b];
      adj_ids[q * cap + b] = h.id[e & SLOT_MASK] | (e & ~SLOT_MASK);
    }
  }
  FILE* f = fopen(path, "wb");
  if (!f) return fail(sys, PRX_EIO, std::string("cannot open ") + path);
  bool ok = true;
  auto W = [&](const void* p, size_t sz) {
    if (sz && fwrite(p, 1, sz, f) != sz) ok = false;
  };
  const uint64_t magic = kCkptMagic, step = sys->ctl_host->step;
  W(&magic, 8);
  W(&sys->d, sizeof(sys->d));
  // the reaction count (0 or 1 in files with at most one reaction), then
  // the first reaction and, with several, the others
  const int nrx = sys->has_rx ? (int)sys->nrx : 0;
  W(&nrx, sizeof(int));
  W(&sys->rxd, sizeof(sys->rxd));
  for (int q = 1; q < nrx; ++q) W(&sys->rxs[q], sizeof(sys->rxs[q]));
  W(&step, 8);
  W(&nb, 8);
  W(&sys->grid_rcut, 8);
  W(h.id.data(), 4 * n);
  W(cells.data(), 4 * n);
  W(h.x.data(), 8 * n);
  W(h.y.data(), 8 * n);
  W(h.z.data(), 8 * n);
  W(h.vx.data(), 8 * n);
  W(h.vy.data(), 8 * n);
  W(h.vz.data(), 8 * n);
  W(h.type.data(), n);
  W(h.state.data(), n);
  W(h.nadj.data(), n);
  W(adj_ids.data(), 4 * n * cap);
  W(bonds.data(), sizeof(prx_bond) * nb);
  W(&lcap, sizeof(int));
  W(wref.data(), 4 * n);
  W(nn.data(), n);
  W(nl.data(), 4 * (size_t)lcap * n);
  if (fclose(f) != 0) ok = false;
  return ok ? PRX_OK : fail(sys, PRX_EIO, "write failed");
}

int prx_load(const char* path, void* cuda_stream, prx_system** out) {
  if (!path || !out) return PRX_EINVAL;
  FILE* f = fopen(path, "rb");
  if (!f) return PRX_EIO;
  bool ok = true;
  auto R = [&](void* p, size_t sz) {
    if (sz && fread(p, 1, sz, f) != sz) ok = false;
  };
  uint64_t magic = 0, step = 0, nb = 0;
  prx_system_desc d;
  prx_reaction_desc rxs[PRX_MAX_REACTIONS];
  int has_rx = 0;
  double grid_rcut = 0.0;
  R(&magic, 8);
  if (!ok || magic != kCkptMagic) {
    fclose(f);
    return PRX_EIO;
  }
  R(&d, sizeof(d));
  R(&has_rx, sizeof(int));
  if (has_rx < 0 || has_rx > PRX_MAX_REACTIONS) ok = false;
  R(&rxs[0], sizeof(rxs[0]));
  for (int q = 1; ok && q < has_rx; ++q) R(&rxs[q], sizeof(rxs[q]));
  R(&step, 8);
  R(&nb, 8);
  R(&grid_rcut, 8);
  const uint64_t n = d.n, cap = d.adj_cap;
  if (!ok || cap < 1 || cap > PRX_MAX_ADJ || n > 0x7FFFFFF0ull) {
    fclose(f);
    return PRX_EIO;
  }
  std::vector<uint32_t> ids(n), cells(n), adj_ids(n * cap);
  std::vector<double> x(n), y(n), z(n), vx(n), vy(n), vz(n), pos(3 * n), vel(3 * n);
  std::vector<uint8_t> type(n), nadj(n), type_id(n);
  std::vector<int8_t> state(n), state_id(n);
  std::vector<prx_bond> bonds(nb);
  R(ids.data(), 4 * n);
  R(cells.data(), 4 * n);
  R(x.data(), 8 * n);
  R(y.data(), 8 * n);
  R(z.data(), 8 * n);
  R(vx.data(), 8 * n);
  R(vy.data(), 8 * n);
  R(vz.data(), 8 * n);
  R(type.data(), n);
  R(state.data(), n);
  R(nadj.data(), n);
  R(adj_ids.data(), 4 * n * cap);
  R(bonds.data(), sizeof(prx_bond) * nb);
  int lcap = 0;
  R(&lcap, sizeof(int));
  if (!ok || lcap < 1 || lcap > 255) {
    fclose(f);
    return PRX_EIO;
  }
  std::vector<uint32_t> wref(n);
  std::vector<uint8_t> nn(n);
  std::vector<int32_t> nl((size_t)lcap * n);
  R(wref.data(), 4 * n);
  R(nn.data(), n);
  R(nl.data(), 4 * (size_t)lcap * n);
  fclose(f);
  if (!ok) return PRX_EIO;
  for (uint64_t s = 0; s < n; ++s) {
    const uint32_t p = ids[s];
    if (p >= n) return PRX_EIO;
    pos[3 * p] = x[s];
    pos[3 * p + 1] = y[s];
    pos[3 * p + 2] = z[s];
    vel[3 * p] = vx[s];
    vel[3 * p + 1] = vy[s];
    vel[3 * p + 2] = vz[s];
    type_id[p] = type[s];
    state_id[p] = state[s];
  }
  // recreate with the reaction's grid so that the saved cells are valid
  prx_system* sys = nullptr;
  int rc = create_impl(&d, pos.data(), vel.data(), type_id.data(), state_id.data(), bonds.data(), nb, cuda_stream,
                       ids.data(), cells.data(), adj_ids.data(), nadj.data(), step, grid_rcut,
                       wref.data(), nn.data(), nl.data(), lcap, &sys);
  if (rc) return rc;
  if (has_rx) {
    rc = prx_set_reactions(sys, rxs, (uint32_t)has_rx);
    if (rc) {
      prx_destroy(sys);
      return rc;
    }
  }
  *out = sys;
  return PRX_OK;
}

// ---- analysis ---------------------------------------------------------------------

int prx_pair_histogram(prx_system* sys, const prx_class* a, const prx_class* b, double r_max,
                       uint32_t nbins, uint64_t* counts, uint64_t* n_a, uint64_t* n_b) {
  if (!sys || !a || !b || !counts || nbins < 1 || nbins > 2048) return PRX_EINVAL;
  if (!(r_max > 0.0) || r_max > sys->grid_rcut)
    return fail(sys, PRX_EINVAL, "r_max beyond the cutoff the Verlet lists guarantee");
  std::vector<double> e2(nbins + 1);
  for (uint32_t k = 0; k <= nbins; ++k) {
    const double e = r_max * (double)k / (double)nbins;
    e2[k] = e * e;
  }
  double* d_e2 = nullptr;
  unsigned long long* d_c = nullptr;
  CK(cudaMalloc(&d_e2, sizeof(double) * (nbins + 1)));
  if (cudaMalloc(&d_c, sizeof(unsigned long long) * (nbins + 2)) != cudaSuccess) {
    cudaFree(d_e2);
    return fail(sys, PRX_ENOMEM, "histogram buffers");
  }
  std::vector<unsigned long long> h(nbins + 2, 0ull);
  cudaError_t e = cudaMemcpyAsync(d_e2, e2.data(), sizeof(double) * (nbins + 1), cudaMemcpyHostToDevice,
                                  sys->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_c, 0, sizeof(unsigned long long) * (nbins + 2), sys->stream);
  if (e == cudaSuccess && sys->S.n) {
    launch_pair_hist(sys->S, sys->stream, PairClass{a->type_mask, a->s_lo, a->s_hi},
                     PairClass{b->type_mask, b->s_lo, b->s_hi}, d_e2, (int)nbins, d_c, d_c + nbins);
    sys->other_launches++;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), d_c, sizeof(unsigned long long) * (nbins + 2), cudaMemcpyDeviceToHost,
                        sys->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(sys->stream);
  cudaFree(d_e2);
  cudaFree(d_c);
  if (e != cudaSuccess) return fail(sys, PRX_ECUDA, std::string("pair histogram: ") + cudaGetErrorString(e));
  for (uint32_t k = 0; k < nbins; ++k) counts[k] = h[k];
  if (n_a) *n_a = h[nbins];
  if (n_b) *n_b = h[nbins + 1];
  return sync_status(sys);
}

// ---- autotuner -------------------------------------------------------------------

int prx_autotune_skin(const prx_system_desc* desc, const double* pos, const double* vel,
                      const uint8_t* type, const int8_t* state, const prx_reaction_desc* rx,
                      uint32_t steps, const double* skins, uint32_t n_skins, double* best_skin,
                      double* ms_per_step) {
  if (!desc || !skins || !n_skins || !best_skin || steps == 0) return PRX_EINVAL;
  double best = -1.0, best_ms = 0.0;
  for (uint32_t c = 0; c < n_skins; ++c) {
    if (ms_per_step) ms_per_step[c] = -1.0;
    prx_system_desc d = *desc;
    d.skin = skins[c];
    prx_system* sys = nullptr;
    if (prx_create(&d, pos, vel, type, state, nullptr, 0, nullptr, &sys) != PRX_OK) continue;
    bool ok = !rx || prx_set_reaction(sys, rx) == PRX_OK;
    cudaEvent_t a = nullptr, b = nullptr;
    float ms = 0.f;
    ok = ok && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
    ok = ok && prx_run(sys, steps / 4 + 1) == PRX_OK && prx_sync(sys) == PRX_OK;
    ok = ok && cudaEventRecord(a, sys->stream) == cudaSuccess;
    ok = ok && prx_run(sys, steps) == PRX_OK;
    ok = ok && cudaEventRecord(b, sys->stream) == cudaSuccess;
    ok = ok && prx_sync(sys) == PRX_OK && cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    prx_destroy(sys);
    if (!ok) continue;
    const double per = ms / steps;
    if (ms_per_step) ms_per_step[c] = per;
    if (best < 0.0 || per < best_ms) {
      best = skins[c];
      best_ms = per;
    }
  }
  if (best < 0.0) {
    g_create_error = "no candidate skin could be run";
    return PRX_EINVAL;
  }
  *best_skin = best;
  return PRX_OK;
}

int prx_set_launch_config(prx_system* sys, const prx_launch_config* cfg) {
  if (!sys || !cfg) return PRX_EINVAL;
  if (sys->batch) return refuse_member(sys);
  const uint32_t bt = cfg->step_threads ? cfg->step_threads : 256u;
  const uint32_t lanes = cfg->step_lanes ? cfg->step_lanes : 1u;
  if ((bt != 128u && bt != 256u && bt != 512u) || (lanes != 1u && lanes != 4u) ||
      cfg->chunk_intervals > 64u || cfg->step_blocks_per_sm > 32u)
    return fail(sys, PRX_EINVAL, "launch configuration out of range");
  if (sys->d.force_precision == PRX_FORCE_FP64 && (bt != 256u || lanes != 1u))
    return fail(sys, PRX_EINVAL, "the FP64 force mode has fixed kernels");
  CK(cudaStreamSynchronize(sys->stream));
  sys->S.step_bt = (int)bt;
  sys->S.step_lanes = (int)lanes;
  sys->S.step_bpsm = (int)cfg->step_blocks_per_sm;
  sys->chunk_m = cfg->chunk_intervals ? cfg->chunk_intervals : 1u;
  destroy_graphs(sys);
  return PRX_OK;
}

int prx_get_launch_config(prx_system* sys, prx_launch_config* cfg) {
  if (!sys || !cfg) return PRX_EINVAL;
  cfg->step_threads = (uint32_t)sys->S.step_bt;
  cfg->step_blocks_per_sm = (uint32_t)sys->S.step_bpsm;
  cfg->chunk_intervals = sys->chunk_m;
  cfg->step_lanes = (uint32_t)sys->S.step_lanes;
  return PRX_OK;
}

}  // extern "C"

namespace {

std::mutex g_tune_mu;
std::map<std::string, prx_tune_choice> g_tune_cache;

// The cache key: what the timing depends on.
std::string tune_key(const prx_system_desc& d, const prx_reaction_desc* rx, uint32_t steps,
                     const double* skins, uint32_t n_skins, const uint32_t* threads,
                     const uint32_t* bpsm, const uint32_t* lanes, uint32_t n_shapes,
                     const uint32_t* chunks, uint32_t n_chunks) {
  char buf[512];
  const double V = d.box[0] * d.box[1] * d.box[2];
  snprintf(buf, sizeof(buf), "n=%u rho=%.4f cap=%u fp64=%d gamma=%.3g rx=%d rr=%.4g theta=%u k=%.4g steps=%u|",
           d.n, d.n / V, d.adj_cap, d.force_precision, d.gamma, rx ? 1 : 0, rx ? rx->r_react : 0.0,
           rx ? rx->theta : 0u, rx ? rx->k : 0.0, steps);
  std::string k(buf);
  for (uint32_t q = 0; q < n_skins; ++q) k += std::to_string(skins[q]) + ",";
  k += "|";
  for (uint32_t q = 0; q < n_shapes; ++q)
    k += std::to_string(threads[q]) + "x" + std::to_string(bpsm[q]) + "x" + std::to_string(lanes[q]) + ",";
  k += "|";
  for (uint32_t q = 0; q < n_chunks; ++q) k += std::to_string(chunks[q]) + ",";
  for (char& c : k)
    if (c == '\t' || c == '\n') c = ' ';
  return k;
}

bool tune_file_lookup(const char* path, const std::string& key, prx_tune_choice* out) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[2048];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    char* tab = strchr(line, '\t');
    if (!tab) continue;
    *tab = 0;
    if (key != line) continue;
    prx_tune_choice c{};
    unsigned t = 0, b = 0, m = 0;
    unsigned l = 1;
    if (sscanf(tab + 1, "%lf %u %u %u %u %lf", &c.skin, &t, &b, &m, &l, &c.ms_per_step) == 6) {
      c.launch.step_threads = t;
      c.launch.step_blocks_per_sm = b;
      c.launch.chunk_intervals = m;
      c.launch.step_lanes = l;
      *out = c;
      found = true;  // the last line for a key wins
    }
  }
  fclose(f);
  return found;
}

void tune_file_store(const char* path, const std::string& key, const prx_tune_choice& c) {
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s\t%.17g %u %u %u %u %.9g\n", key.c_str(), c.skin, c.launch.step_threads,
          c.launch.step_blocks_per_sm, c.launch.chunk_intervals, c.launch.step_lanes, c.ms_per_step);
  fclose(f);
}

// Times one candidate on a temporary system: warm-up, then `steps` steps
// rounded up to whole graph chunks; -1 when it cannot run.
double time_candidate(const prx_system_desc* desc, const double* pos, const double* vel,
                      const uint8_t* type, const int8_t* state, const prx_reaction_desc* rx,
                      uint32_t steps, double skin, const prx_launch_config& lc) {
  prx_system_desc d = *desc;
  d.skin = skin;
  prx_system* sys = nullptr;
  if (prx_create(&d, pos, vel, type, state, nullptr, 0, nullptr, &sys) != PRX_OK) return -1.0;
  bool ok = !rx || prx_set_reaction(sys, rx) == PRX_OK;
  ok = ok && prx_set_launch_config(sys, &lc) == PRX_OK;
  const uint64_t chunk = (uint64_t)(rx ? rx->theta : kNoRxChunk) * (lc.chunk_intervals ? lc.chunk_intervals : 1u);
  const uint64_t n = (steps + chunk - 1) / chunk * chunk;
  cudaEvent_t a = nullptr, b = nullptr;
  float ms = 0.f;
  ok = ok && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
  ok = ok && prx_run(sys, n / 4 / chunk * chunk + chunk) == PRX_OK && prx_sync(sys) == PRX_OK;
  ok = ok && cudaEventRecord(a, sys->stream) == cudaSuccess;
  ok = ok && prx_run(sys, n) == PRX_OK;
  ok = ok && cudaEventRecord(b, sys->stream) == cudaSuccess;
  ok = ok && prx_sync(sys) == PRX_OK && cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  prx_destroy(sys);
  return ok ? (double)ms / (double)n : -1.0;
}

}  // namespace

extern "C" {

int prx_autotune(const prx_system_desc* desc, const double* pos, const double* vel,
                 const uint8_t* type, const int8_t* state, const prx_reaction_desc* rx,
                 uint32_t steps, const double* skins, uint32_t n_skins, const uint32_t* threads,
                 const uint32_t* blocks_per_sm, const uint32_t* lanes, uint32_t n_shapes,
                 const uint32_t* chunks, uint32_t n_chunks, const char* cache_path,
                 prx_tune_choice* best, prx_tune_choice* tried, uint32_t tried_cap,
                 uint32_t* n_tried) {
  if (n_tried) *n_tried = 0;
  if (!desc || !best || steps == 0 || (n_skins && !skins) ||
      (n_shapes && (!threads || !blocks_per_sm || !lanes)) || (n_chunks && !chunks))
    return PRX_EINVAL;
  const std::string key = tune_key(*desc, rx, steps, skins, n_skins, threads, blocks_per_sm, lanes,
                                   n_shapes, chunks, n_chunks);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    prx_tune_choice c{};
    if (it != g_tune_cache.end()) {
      c = it->second;
    } else if (cache_path && tune_file_lookup(cache_path, key, &c)) {
      g_tune_cache[key] = c;
    } else {
      c.ms_per_step = -2.0;
    }
    if (c.ms_per_step != -2.0) {
      *best = c;
      best->cached = 1u;
      best->stage = 2u;
      return PRX_OK;
    }
  }
  uint32_t nt = 0;
  auto record = [&](const prx_tune_choice& c) {
    if (tried && nt < tried_cap) tried[nt] = c;
    ++nt;
  };
  prx_tune_choice cur{};
  cur.skin = desc->skin;
  cur.launch.step_threads = 256u;
  cur.launch.chunk_intervals = 1u;
  cur.launch.step_lanes = 1u;
  cur.ms_per_step = -1.0;
  auto stage = [&](uint32_t st, uint32_t count, auto apply) {
    prx_tune_choice stage_best{};
    stage_best.ms_per_step = -1.0;
    for (uint32_t q = 0; q < count; ++q) {
      prx_tune_choice c = cur;
      apply(c, q);
      c.stage = st;
      c.cached = 0u;
      c.ms_per_step = time_candidate(desc, pos, vel, type, state, rx, steps, c.skin, c.launch);
      record(c);
      if (c.ms_per_step >= 0.0 && (stage_best.ms_per_step < 0.0 || c.ms_per_step < stage_best.ms_per_step))
        stage_best = c;
    }
    if (stage_best.ms_per_step >= 0.0) cur = stage_best;
  };
  stage(0u, n_skins, [&](prx_tune_choice& c, uint32_t q) { c.skin = skins[q]; });
  stage(1u, n_shapes, [&](prx_tune_choice& c, uint32_t q) {
    c.launch.step_threads = threads[q];
    c.launch.step_blocks_per_sm = blocks_per_sm[q];
    c.launch.step_lanes = lanes[q];
  });
  stage(2u, n_chunks, [&](prx_tune_choice& c, uint32_t q) { c.launch.chunk_intervals = chunks[q]; });
  if (n_tried) *n_tried = nt;
  if (cur.ms_per_step < 0.0) {
    g_create_error = "no autotuner candidate could run";
    return PRX_EINVAL;
  }
  *best = cur;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = cur;
    if (cache_path) tune_file_store(cache_path, key, cur);
  }
  return PRX_OK;
}

// ---- batched ensemble ---------------------------------------------------------

int prx_batch_create(uint32_t max_slots, uint64_t mem_budget, void* cuda_stream, prx_batch** out) {
  if (!out) return PRX_EINVAL;
  *out = nullptr;
  prx_batch* b = new (std::nothrow) prx_batch();
  if (!b) return PRX_ENOMEM;
  b->max_slots = max_slots;
  b->mem_budget = mem_budget;
  bool ok = true;
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess;
    b->own_stream = ok;
  }
  ok = ok && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaMalloc(&b->bctl, sizeof(BatchCtl)) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->bctl_host, sizeof(BatchCtl)) == cudaSuccess;
  ok = ok && cudaMemset(b->bctl, 0, sizeof(BatchCtl)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    g_create_error = "batch creation failed (stream or device memory)";
    prx_batch_destroy(b);
    return PRX_ECUDA;
  }
  *out = b;
  return PRX_OK;
}

void prx_batch_destroy(prx_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (prx_system* m : b->members) {
    m->stream = m->solo_stream;
    m->batch = nullptr;
  }
  for (prx_batch::Slot& sl : b->slots) {
    if (sl.sys) {
      sl.sys->slot = -1;
      sl.sys->slot_batch = nullptr;
    }
    if (sl.done) cudaEventDestroy(sl.done);
  }
  for (cudaEvent_t e : b->inflight) cudaEventDestroy(e);
  for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
  for (prx_batch::Stage& sg : b->stage) {
    if (sg.host) cudaFreeHost(sg.host);
    if (sg.used) cudaEventDestroy(sg.used);
  }
  batch_destroy_graphs(b);
  if (b->T) cudaFree(b->T);
  if (b->maps) cudaFree(b->maps);
  if (b->act_n) cudaFree(b->act_n);
  if (b->bctl) cudaFree(b->bctl);
  if (b->bctl_host) cudaFreeHost(b->bctl_host);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"

namespace {

// The conditions prx_batch_add and prx_batch_admit share.
int check_member(prx_batch* b, prx_system* sys) {
  if (sys->batch || sys->slot_batch) return bfail(b, PRX_EINVAL, "system is already a member of a batch");
  if (sys->d.force_precision != PRX_FORCE_FP32)
    return bfail(b, PRX_EINVAL, "batches run PRX_FORCE_FP32 systems only");
  if (sys->profiling) return bfail(b, PRX_EINVAL, "system is being profiled");
  if (sys->S.step_lanes != 1)
    return bfail(b, PRX_EINVAL, "batch members run the one-lane step kernel (step_lanes 1)");
  if (sys->has_rx) {
    const uint64_t th = sys->rxd.theta;
    if (b->theta && th != b->theta)
      return bfail(b, PRX_EINVAL, "reaction interval differs from the batch's");
    if (b->theta && sys->host_step % th != b->phase)
      return bfail(b, PRX_EINVAL, "system is at another point of the reaction cycle");
  }
  return PRX_OK;
}

void join(prx_batch* b, prx_system* sys) {
  if (sys->has_rx && !b->theta) {
    b->theta = sys->rxd.theta;
    b->phase = sys->host_step % b->theta;
  }
  sys->solo_stream = sys->stream;
  sys->stream = b->stream;
  sys->batch = b;
  b->members.push_back(sys);
  b->valid = false;
}

// Takes a member out of the batch without waiting: its own stream waits for
// the work queued on the batch's stream so far, and further calls on the
// system go to its own stream.
int leave(prx_batch* b, prx_system* sys) {
  if (!sys->join_ev && cudaEventCreateWithFlags(&sys->join_ev, cudaEventDisableTiming) != cudaSuccess)
    return bfail(b, PRX_ECUDA, "event creation failed");
  CKB(cudaEventRecord(sys->join_ev, b->stream));
  CKB(cudaStreamWaitEvent(sys->solo_stream, sys->join_ev, 0));
  b->members.erase(std::find(b->members.begin(), b->members.end(), sys));
  sys->stream = sys->solo_stream;
  sys->batch = nullptr;
  b->valid = false;
  bool rx = false;
  for (prx_system* m : b->members) rx = rx || m->has_rx;
  if (!rx) b->theta = 0, b->phase = 0;
  return PRX_OK;
}

// Releases an admission slot (after poll, removal or destruction).
void free_slot(prx_batch* b, prx_system* sys) {
  if (sys->slot < 0 || sys->slot_batch != b) return;
  prx_batch::Slot& sl = b->slots[(size_t)sys->slot];
  b->bytes_in_use -= sl.bytes;
  if (sl.done) cudaEventDestroy(sl.done);
  sl = prx_batch::Slot{};
  sys->slot = -1;
  sys->slot_batch = nullptr;
}

// Takes a slot for sys (PRX_ENOMEM when none is free or the budget is spent).
int take_slot(prx_batch* b, prx_system* sys, uint64_t bytes, bool targeted, uint64_t nsteps) {
  if (b->mem_budget && b->bytes_in_use + bytes > b->mem_budget)
    return bfail(b, PRX_ENOMEM, "memory budget: " + std::to_string(b->bytes_in_use) + " + " +
                                    std::to_string(bytes) + " > " + std::to_string(b->mem_budget) + " bytes");
  size_t q = 0;
  while (q < b->slots.size() && b->slots[q].sys) ++q;
  if (b->max_slots && q >= b->max_slots) return bfail(b, PRX_ENOMEM, "no free slot");
  if (q == b->slots.size()) b->slots.emplace_back();
  prx_batch::Slot& sl = b->slots[q];
  if (cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
    return bfail(b, PRX_ECUDA, "event creation failed");
  sl.sys = sys;
  sl.bytes = bytes;
  sl.targeted = targeted;
  sl.left = nsteps;
  b->bytes_in_use += bytes;
  sys->slot = (int32_t)q;
  sys->slot_batch = b;
  return PRX_OK;
}

bool has_targets(const prx_batch* b) {
  for (const prx_batch::Slot& sl : b->slots)
    if (sl.sys && sl.targeted && !sl.finishing) return true;
  return false;
}

// Queues nsteps steps of every member (graph replays on the batch stream).
int batch_launch(prx_batch* b, uint64_t nsteps) {
  int rc = batch_prepare(b);
  if (rc) return rc;
  const uint64_t total = nsteps;
  if (b->n_active && b->dg_ok && nsteps) {
    // one device-driven chain (dg.cu) behind one host launch
    const uint64_t theta = b->any_rx ? b->theta : 0;
    const uint64_t ph = b->any_rx ? b->phase : 0;
    launch_dgb_arm(b->bctl, b->stream, nsteps, ph, theta, b->any_rx ? 1 : 0,
                   (unsigned long long)b->dg_rebuild, (unsigned long long)b->dg_react);
    const cudaError_t e = cudaGraphLaunch(b->dg_step, b->stream);
    if (e != cudaSuccess) return bfail(b, PRX_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    b->graph_launches++;
    if (b->any_rx) b->rx_runs += (ph + nsteps) / theta;
    nsteps = 0;
  }
  if (b->n_active) {
    const uint64_t theta = b->any_rx ? b->theta : (uint64_t)kNoRxChunk;
    uint64_t ph = b->any_rx ? b->phase : 0;
    while (nsteps > 0) {
      cudaError_t e;
      if (ph == 0 && nsteps >= theta) {
        e = cudaGraphLaunch(b->g_chunk, b->stream);
        nsteps -= theta;
        if (b->any_rx) b->rx_runs++;
      } else {
        e = cudaGraphLaunch(b->g_step, b->stream);
        nsteps--;
        ph = (ph + 1) % theta;
        if (b->any_rx && ph == 0 && e == cudaSuccess) {
          e = cudaGraphLaunch(b->g_react, b->stream);
          b->graph_launches++;
          b->rx_runs++;
        }
      }
      if (e != cudaSuccess) return bfail(b, PRX_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
      b->graph_launches++;
    }
  }
  b->steps += total;
  if (b->theta) b->phase = (b->phase + total) % b->theta;
  if (b->n_active) {
    b->kernel_steps += total * (uint64_t)b->n_step_variants;
    if (b->dg_ok && total) b->kernel_steps += total + 1;  // k_dgb_next per step, the arm kernel
  }
  for (prx_system* m : b->members) m->host_step += total;
  return PRX_OK;
}

}  // namespace

extern "C" {

int prx_batch_add(prx_batch* b, prx_system* sys) {
  if (!b || !sys) return PRX_EINVAL;
  int rc = check_member(b, sys);
  if (rc) return rc;
  if (cudaStreamSynchronize(sys->stream) != cudaSuccess)
    return bfail(b, PRX_ECUDA, "synchronising the system's stream failed");
  if (b->max_slots || b->mem_budget) {
    if ((rc = take_slot(b, sys, estimate_bytes(sys->d, max_r_react(sys)), false, 0)))
      return rc;
  }
  join(b, sys);
  return PRX_OK;
}

int prx_batch_admit(prx_batch* b, prx_system* sys, uint64_t nsteps, int32_t* slot) {
  if (!b || !sys || !slot) return PRX_EINVAL;
  *slot = -1;
  int rc = check_member(b, sys);
  if (rc) return rc;
  if ((rc = take_slot(b, sys, estimate_bytes(sys->d, max_r_react(sys)), true, nsteps)))
    return rc;
  // the system's queued work (creation, earlier runs) comes before the batch's
  if (!sys->join_ev && cudaEventCreateWithFlags(&sys->join_ev, cudaEventDisableTiming) != cudaSuccess) {
    free_slot(b, sys);
    return bfail(b, PRX_ECUDA, "event creation failed");
  }
  if (cudaEventRecord(sys->join_ev, sys->stream) != cudaSuccess ||
      cudaStreamWaitEvent(b->stream, sys->join_ev, 0) != cudaSuccess) {
    free_slot(b, sys);
    return bfail(b, PRX_ECUDA, "ordering the system before the batch failed");
  }
  *slot = sys->slot;
  join(b, sys);
  return PRX_OK;
}

int prx_batch_remove(prx_batch* b, prx_system* sys) {
  if (!b || !sys || sys->batch != b) return PRX_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess)
    return bfail(b, PRX_ECUDA, "synchronising the batch stream failed");
  b->members.erase(std::find(b->members.begin(), b->members.end(), sys));
  sys->stream = sys->solo_stream;
  sys->batch = nullptr;
  b->valid = false;
  free_slot(b, sys);
  bool rx = false;
  for (prx_system* m : b->members) rx = rx || m->has_rx;
  if (!rx) b->theta = 0, b->phase = 0;
  return PRX_OK;
}

int prx_batch_run(prx_batch* b, uint64_t nsteps) {
  if (!b) return PRX_EINVAL;
  if (has_targets(b))
    return bfail(b, PRX_EINVAL, "members admitted with step targets advance by prx_batch_step_epoch");
  return batch_launch(b, nsteps);
}

int prx_batch_step_epoch(prx_batch* b, uint64_t max_steps, uint64_t* steps_run) {
  if (steps_run) *steps_run = 0;
  if (!b) return PRX_EINVAL;
  int rc;
  // flow control: at most two earlier epochs queued on the device
  while (!b->inflight.empty()) {
    cudaError_t q = cudaEventQuery(b->inflight.front());
    if (q == cudaErrorNotReady) {
      if (b->inflight.size() < 2) break;
      q = cudaEventSynchronize(b->inflight.front());
    }
    if (q != cudaSuccess) return bfail(b, PRX_ECUDA, std::string("epoch wait: ") + cudaGetErrorString(q));
    b->ev_pool.push_back(b->inflight.front());
    b->inflight.erase(b->inflight.begin());
  }
  const uint64_t chunk = b->theta ? b->theta : (uint64_t)kNoRxChunk;
  // 1. members with less than a chunk left finish alone, after the batch's queued work
  for (prx_batch::Slot& sl : b->slots) {
    if (!sl.sys || !sl.targeted || sl.finishing || sl.left >= chunk) continue;
    prx_system* m = sl.sys;
    if ((rc = leave(b, m))) return rc;
    if (sl.left && (rc = prx_run(m, sl.left))) return bfail(b, rc, "running a member's last steps: " + m->err);
    sl.left = 0;
    sl.finishing = true;
    CKB(cudaEventRecord(sl.done, m->stream));
  }
  // 2. the epoch
  uint64_t E = max_steps;
  for (const prx_batch::Slot& sl : b->slots)
    if (sl.sys && sl.targeted && !sl.finishing) E = std::min(E, sl.left);
  const uint64_t ch = b->theta ? b->theta : (uint64_t)kNoRxChunk;
  if (E >= ch) E -= E % ch;
  if (b->members.empty()) E = 0;
  if (E) {
    if ((rc = batch_launch(b, E))) return rc;
    b->epochs++;
    for (prx_batch::Slot& sl : b->slots)
      if (sl.sys && sl.targeted && !sl.finishing) sl.left -= E;
    cudaEvent_t ev = nullptr;
    if (!b->ev_pool.empty()) {
      ev = b->ev_pool.back();
      b->ev_pool.pop_back();
    } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      return bfail(b, PRX_ECUDA, "event creation failed");
    }
    CKB(cudaEventRecord(ev, b->stream));
    b->inflight.push_back(ev);
  }
  // 3. members whose steps are done leave; they complete with this epoch
  for (prx_batch::Slot& sl : b->slots) {
    if (!sl.sys || !sl.targeted || sl.finishing || sl.left) continue;
    if ((rc = leave(b, sl.sys))) return rc;
    sl.finishing = true;
    CKB(cudaEventRecord(sl.done, sl.sys->stream));
  }
  if (steps_run) *steps_run = E;
  return PRX_OK;
}

int prx_batch_poll(prx_batch* b, int32_t* done_slots, int32_t cap, int32_t* n_done) {
  if (!b || !n_done || cap < 0 || (cap && !done_slots)) return PRX_EINVAL;
  *n_done = 0;
  for (size_t q = 0; q < b->slots.size() && *n_done < cap; ++q) {
    prx_batch::Slot& sl = b->slots[q];
    if (!sl.sys || !sl.finishing) continue;
    const cudaError_t e = cudaEventQuery(sl.done);
    if (e == cudaErrorNotReady) continue;
    if (e != cudaSuccess) return bfail(b, PRX_ECUDA, std::string("poll: ") + cudaGetErrorString(e));
    done_slots[(*n_done)++] = (int32_t)q;
    free_slot(b, sl.sys);
  }
  return PRX_OK;
}

int prx_batch_sync(prx_batch* b, int32_t* failed) {
  if (failed) *failed = -1;
  if (!b) return PRX_EINVAL;
  for (prx_system* m : b->members)
    if (cudaMemcpyAsync(m->ctl_host, m->S.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
      return bfail(b, PRX_ECUDA, "reading a member's control block failed");
  if (b->dg_ok &&
      cudaMemcpyAsync(b->bctl_host, b->bctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
    return bfail(b, PRX_ECUDA, "reading the batch's control block failed");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, PRX_ECUDA, std::string("batch stream: ") + cudaGetErrorString(e));
  if (b->dg_ok && b->bctl_host->dg_err) return bfail(b, PRX_ECUDA, "a device-side graph launch failed");
  for (size_t q = 0; q < b->members.size(); ++q) {
    const int st = b->members[q]->ctl_host->status;
    if (st) {
      if (failed) *failed = (int32_t)q;
      b->members[q]->err = std::string("device reported ") + prx_status_string(st);
      return bfail(b, st, "member " + std::to_string(q) + ": device reported " + prx_status_string(st));
    }
  }
  return PRX_OK;
}

int prx_batch_stats_get(prx_batch* b, prx_batch_stats* out) {
  if (!b || !out) return PRX_EINVAL;
  memset(out, 0, sizeof(*out));
  cudaError_t e = cudaMemcpyAsync(b->bctl_host, b->bctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, PRX_ECUDA, std::string("batch stream: ") + cudaGetErrorString(e));
  out->members = (uint32_t)b->members.size();
  for (prx_system* m : b->members) {
    out->particles += m->S.n;
    if (m->S.n) out->active++;
  }
  out->steps = b->steps;
  out->rebuilds = b->bctl_host->rebuilds;
  out->reactions = b->rx_runs;
  out->kernel_launches = b->kernel_steps + out->rebuilds * (uint64_t)batch_rebuild_kernel_count() +
                         b->rx_runs * (uint64_t)batch_rx_kernel_count();
  out->graph_launches = b->graph_launches;
  out->max_slots = b->max_slots;
  out->mem_budget = b->mem_budget;
  out->bytes_admitted = b->bytes_in_use;
  for (const prx_batch::Slot& sl : b->slots) out->slots_used += sl.sys ? 1u : 0u;
  out->epochs = b->epochs;
  return PRX_OK;
}

const char* prx_batch_last_error(const prx_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
