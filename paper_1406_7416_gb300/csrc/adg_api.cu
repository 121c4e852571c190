// C ABI of libadg (declared in include/adg.h): state management, device
// memory, host <-> device transfers and the order of the kernel launches of
// one time step.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "adg_internal.h"

using namespace adg;

struct adg_state {
  Geo geo;
  int N = 0, dim = 0, nv = 0, prec = 0;
  double gamma = 1.4, eps = 1e-3, floor = 1e-4;
  int force = 0, iters = 0, fp64_sweeps = 1;
  int cascade = 1;          // first-order layer after WENO3
  int flux = ADG_FLUX_RUSANOV;
  bool host_passes = false; // true: the host waits for the troubled count and launches
                            // the passes; false: one CUDA graph per step, passes sized
                            // on the device by a conditional loop
  int sub_fp64 = 0;         // mixed precision: FP64 sweeps of the degree-2 subcell predictor
  int sub_f32 = 1;          // mixed precision: FP32 subcell reconstruction and sub-face fluxes
  int sub_reg = 1;          // FP32 subcell predictor: register form (1) or shared-memory form (0)
  int project_delta = 1;    // mixed precision: detector projection from the kept P(u^n)
  int pred_opt = -1;        // ADG_OPT_PREDICTOR: fixed predictor shape (PRED_*); -1 autotune
                            // among the shapes of the default arithmetic, -2 among all
  int pred_tuned = -1;      // the autotuner's choice (-1: not tuned yet)
  double tune_ms[PRED_COUNT] = {};   // the autotuner's per-shape milliseconds (NaN: n/a)
  int bstate_set = 0;       // bit f: inflow face f has a state
  int front_set = 0;        // bit f: front face f has its front
  // pinned host mirror of the device Params, counters and dt, read once per
  // step after the DG phase when host_passes is on
  struct Probe {
    Params p;
    int counters[CNT_COUNT];
    double dt;
  };
  Probe* probe = nullptr;
  long long launch_count = 0;       // kernels issued by steps (batched: on each group's first state)
  long long cap_req = -1;
  int cap = 0, chunk = 0;
  void* (*alloc)(size_t, void*) = nullptr;
  void (*freef)(void*, void*) = nullptr;
  void* actx = nullptr;
  cudaStream_t stream = 0;
  Ops ops_host;
  Ops* ops_dev = nullptr;
  Bufs b;
  bool allocated = false, loaded = false;
  int cur = 0;
  int stamp = 0;
  std::vector<void*> owned;
  size_t bytes_held = 0;
  std::string err;
  bool profile = false;
  bool lam_mode = false;    // steps keep the per-cell wave speeds current
  bool lam_valid = false;   // b.lam describes the current level
  // device copy of the Params: during steps the device owns cur and stamp
  Params* dparams = nullptr;
  Params** d_pps1 = nullptr;        // [1] = dparams
  long long* d_pre1 = nullptr;      // cells[2], faces[3][2], fix[2], fb[2], refix[2], lim[2 + 2]
  double* d_dts1 = nullptr;         // [1]
  bool params_dirty = true;         // host fields changed since the last upload
  bool cur_known = true;            // host cur / stamp equal the device's
  double t_end = 0.0;               // end time of the simulated interval (0: none)
  double cfl = 0.0;                 // CFL number of batched CFL steps with cfl <= 0
  size_t scratch_budget = 0;        // bytes of limiter scratch (0: from free memory at allocation)
  Params hparams;                   // source of the last upload
  // phase events of profiled steps: a ring of kEventSets sets used in turn, so
  // that the host runs up to kEventSets - 1 steps ahead of the device; a set
  // is read when it comes round again (or by adg_phase_times)
  static constexpr int kEventSets = 3;
  cudaEvent_t ev[kEventSets][PHASE_COUNT] = {};
  bool pending[kEventSets] = {};
  int ev_next = 0;
  double phase_ms[PHASE_COUNT] = {};
  int timed_steps = 0;
  // the step graph (host_passes off): captured on cap_stream (the limiter
  // pass body on body_stream), replayed on `stream` while `gsl` is unchanged
  // one graph per event set when profiling (the event nodes differ), else slot 0
  cudaGraph_t graph[kEventSets] = {};
  cudaGraphExec_t gexec[kEventSets] = {};
  StepLaunch gsl[kEventSets];
  cudaStream_t cap_stream = nullptr, body_stream = nullptr;
};

namespace {

int fail(adg_state* st, int code, const std::string& msg) {
  if (st) st->err = msg;
  return code;
}

#define CUDA_TRY(st, call)                                                              \
  do {                                                                                  \
    cudaError_t _e = (call);                                                            \
    if (_e != cudaSuccess)                                                              \
      return fail(st, ADG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

void* dev_alloc(adg_state* st, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (st->alloc) {
    p = st->alloc(bytes, st->actx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    st->owned.push_back(p);
    st->bytes_held += bytes;
  }
  return p;
}

void dev_free(adg_state* st, void* p) {
  if (!p) return;
  if (st->freef) st->freef(p, st->actx);
  else cudaFree(p);
}

void drop_graph(adg_state* st, int slot) {
  if (st->gexec[slot]) cudaGraphExecDestroy(st->gexec[slot]);
  if (st->graph[slot]) cudaGraphDestroy(st->graph[slot]);
  st->gexec[slot] = nullptr;
  st->graph[slot] = nullptr;
}

void free_all(adg_state* st) {
  if (st->stream) cudaStreamSynchronize(st->stream);
  else cudaDeviceSynchronize();
  for (int k = 0; k < adg_state::kEventSets; ++k) drop_graph(st, k);
  if (st->probe) cudaFreeHost(st->probe);
  st->probe = nullptr;
  for (void* p : st->owned) dev_free(st, p);
  st->owned.clear();
  st->bytes_held = 0;
  st->allocated = false;
  st->loaded = false;
}

int nodes_per_cell(const adg_state* st) {
  int r = 1;
  for (int k = 0; k < st->dim; ++k) r *= st->N + 1;
  return r;
}
int subcells_per_cell(const adg_state* st) {
  int r = 1;
  for (int k = 0; k < st->dim; ++k) r *= 2 * st->N + 1;
  return r;
}

Params make_params(const adg_state* st) {
  Params p;
  p.geo = st->geo;
  p.N = st->N;
  p.dim = st->dim;
  p.nv = st->nv;
  p.prec = st->prec;
  p.iters = st->iters;
  p.force = st->force;
  p.cap = st->cap;
  p.chunk = st->chunk;
  p.gamma = st->gamma;
  p.gam2f = (float)(st->gamma * (st->gamma - 1.0));
  p.eps = st->eps;
  p.floor = st->floor;
  p.ops = st->ops_dev;
  p.b = st->b;
  p.cur = st->cur;
  p.stamp = st->stamp;
  p.lam_mode = st->lam_mode ? 1 : 0;
  p.fp64_sweeps = st->fp64_sweeps < st->iters ? st->fp64_sweeps : st->iters;
  p.cfl = st->cfl;
  p.cascade = st->cascade;
  p.flux = st->flux;
  return p;
}

cudaError_t dispatch(const adg_state* st, LaunchArgs& a) {
  if (st->dim == 2) return st->N <= 5 ? dispatch_2d_lo(st->N, a) : dispatch_2d_hi(st->N, a);
  return dispatch_3d(st->N, a);
}

int refresh(adg_state* st);

int launch(adg_state* st, LaunchArgs& a, const char* what) {
  int rc = refresh(st);
  if (rc) return rc;
  Params p = make_params(st);
  a.p = &p;
  a.stream = st->stream;
  cudaError_t e = dispatch(st, a);
  if (e != cudaSuccess) return fail(st, ADG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return ADG_OK;
}

#define ALLOC(ptr, type, count)                                                          \
  do {                                                                                   \
    ptr = (type*)dev_alloc(st, sizeof(type) * (size_t)(count));                          \
    if (!ptr) {                                                                          \
      free_all(st);                                                                      \
      return fail(st, ADG_ERR_OOM, "device allocation of " #ptr " failed");             \
    }                                                                                    \
  } while (0)

int ensure_allocated(adg_state* st) {
  if (st->allocated) return ADG_OK;
  {
    // the FP32 Picard operators of this degree, in the launching unit's constant memory
    const cudaError_t e = st->dim == 3 ? upload_constants_3d(st->N, st->ops_host)
                          : st->N <= 5 ? upload_constants_2d_lo(st->N, st->ops_host)
                                       : upload_constants_2d_hi(st->N, st->ops_host);
    if (e != cudaSuccess) return fail(st, ADG_ERR_CUDA, std::string("operator upload: ") + cudaGetErrorString(e));
  }
  const long long cells = st->geo.cells;
  const int nv = st->nv, nd = nodes_per_cell(st), nsd = subcells_per_cell(st);
  const int n = st->N + 1, Ns = 2 * st->N + 1;
  int nf = 1, nsf = 1;
  for (int k = 0; k < st->dim - 1; ++k) {
    nf *= n;
    nsf *= Ns;
  }
  long long cap = st->cap_req;
  if (cap <= 0) {
    // a slot for every cell when the two subcell stores fit in 8 GiB,
    // otherwise for a quarter of the cells
    const double store_bytes = 2.0 * (double)cells * nv * nsd * sizeof(double);
    cap = store_bytes <= 8.0 * (1 << 30) ? cells : cells / 4;
    if (cap < 4096) cap = 4096;
  }
  if (cap > cells) cap = cells;
  st->cap = (int)cap;
  size_t parts[6];
  const size_t per = limiter_scratch_doubles(st->dim, st->N, &parts[0], &parts[1], &parts[2],
                                             &parts[3], &parts[4], &parts[5]);
  // limiter scratch: room for a quarter of the cells (at least 256) per pass,
  // within the state's scratch budget (default 2 GiB)
  size_t budget = st->scratch_budget;
  if (budget == 0) {
    // an eighth of the free device memory, between 2 and 32 GiB: a 3D troubled
    // cell needs ~4 MB of scratch at N = 3, so a fixed small budget would cut
    // the limiter into many passes of a few hundred cells each
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = 0;
    }
    budget = free_b / 8;
    if (budget < ((size_t)2 << 30)) budget = (size_t)2 << 30;
    if (budget > ((size_t)32 << 30)) budget = (size_t)32 << 30;
  }
  long long chunk = (long long)(budget / (per * sizeof(double)));
  long long want = cells / 4;
  if (want < 256) want = 256;
  if (chunk > want) chunk = want;
  if (chunk < 1) chunk = 1;
  if (chunk > cap) chunk = cap;
  st->chunk = (int)chunk;

  Bufs& b = st->b;
  std::memset(&b, 0, sizeof(Bufs));
  for (int i = 0; i < 2; ++i) {
    ALLOC(b.U[i], double, cells * nv * nd);
    ALLOC(b.beta[i], uint8_t, cells);
    ALLOC(b.cmm[i], double, cells * nv * 2);
    ALLOC(b.slot[i], int, cells);
    ALLOC(b.list[i], int, cap);
    ALLOC(b.store[i], double, cap * nv * nsd);
  }
  ALLOC(b.trace, double, cells * st->dim * 2 * nv * nf * n);
  if (st->prec == ADG_PREC_MIXED_FP32 && st->project_delta) {
    ALLOC(b.vstar, double, cells * nv * nsd);
    ALLOC(b.vok, uint8_t, cells);
  }
  for (int k = 0; k < st->dim; ++k) {
    long long faces = 1;
    for (int j = 0; j < st->dim; ++j) faces *= (j == k) ? st->geo.n[j] + 1 : st->geo.n[j];
    ALLOC(b.G[k], double, faces * nv * nf);
  }
  ALLOC(b.lam, double, cells);
  ALLOC(b.counters, int, CNT_COUNT);
  ALLOC(b.fixlist, int, cells);
  ALLOC(b.fixstamp, int, cells);
  ALLOC(b.edge, double, cap * st->dim * 2 * nv * nsf);
  ALLOC(b.hist, int, HIST_LEN);
  ALLOC(b.fblist, int, 3 * cap);
  b.fbflag = b.fblist + cap;
  b.refixlist = b.fblist + 2 * cap;
  ALLOC(b.dt, double, 16);
  ALLOC(b.lamkey, long long, 1);
  b.lamred = b.dt + 1;
  b.clock = b.dt + 2;
  b.tstart = b.dt + 5;
  b.coef = b.dt + 6;
  b.coef_f = reinterpret_cast<float*>(b.dt + 12);
  ALLOC(st->dparams, Params, 1);
  ALLOC(st->d_pps1, Params*, 1);
  ALLOC(st->d_pre1, long long, 20);
  ALLOC(st->d_dts1, double, 1);
  ALLOC(b.patch, double, chunk * parts[0]);
  ALLOC(b.sweep[0], double, chunk * parts[1]);
  ALLOC(b.sweep[1], double, chunk * parts[2]);
  if (st->dim == 3) ALLOC(b.sweep[2], double, chunk * parts[3]);
  ALLOC(b.qsub, double, chunk * parts[4]);
  for (int k = 0; k < st->dim; ++k) ALLOC(b.fsub[k], double, chunk * parts[5]);
  ALLOC(st->ops_dev, Ops, 1);
  CUDA_TRY(st, cudaMemcpyAsync(st->ops_dev, &st->ops_host, sizeof(Ops), cudaMemcpyHostToDevice,
                               st->stream));
  CUDA_TRY(st, cudaMemsetAsync(b.counters, 0, sizeof(int) * CNT_COUNT, st->stream));
  CUDA_TRY(st, cudaMemsetAsync(b.fixstamp, 0xff, sizeof(int) * cells, st->stream));
  CUDA_TRY(st, cudaMemsetAsync(b.fbflag, 0xff, sizeof(int) * cap, st->stream));
  CUDA_TRY(st, cudaMemsetAsync(b.dt, 0, sizeof(double) * 12, st->stream));
  CUDA_TRY(st, cudaMemsetAsync(b.lamkey, 0, sizeof(long long), st->stream));
  {
    long long pre[20] = {0, cells, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < st->dim; ++k) {
      long long faces = 1;
      for (int j = 0; j < st->dim; ++j) faces *= (j == k) ? st->geo.n[j] + 1 : st->geo.n[j];
      pre[2 + 2 * k + 1] = faces * nf;
    }
    CUDA_TRY(st, cudaMemcpy(st->d_pre1, pre, sizeof(pre), cudaMemcpyHostToDevice));
    Params* pp = st->dparams;
    CUDA_TRY(st, cudaMemcpy(st->d_pps1, &pp, sizeof(Params*), cudaMemcpyHostToDevice));
  }
  st->allocated = true;
  st->params_dirty = true;
  st->cur_known = true;
  return ADG_OK;
}

int sync(adg_state* st) {
  CUDA_TRY(st, cudaStreamSynchronize(st->stream));
  return ADG_OK;
}

// Bring the host's cur / stamp up to date with the device Params.
int refresh(adg_state* st) {
  if (st->cur_known || !st->allocated) return ADG_OK;
  Params p;
  CUDA_TRY(st, cudaMemcpyAsync(&p, st->dparams, sizeof(Params), cudaMemcpyDeviceToHost, st->stream));
  CUDA_TRY(st, cudaStreamSynchronize(st->stream));
  st->cur = p.cur;
  st->stamp = p.stamp;
  st->cur_known = true;
  return ADG_OK;
}

// Upload the host Params (after a refresh, so device cur / stamp survive).
int upload_params(adg_state* st) {
  int rc = refresh(st);
  if (rc) return rc;
  st->hparams = make_params(st);
  CUDA_TRY(st, cudaMemcpyAsync(st->dparams, &st->hparams, sizeof(Params), cudaMemcpyHostToDevice,
                               st->stream));
  CUDA_TRY(st, cudaStreamSynchronize(st->stream));
  st->params_dirty = false;
  return ADG_OK;
}

// Reset the current level's counters and the clock before a load
int begin_load(adg_state* st) {
  for (int f = 0; f < 2 * st->dim; ++f) {
    if (st->geo.bc[f] == ADG_BC_INFLOW && !(st->bstate_set & (1 << f)))
      return fail(st, ADG_ERR_ARG, "inflow face " + std::to_string(f) +
                                       " has no state (adg_set_boundary_state)");
    if (st->geo.bc[f] == ADG_BC_FRONT && !(st->front_set & (1 << f)))
      return fail(st, ADG_ERR_ARG, "front face " + std::to_string(f) +
                                       " has no front (adg_set_boundary_front)");
  }
  int rc = ensure_allocated(st);
  if (rc) return rc;
  rc = refresh(st);
  if (rc) return rc;
  st->cur = 0;
  st->params_dirty = true;
  // every counter but the cumulative pass count (adg_info's launch count)
  CUDA_TRY(st, cudaMemsetAsync(st->b.counters, 0, sizeof(int) * CNT_PASSES, st->stream));
  if (st->b.vok) CUDA_TRY(st, cudaMemsetAsync(st->b.vok, 0, st->geo.cells, st->stream));
  const double clk[3] = {0.0, st->t_end, 0.0};
  CUDA_TRY(st, cudaMemcpyAsync(st->b.clock, clk, sizeof(clk), cudaMemcpyHostToDevice, st->stream));
  CUDA_TRY(st, cudaStreamSynchronize(st->stream));
  return ADG_OK;
}

// Temporary device buffer outside the state's owned list
struct Temp {
  adg_state* st;
  void* p = nullptr;
  Temp(adg_state* s, size_t bytes) : st(s) {
    p = dev_alloc(s, bytes);
    if (p) {
      s->owned.pop_back();
      s->bytes_held -= bytes == 0 ? 16 : bytes;
    }
  }
  ~Temp() {
    if (p) {
      cudaStreamSynchronize(st->stream);
      dev_free(st, p);
    }
  }
};

int load_detect(adg_state* st, const double* exact_dev);

}  // namespace
namespace {

int load_detect(adg_state* st, const double* exact_dev) {
  Temp tc(st, exact_dev ? sizeof(double) * st->geo.cells * st->nv * 2 : 16);
  double* cmm_ex = exact_dev ? (double*)tc.p : nullptr;
  if (exact_dev) {
    if (!cmm_ex) return fail(st, ADG_ERR_OOM, "allocation of the initial bounds failed");
    LaunchArgs m{};
    m.op = OP_SUB_MINMAX;
    m.sub = exact_dev;
    m.out = cmm_ex;
    int rc = launch(st, m, "initial bounds");
    if (rc) return rc;
  }
  LaunchArgs a{};
  a.op = OP_LOAD_DETECT;
  a.exact = exact_dev;
  a.cmm_ex = cmm_ex;
  int rc = launch(st, a, "initial detection");
  if (rc) return rc;
  rc = sync(st);
  if (rc) return rc;
  int status = 0;
  CUDA_TRY(st, cudaMemcpy(&status, st->b.counters + CNT_STATUS, sizeof(int), cudaMemcpyDeviceToHost));
  if (status & 1) return fail(st, ADG_ERR_CAPACITY, "more flagged cells than subcell slots");
  st->loaded = true;
  st->lam_valid = true;
  return ADG_OK;
}

// Fold the events of the profiled step recorded in set k into the sums.
int collect_phases(adg_state* st, int k) {
  if (!st->pending[k]) return ADG_OK;
  CUDA_TRY(st, cudaEventSynchronize(st->ev[k][PHASE_END]));
  for (int i = 0; i < PHASE_END; ++i) {
    float ms = 0.f;
    CUDA_TRY(st, cudaEventElapsedTime(&ms, st->ev[k][i], st->ev[k][i + 1]));
    st->phase_ms[i] += ms;
  }
  st->timed_steps += 1;
  st->pending[k] = false;
  return ADG_OK;
}

// Whether the state's predictor runs the split final stage (mixed precision
// with no FP64 sweep) at a degree the warp-per-cell kernel covers.
bool split_capable(const adg_state* st) {
  const int f64 = st->fp64_sweeps < st->iters ? st->fp64_sweeps : st->iters;
  return st->prec == ADG_PREC_MIXED_FP32 && f64 == 0 && st->iters > 0 &&
         !(st->dim == 2 && st->N >= 6);
}

// Predictor shapes that apply to the state (PRED_*).
bool shape_applies(const adg_state* st, int shape) {
  if (shape == PRED_BLOCK || shape == PRED_BLOCK_ALT) return true;
  return st->prec == ADG_PREC_MIXED_FP32 && split_capable(st) &&
         (shape == PRED_WARP1 || shape == PRED_WARP2 || shape == PRED_WARP4 ||
          shape == PRED_WARP4_TC);
}

// Shapes whose outputs are bit for bit those of the default shape: the
// block-per-cell kernel at either width (FP64, and mixed precision with an
// FP64 sweep); the warp-per-cell mixed kernel at 1, 2 or 4 cells per block
// (the same per-output code).
bool shape_same_arith(const adg_state* st, int shape) {
  if (!shape_applies(st, shape)) return false;
  if (st->prec != ADG_PREC_MIXED_FP32 || !split_capable(st))
    return shape == PRED_BLOCK || shape == PRED_BLOCK_ALT;
  return shape == PRED_WARP1 || shape == PRED_WARP2 || shape == PRED_WARP4;
}

// Shapes the autotuner times: those of the default arithmetic, or with
// ADG_OPT_PREDICTOR = -2 every shape that applies (the tensor-pipe
// contractions and the block-per-cell mixed kernel round differently).
bool tune_candidate(const adg_state* st, int shape) {
  return st->pred_opt == -2 ? shape_applies(st, shape) : shape_same_arith(st, shape);
}

// The shape the state's steps launch: the fixed option, else the tuned
// choice, else the default (warp-per-cell with 4 cells per block where it
// applies, the block-per-cell kernel otherwise).
int effective_pred(const adg_state* st) {
  if (st->pred_opt >= 0 && shape_applies(st, st->pred_opt)) return st->pred_opt;
  if (st->pred_tuned >= 0 && shape_applies(st, st->pred_tuned)) return st->pred_tuned;
  return split_capable(st) ? PRED_WARP4 : PRED_BLOCK;
}

StepLaunch single_launch(adg_state* st) {
  StepLaunch sl;
  std::memset(&sl, 0, sizeof(sl));
  sl.pps = st->d_pps1;
  sl.n = 1;
  sl.pre_cells = st->d_pre1;
  for (int k = 0; k < 3; ++k) sl.pre_faces[k] = st->d_pre1 + 2 + 2 * k;
  sl.pre_fix = st->d_pre1 + 8;
  sl.pre_fb = st->d_pre1 + 10;
  sl.pre_refix = st->d_pre1 + 12;
  sl.pre_lim = st->d_pre1 + 14;
  sl.cascade = st->cascade;
  sl.sub32 = 3 - st->sub_fp64;
  sl.sub_f32 = st->sub_f32;
  sl.sub_reg = st->sub_reg;
  sl.flux = st->flux;
  sl.total_cells = st->geo.cells;
  for (int k = 0; k < st->dim; ++k) {
    long long faces = 1;
    for (int j = 0; j < st->dim; ++j) faces *= (j == k) ? st->geo.n[j] + 1 : st->geo.n[j];
    long long nf = 1;
    for (int j = 0; j < st->dim - 1; ++j) nf *= st->N + 1;
    sl.total_faces[k] = faces * nf;
  }
  sl.sum_chunk = st->chunk;
  sl.max_passes = (st->cap + st->chunk - 1) / st->chunk;
  sl.prec = st->prec;
  sl.pred = effective_pred(st);
  sl.ev = st->profile ? st->ev[st->ev_next] : nullptr;
  return sl;
}

// Autotuner: times the predictor in every shape that applies to the state on
// its current level (the dt and coefficients of the last step), `reps`
// launches each after one warm-up launch, with CUDA events on the state's
// stream, and keeps the fastest.  The predictor's outputs (the next level's
// volume part and the face traces) are rewritten by the next step, so the
// state is unchanged.  Needs a state that has taken a step (dt > 0).
int autotune_predictor(adg_state* st, int reps, bool* done) {
  *done = false;
  for (int k = 0; k < PRED_COUNT; ++k) st->tune_ms[k] = NAN;
  int rc = refresh(st);
  if (rc) return rc;
  if (st->params_dirty && (rc = upload_params(st))) return rc;
  double dt = 0.0;
  CUDA_TRY(st, cudaMemcpyAsync(&dt, st->b.dt, sizeof(double), cudaMemcpyDeviceToHost, st->stream));
  CUDA_TRY(st, cudaStreamSynchronize(st->stream));
  if (!(dt > 0.0)) return ADG_OK;
  cudaEvent_t e0, e1;
  CUDA_TRY(st, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(st, ADG_ERR_CUDA, "event creation failed");
  }
  StepLaunch sl = single_launch(st);
  sl.ev = nullptr;
  int best = -1;
  double best_ms = 0.0;
  cudaError_t e = cudaSuccess;
  for (int shape = 0; shape < PRED_COUNT && e == cudaSuccess; ++shape) {
    if (!(st->pred_opt >= 0 ? shape_applies(st, shape) : tune_candidate(st, shape))) continue;
    sl.pred = shape;
    LaunchArgs a{};
    a.op = OP_PREDICTOR;
    a.step = &sl;
    a.stream = st->stream;
    e = dispatch(st, a);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st->stream);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = dispatch(st, a);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) break;
    st->tune_ms[shape] = ms / reps;
    if (best < 0 || st->tune_ms[shape] < best_ms) {
      best = shape;
      best_ms = st->tune_ms[shape];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(st, ADG_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
  st->pred_tuned = best;
  *done = true;
  return ADG_OK;
}

// Shapes the autotuner chooses among (a choice when > 1).
int tune_candidates(const adg_state* st) {
  int c = 0;
  for (int k = 0; k < PRED_COUNT; ++k) c += tune_candidate(st, k) ? 1 : 0;
  return c;
}

// Kernels of one step: the wave-speed maximum and the step begin; predictor,
// d face-flux kernels, corrector;
// per limiter pass a prefix, the patch, d sweeps, the subcell predictor, d
// flux kernels and the update; the first-order layer (two prefixes, two
// kernels); the fix prefix and the fix; step end.
long long kernels_per_step(int dim, int passes, int cascade) {
  return 2 + (1 + dim + 1) + (long long)passes * (2 * dim + 4) + (cascade ? 4 : 0) + 2 + 1;
}

// Enqueue one step of the states described by `sl` (all of one dimension,
// degree and precision; `st` selects the kernel instantiation) without
// counting its launches.
int enqueue_step(adg_state* st, const StepLaunch& sl, cudaStream_t stream) {
  CUDA_TRY(st, launch_step_begin(sl, stream));
  LaunchArgs a{};
  a.step = &sl;
  a.stream = stream;
  a.op = OP_STEP_DG;
  cudaError_t e = dispatch(st, a);
  if (e != cudaSuccess) return fail(st, ADG_ERR_CUDA, std::string("DG step: ") + cudaGetErrorString(e));
  a.op = OP_STEP_LIMITER;
  e = dispatch(st, a);
  if (e != cudaSuccess)
    return fail(st, ADG_ERR_CUDA, std::string("subcell limiter: ") + cudaGetErrorString(e));
  CUDA_TRY(st, launch_step_end(sl, stream));
  return ADG_OK;
}

int run_step(adg_state* st, const StepLaunch& sl, cudaStream_t stream) {
  const int rc = enqueue_step(st, sl, stream);
  if (rc) return rc;
  st->launch_count += kernels_per_step(st->dim, sl.max_passes, sl.cascade);
  return ADG_OK;
}

// Kernels of a step whose passes loop on the device, besides the passes
// themselves (each pass adds 2d + 5, counted on the device in CNT_PASSES).
long long kernels_per_loop_step(int dim, int cascade) {
  return kernels_per_step(dim, 0, cascade) + 1;
}

// Capture the steps `sl` describes into a new graph `*out` (captured on
// `cap`, the pass body on `body`): one conditional handle per launch group.
int capture_step_graph(adg_state* st, StepLaunch* sls, adg_state* const* reps, int count,
                       cudaStream_t cap, cudaStream_t body, cudaGraph_t* out) {
  *out = nullptr;
  cudaGraph_t g = nullptr;
  CUDA_TRY(st, cudaGraphCreate(&g, 0));
  for (int i = 0; i < count; ++i) {
    sls[i].loop = 1;
    sls[i].body = body;
    const cudaError_t e = cudaGraphConditionalHandleCreate(&sls[i].cond, g, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return fail(st, ADG_ERR_CUDA, std::string("conditional handle: ") + cudaGetErrorString(e));
    }
  }
  cudaError_t e = cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(st, ADG_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  }
  int rc = ADG_OK;
  for (int i = 0; i < count && rc == ADG_OK; ++i) rc = enqueue_step(reps[i], sls[i], cap);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(cap, &captured);
  if (rc || e != cudaSuccess) {
    cudaGraphDestroy(g);
    if (rc) return rc;
    return fail(st, ADG_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  }
  *out = g;
  return ADG_OK;
}

// One step as one graph launch: the DG phase, the limiter passes in a
// conditional loop sized on the device from the troubled count, the
// first-order layer, the fix and the level swap, with no host wait.  The
// graph is captured on the first step and replayed while the launch
// description (grid, options, dt source, CFL number, phase events) stays the
// same.
int run_step_graph(adg_state* st, const StepLaunch& sl) {
  const int k = st->profile ? st->ev_next : 0;
  if (!(st->gexec[k] && std::memcmp(&st->gsl[k], &sl, sizeof(sl)) == 0)) {
    drop_graph(st, k);
    if (!st->cap_stream) CUDA_TRY(st, cudaStreamCreateWithFlags(&st->cap_stream, cudaStreamNonBlocking));
    if (!st->body_stream) CUDA_TRY(st, cudaStreamCreateWithFlags(&st->body_stream, cudaStreamNonBlocking));
    StepLaunch cl = sl;
    adg_state* rep = st;
    cudaGraph_t g = nullptr;
    int rc = capture_step_graph(st, &cl, &rep, 1, st->cap_stream, st->body_stream, &g);
    if (rc) return rc;
    const cudaError_t e = cudaGraphInstantiate(&st->gexec[k], g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      st->gexec[k] = nullptr;
      return fail(st, ADG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    st->graph[k] = g;
    st->gsl[k] = sl;
  }
  CUDA_TRY(st, cudaGraphLaunch(st->gexec[k], st->stream));
  st->launch_count += kernels_per_loop_step(st->dim, sl.cascade);
  return ADG_OK;
}

// One step whose limiter passes the host sizes from the step's troubled count:
// after the DG phase the device Params (level and stamp at the step's start),
// counters and dt come back in one wait, the limiter runs ceil(n_T / chunk)
// passes instead of the capacity's worth, and the host knows the level the
// step leaves behind.
int run_step_host_passes(adg_state* st, StepLaunch& sl) {
  cudaStream_t stream = st->stream;
  if (!st->probe) {
    void* h = nullptr;
    CUDA_TRY(st, cudaHostAlloc(&h, sizeof(adg_state::Probe), cudaHostAllocDefault));
    st->probe = static_cast<adg_state::Probe*>(h);
  }
  CUDA_TRY(st, launch_step_begin(sl, stream));
  LaunchArgs a{};
  a.step = &sl;
  a.stream = stream;
  a.op = OP_STEP_DG;
  cudaError_t e = dispatch(st, a);
  if (e != cudaSuccess) return fail(st, ADG_ERR_CUDA, std::string("DG step: ") + cudaGetErrorString(e));
  adg_state::Probe* pr = st->probe;
  CUDA_TRY(st, cudaMemcpyAsync(&pr->p, st->dparams, sizeof(Params), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(st, cudaMemcpyAsync(pr->counters, st->b.counters, sizeof(pr->counters),
                               cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(st, cudaMemcpyAsync(&pr->dt, st->b.dt, sizeof(double), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(st, cudaStreamSynchronize(stream));
  const bool stepped = pr->dt > 0.0;
  long long nT = stepped ? pr->counters[CNT_TROUBLED0 + (1 - pr->p.cur)] : 0;
  if (nT > st->cap) nT = st->cap;
  sl.max_passes = (int)((nT + st->chunk - 1) / st->chunk);
  a.op = OP_STEP_LIMITER;
  e = dispatch(st, a);
  if (e != cudaSuccess)
    return fail(st, ADG_ERR_CUDA, std::string("subcell limiter: ") + cudaGetErrorString(e));
  CUDA_TRY(st, launch_step_end(sl, stream));
  st->launch_count += kernels_per_step(st->dim, sl.max_passes, sl.cascade);
  st->cur = stepped ? 1 - pr->p.cur : pr->p.cur;
  st->stamp = pr->p.stamp;
  return ADG_OK;
}

int common_step(adg_state* st, const double* dts_dev, double cfl, double dt_max) {
  if (st->profile) {
    int rc = collect_phases(st, st->ev_next);     // the set this step records into
    if (rc) return rc;
  }
  if (st->params_dirty) {
    int rc = upload_params(st);
    if (rc) return rc;
  }
  StepLaunch sl = single_launch(st);
  sl.dts = dts_dev;
  sl.cfl = cfl;
  sl.dt_max = dt_max;
  if (st->host_passes) {
    int rc = run_step_host_passes(st, sl);
    if (rc) return rc;
    st->cur_known = true;
  } else {
    int rc = run_step_graph(st, sl);
    if (rc) return rc;
    st->cur_known = false;          // the device swapped levels (unless the state idled)
  }
  if (st->profile) {
    st->pending[st->ev_next] = true;
    st->ev_next = (st->ev_next + 1) % adg_state::kEventSets;
  }
  st->lam_valid = st->lam_mode;
  if (st->pred_opt < 0 && st->pred_tuned < 0 && tune_candidates(st) > 1) {
    // the first step of an untuned state: time the predictor shapes on the
    // level it left (later steps launch the fastest; the next graph capture
    // picks it up)
    bool done = false;
    int rc = autotune_predictor(st, 3, &done);
    if (rc) return rc;
  }
  return ADG_OK;
}

// Make b.lam describe the current level; later steps keep it current.
int ensure_lambda(adg_state* st) {
  if (!st->lam_mode) {
    st->lam_mode = true;
    st->params_dirty = true;
  }
  if (st->lam_valid) return ADG_OK;
  int rc0 = refresh(st);
  if (rc0) return rc0;
  LaunchArgs a{};
  a.op = OP_LAMBDA;
  int rc = launch(st, a, "wave speeds");
  if (rc) return rc;
  st->lam_valid = true;
  return ADG_OK;
}

}  // namespace

struct adg_batch {
  std::vector<adg_state*> states;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  struct Group {
    adg_state* rep;                 // selects the kernel instantiation
    std::vector<int> idx;
    StepLaunch sl;
    int dts_off;
  };
  std::vector<Group> groups;
  std::vector<void*> mem;
  double* d_dts = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double graph_cfl = -1.0;
  int cfl_steps = 0;
  cudaStream_t cap = nullptr, body = nullptr;   // capture streams of the step graph
};

namespace {

void batch_free(adg_batch* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->body) cudaStreamDestroy(b->body);
  for (void* p : b->mem) cudaFree(p);
  if (b->own_stream) {
    for (adg_state* st : b->states) st->stream = nullptr;
    cudaStreamDestroy(b->stream);
  }
  delete b;
}

int batch_run(adg_batch* b, bool fixed, double cfl) {
  for (auto& g : b->groups) {
    StepLaunch sl = g.sl;
    sl.dts = fixed ? b->d_dts + g.dts_off : nullptr;
    sl.cfl = cfl;
    sl.dt_max = 0.0;
    int rc = run_step(g.rep, sl, b->stream);
    if (rc) return rc;
  }
  return ADG_OK;
}

}  // namespace

extern "C" {

int adg_batch_create(adg_state* const* states, int count, void* stream, adg_batch** out) {
  if (!out || !states || count < 1) return ADG_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < count; ++i)
    if (!states[i] || !states[i]->loaded) return ADG_ERR_ARG;
  adg_batch* b = new (std::nothrow) adg_batch();
  if (!b) return ADG_ERR_OOM;
  b->states.assign(states, states + count);
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return ADG_ERR_CUDA;
    }
    b->own_stream = true;
  }
  // every state: host view current, Params uploaded, work on the batch stream
  for (adg_state* st : b->states) {
    if (refresh(st) || (st->stream && cudaStreamSynchronize(st->stream) != cudaSuccess)) {
      batch_free(b);
      return ADG_ERR_CUDA;
    }
    st->stream = b->stream;
    if (st->params_dirty && upload_params(st)) {
      batch_free(b);
      return ADG_ERR_CUDA;
    }
  }
  // groups of equal (dimension, degree, precision)
  std::vector<int> done(count, 0);
  int off = 0;
  for (int i = 0; i < count; ++i) {
    if (done[i]) continue;
    adg_batch::Group g;
    g.rep = states[i];
    for (int j = i; j < count; ++j) {
      const adg_state* a = states[i];
      const adg_state* c = states[j];
      if (!done[j] && a->dim == c->dim && a->N == c->N && a->prec == c->prec &&
          a->sub_fp64 == c->sub_fp64 && a->sub_f32 == c->sub_f32 && a->sub_reg == c->sub_reg &&
          a->flux == c->flux &&
          effective_pred(a) == effective_pred(c)) {
        g.idx.push_back(j);
        done[j] = 1;
      }
    }
    const int n = (int)g.idx.size();
    std::vector<Params*> pps(n);
    std::vector<long long> pc(n + 1, 0), pf[3];
    for (int k = 0; k < 3; ++k) pf[k].assign(n + 1, 0);
    long long sum_chunk = 0;
    int max_passes = 0;
    StepLaunch sl;
    std::memset(&sl, 0, sizeof(sl));
    for (int q = 0; q < n; ++q) {
      adg_state* st = states[g.idx[q]];
      pps[q] = st->dparams;
      const StepLaunch one = single_launch(st);
      pc[q + 1] = pc[q] + one.total_cells;
      for (int k = 0; k < 3; ++k) pf[k][q + 1] = pf[k][q] + one.total_faces[k];
      sum_chunk += st->chunk;
      if (st->cascade) sl.cascade = 1;
      const int passes = (st->cap + st->chunk - 1) / st->chunk;
      if (passes > max_passes) max_passes = passes;
    }
    void* d = nullptr;
    const size_t bytes = sizeof(Params*) * n + sizeof(long long) * ((size_t)(n + 1) * 8 + 2);
    if (cudaMalloc(&d, bytes) != cudaSuccess) {
      batch_free(b);
      return ADG_ERR_OOM;
    }
    b->mem.push_back(d);
    Params** dpps = (Params**)d;
    long long* dpre = (long long*)(dpps + n);
    cudaMemcpy(dpps, pps.data(), sizeof(Params*) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dpre, pc.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice);
    for (int k = 0; k < 3; ++k)
      cudaMemcpy(dpre + (size_t)(k + 1) * (n + 1), pf[k].data(), sizeof(long long) * (n + 1),
                 cudaMemcpyHostToDevice);
    sl.pps = dpps;
    sl.n = n;
    sl.pre_cells = dpre;
    for (int k = 0; k < 3; ++k) sl.pre_faces[k] = dpre + (size_t)(k + 1) * (n + 1);
    sl.pre_fix = dpre + (size_t)4 * (n + 1);
    sl.pre_fb = dpre + (size_t)5 * (n + 1);
    sl.pre_refix = dpre + (size_t)6 * (n + 1);
    sl.pre_lim = dpre + (size_t)7 * (n + 1);          // n + 3 entries
    sl.total_cells = pc[n];
    for (int k = 0; k < 3; ++k) sl.total_faces[k] = pf[k][n];
    sl.sum_chunk = sum_chunk;
    sl.max_passes = max_passes;
    sl.prec = g.rep->prec;
    sl.sub32 = 3 - g.rep->sub_fp64;
    sl.sub_f32 = g.rep->sub_f32;
    sl.sub_reg = g.rep->sub_reg;
    sl.flux = g.rep->flux;
    sl.pred = effective_pred(g.rep);
    sl.ev = nullptr;
    g.sl = sl;
    g.dts_off = off;
    off += n;
    b->groups.push_back(g);
  }
  if (cudaMalloc((void**)&b->d_dts, sizeof(double) * count) != cudaSuccess) {
    batch_free(b);
    return ADG_ERR_OOM;
  }
  b->mem.push_back(b->d_dts);
  if (cudaGetLastError() != cudaSuccess) {
    batch_free(b);
    return ADG_ERR_CUDA;
  }
  *out = b;
  return ADG_OK;
}

int adg_batch_step(adg_batch* b, const double* dts, double cfl) {
  if (!b) return ADG_ERR_ARG;
  adg_state* st0 = b->states[0];
  if (dts) {
    // host steps in group order
    std::vector<double> ordered(b->states.size());
    for (auto& g : b->groups)
      for (size_t q = 0; q < g.idx.size(); ++q) {
        const double dt = dts[g.idx[q]];
        if (!(dt > 0.0) || std::isinf(dt)) return fail(st0, ADG_ERR_ARG, "dt must be positive");
        ordered[g.dts_off + q] = dt;
      }
    CUDA_TRY(st0, cudaMemcpyAsync(b->d_dts, ordered.data(), sizeof(double) * ordered.size(),
                                  cudaMemcpyHostToDevice, b->stream));
    CUDA_TRY(st0, cudaStreamSynchronize(b->stream));   // `ordered` leaves scope
    int rc = batch_run(b, true, 0.0);
    if (rc) return rc;
  } else {
    for (adg_state* st : b->states)
      if (!(cfl > 0.0) && !(st->cfl > 0.0))
        return fail(st0, ADG_ERR_ARG, "cfl must be positive (argument or ADG_OPT_CFL)");
    for (adg_state* st : b->states) {
      int rc = ensure_lambda(st);
      if (!rc && st->params_dirty) rc = upload_params(st);
      if (rc) return rc;
    }
    if (!(b->exec && b->graph_cfl == cfl)) {
      // one graph for the step of every group; each group's limiter passes
      // loop on the device (conditional node), sized by its troubled counts
      if (b->exec) cudaGraphExecDestroy(b->exec);
      if (b->graph) cudaGraphDestroy(b->graph);
      b->exec = nullptr;
      b->graph = nullptr;
      if (!b->cap) CUDA_TRY(st0, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
      if (!b->body) CUDA_TRY(st0, cudaStreamCreateWithFlags(&b->body, cudaStreamNonBlocking));
      std::vector<StepLaunch> sls;
      std::vector<adg_state*> reps;
      for (auto& g : b->groups) {
        StepLaunch sl = g.sl;
        sl.dts = nullptr;
        sl.cfl = cfl;
        sl.dt_max = 0.0;
        sls.push_back(sl);
        reps.push_back(g.rep);
      }
      cudaGraph_t g = nullptr;
      const int rc = capture_step_graph(st0, sls.data(), reps.data(), (int)sls.size(), b->cap, b->body, &g);
      if (rc) return rc;
      const cudaError_t e = cudaGraphInstantiate(&b->exec, g, 0);
      if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        b->exec = nullptr;
        return fail(st0, ADG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      }
      b->graph = g;
      b->graph_cfl = cfl;
    }
    CUDA_TRY(st0, cudaGraphLaunch(b->exec, b->stream));
    for (auto& g : b->groups) g.rep->launch_count += kernels_per_loop_step(g.rep->dim, g.sl.cascade);
    b->cfl_steps += 1;
  }
  for (adg_state* st : b->states) {
    st->cur_known = false;
    st->lam_valid = st->lam_mode;
  }
  return ADG_OK;
}

void adg_batch_destroy(adg_batch* b) {
  if (b) batch_free(b);
}

int adg_step_batch(adg_state* const* states, const double* dts, int count) {
  if (!states || !dts || count < 1 || !states[0]) return ADG_ERR_ARG;
  adg_batch* b = nullptr;
  int rc = adg_batch_create(states, count, states[0]->stream, &b);
  if (rc) return rc;
  rc = adg_batch_step(b, dts, 0.0);
  adg_batch_destroy(b);
  return rc;
}

int adg_time(adg_state* st, double* t, int64_t* steps) {
  if (!st) return ADG_ERR_ARG;
  double clk[3] = {0.0, 0.0, 0.0};
  if (st->allocated) {
    CUDA_TRY(st, cudaMemcpyAsync(clk, st->b.clock, sizeof(clk), cudaMemcpyDeviceToHost, st->stream));
    int rc = sync(st);
    if (rc) return rc;
  }
  if (t) *t = clk[0];
  if (steps) *steps = (int64_t)clk[2];
  return ADG_OK;
}


int adg_create(const adg_grid* grid, int N, double gamma, const int* bc, int prec,
               adg_state** out) {
  if (!out) return ADG_ERR_ARG;
  *out = nullptr;
  if (!grid || !bc) return ADG_ERR_ARG;
  if (grid->dim != 2 && grid->dim != 3) return ADG_ERR_ARG;
  if (N < 1 || N > 9 || (grid->dim == 3 && N > 3)) return ADG_ERR_ARG;
  if (!(gamma > 1.0)) return ADG_ERR_ARG;
  if (prec != ADG_PREC_FP64 && prec != ADG_PREC_MIXED_FP32 && prec != ADG_PREC_MIXED_TF32)
    return ADG_ERR_ARG;
  // the tensor-pipe contractions exist for the split final stage (2D N <= 5, 3D)
  if (prec == ADG_PREC_MIXED_TF32 && grid->dim == 2 && N >= 6) return ADG_ERR_ARG;
  for (int k = 0; k < grid->dim; ++k) {
    if (grid->n[k] < 1 || !(grid->dx[k] > 0.0)) return ADG_ERR_ARG;
    const int lo = bc[2 * k], hi = bc[2 * k + 1];
    if (lo < ADG_BC_PERIODIC || lo > ADG_BC_FRONT || hi < ADG_BC_PERIODIC || hi > ADG_BC_FRONT)
      return ADG_ERR_ARG;
    if ((lo == ADG_BC_PERIODIC) != (hi == ADG_BC_PERIODIC)) return ADG_ERR_ARG;
  }
  long long cells = 1;
  for (int k = 0; k < grid->dim; ++k) cells *= grid->n[k];
  if (cells > (1LL << 31) - 1) return ADG_ERR_ARG;
  adg_state* st = new (std::nothrow) adg_state();
  if (!st) return ADG_ERR_OOM;
  st->dim = grid->dim;
  st->N = N;
  st->nv = grid->dim + 2;
  // ADG_PREC_MIXED_TF32 is the mixed mode with the tensor-pipe predictor shape
  st->prec = prec == ADG_PREC_MIXED_TF32 ? ADG_PREC_MIXED_FP32 : prec;
  if (prec == ADG_PREC_MIXED_TF32) st->pred_opt = PRED_WARP4_TC;
  st->gamma = gamma;
  st->iters = N + 1;
  // mixed precision: up to N = 5 the last FP32 sweep closes on the FP64 u
  // (no FP64 sweep: same flags and mixed-vs-FP64 distance within 15% as with
  // one, the predictor 1.8x faster); from N = 6 the Picard contraction is weak
  // and one FP64 sweep keeps the distance and the troubled cells down
  st->fp64_sweeps = (N >= 6) ? 1 : 0;
  std::memset(&st->geo, 0, sizeof(Geo));
  st->geo.dim = grid->dim;
  for (int k = 0; k < 3; ++k) {
    st->geo.n[k] = (k < grid->dim) ? grid->n[k] : 1;
    st->geo.dx[k] = (k < grid->dim) ? grid->dx[k] : 1.0;
    st->geo.x0[k] = (k < grid->dim) ? grid->x0[k] : 0.0;
    st->geo.periodic[k] = (k < grid->dim) ? (bc[2 * k] == ADG_BC_PERIODIC) : 0;
    st->geo.bc[2 * k] = (k < grid->dim) ? bc[2 * k] : ADG_BC_PERIODIC;
    st->geo.bc[2 * k + 1] = (k < grid->dim) ? bc[2 * k + 1] : ADG_BC_PERIODIC;
  }
  st->geo.cells = cells;
  build_ops(N, &st->ops_host);
  *out = st;
  return ADG_OK;
}

int adg_set_allocator(adg_state* st, void* (*alloc)(size_t, void*), void (*free_fn)(void*, void*),
                      void* ctx) {
  if (!st) return ADG_ERR_ARG;
  if (st->allocated) return fail(st, ADG_ERR_ARG, "allocator must be set before the first load");
  if ((alloc == nullptr) != (free_fn == nullptr)) return fail(st, ADG_ERR_ARG, "alloc/free pair");
  st->alloc = alloc;
  st->freef = free_fn;
  st->actx = ctx;
  return ADG_OK;
}

int adg_set_stream(adg_state* st, void* stream) {
  if (!st) return ADG_ERR_ARG;
  st->stream = (cudaStream_t)stream;
  return ADG_OK;
}

int adg_set_option(adg_state* st, int key, double value) {
  if (!st) return ADG_ERR_ARG;
  st->params_dirty = true;
  switch (key) {
    case ADG_OPT_DMP_EPS:
      if (!(value >= 0.0)) return fail(st, ADG_ERR_ARG, "eps must be >= 0");
      st->eps = value;
      return ADG_OK;
    case ADG_OPT_DMP_FLOOR:
      if (!(value >= 0.0)) return fail(st, ADG_ERR_ARG, "floor must be >= 0");
      st->floor = value;
      return ADG_OK;
    case ADG_OPT_FORCE_LIMITER:
      st->force = value != 0.0;
      return ADG_OK;
    case ADG_OPT_PICARD_ITERS:
      if (!(value >= 1.0 && value <= 64.0)) return fail(st, ADG_ERR_ARG, "iterations in 1..64");
      st->iters = (int)value;
      return ADG_OK;
    case ADG_OPT_FP64_SWEEPS:
      if (!(value >= 0.0 && value <= 64.0)) return fail(st, ADG_ERR_ARG, "FP64 sweeps in 0..64");
      st->fp64_sweeps = (int)value;
      return ADG_OK;
    case ADG_OPT_END_TIME:
      if (!(value >= 0.0)) return fail(st, ADG_ERR_ARG, "end time must be >= 0");
      st->t_end = value;
      if (st->allocated)
        CUDA_TRY(st, cudaMemcpyAsync(st->b.clock + 1, &st->t_end, sizeof(double),
                                     cudaMemcpyHostToDevice, st->stream));
      if (st->allocated) CUDA_TRY(st, cudaStreamSynchronize(st->stream));
      return ADG_OK;
    case ADG_OPT_SCRATCH_BYTES:
      if (st->allocated) return fail(st, ADG_ERR_ARG, "scratch budget must be set before the first load");
      if (!(value >= 1.0)) return fail(st, ADG_ERR_ARG, "scratch budget must be positive");
      st->scratch_budget = (size_t)value;
      return ADG_OK;
    case ADG_OPT_CASCADE:
      st->cascade = value != 0.0;
      return ADG_OK;
    case ADG_OPT_SUBCELL_FP64_SWEEPS:
      if (!(value >= 0.0 && value <= 3.0)) return fail(st, ADG_ERR_ARG, "subcell FP64 sweeps in 0..3");
      st->sub_fp64 = (int)value;
      return ADG_OK;
    case ADG_OPT_SUBCELL_FP32:
      st->sub_f32 = value != 0.0;
      return ADG_OK;
    case ADG_OPT_SUBCELL_REGISTERS:
      st->sub_reg = value != 0.0;
      return ADG_OK;
    case ADG_OPT_HOST_PASSES:
      st->host_passes = value != 0.0;
      return ADG_OK;
    case ADG_OPT_PROJECT_DELTA:
      if (st->allocated) return fail(st, ADG_ERR_ARG, "set ADG_OPT_PROJECT_DELTA before the first load");
      st->project_delta = value != 0.0;
      return ADG_OK;
    case ADG_OPT_FLUX:
      if (value != ADG_FLUX_RUSANOV && value != ADG_FLUX_OSHER)
        return fail(st, ADG_ERR_ARG, "flux must be ADG_FLUX_RUSANOV or ADG_FLUX_OSHER");
      st->flux = (int)value;
      return ADG_OK;
    case ADG_OPT_CFL:
      if (!(value >= 0.0)) return fail(st, ADG_ERR_ARG, "cfl must be >= 0");
      st->cfl = value;
      return ADG_OK;
    case ADG_OPT_PROFILE:
      if (value != 0.0 && !st->ev[0][0])
        for (int k = 0; k < adg_state::kEventSets; ++k)
          for (int i = 0; i < PHASE_COUNT; ++i) CUDA_TRY(st, cudaEventCreate(&st->ev[k][i]));
      st->profile = value != 0.0;
      return ADG_OK;
    case ADG_OPT_PREDICTOR:
      if (!(value == -1.0 || value == -2.0 ||
            (value >= 0.0 && value < PRED_COUNT && value == (int)value)))
        return fail(st, ADG_ERR_ARG, "predictor shape must be -1, -2 (autotune) or 0..5");
      if (value >= 0.0 && !shape_applies(st, (int)value))
        return fail(st, ADG_ERR_ARG, "that predictor shape does not apply to this state");
      if ((int)value != st->pred_opt) st->pred_tuned = -1;    // tune again in the new mode
      st->pred_opt = (int)value;
      return ADG_OK;
    case ADG_OPT_SLOT_CAPACITY:
      if (st->allocated) return fail(st, ADG_ERR_ARG, "capacity must be set before the first load");
      if (!(value >= 1.0)) return fail(st, ADG_ERR_ARG, "capacity must be >= 1");
      st->cap_req = (long long)value;
      return ADG_OK;
  }
  return fail(st, ADG_ERR_ARG, "unknown option");
}

int adg_load(adg_state* st, const double* dofs, const double* exact) {
  if (!st || !dofs) return ADG_ERR_ARG;
  int rc = begin_load(st);
  if (rc) return rc;
  const size_t nd = (size_t)st->geo.cells * st->nv * nodes_per_cell(st);
  CUDA_TRY(st, cudaMemcpyAsync(st->b.U[0], dofs, nd * sizeof(double), cudaMemcpyHostToDevice,
                               st->stream));
  if (!exact) return load_detect(st, nullptr);
  const size_t ns = (size_t)st->geo.cells * st->nv * subcells_per_cell(st);
  Temp t(st, ns * sizeof(double));
  if (!t.p) return fail(st, ADG_ERR_OOM, "allocation of the exact averages failed");
  CUDA_TRY(st, cudaMemcpyAsync(t.p, exact, ns * sizeof(double), cudaMemcpyHostToDevice, st->stream));
  return load_detect(st, (const double*)t.p);
}

int adg_init_problem(adg_state* st, const adg_problem* pr) {
  if (!st || !pr) return ADG_ERR_ARG;
  if (pr->kind != ADG_IC_RADIAL && pr->kind != ADG_IC_QUADRANT && pr->kind != ADG_IC_PLANAR)
    return fail(st, ADG_ERR_ARG, "unknown problem kind");
  if (pr->kind == ADG_IC_QUADRANT && st->dim != 2)
    return fail(st, ADG_ERR_ARG, "quadrant problems are 2D");
  int rc = begin_load(st);
  if (rc) return rc;
  const size_t ns = (size_t)st->geo.cells * st->nv * subcells_per_cell(st);
  Temp t(st, ns * sizeof(double));
  if (!t.p) return fail(st, ADG_ERR_OOM, "allocation of the exact averages failed");
  Temp f(st, pr->cell_rho_factor ? st->geo.cells * sizeof(double) : 16);
  if (!f.p) return fail(st, ADG_ERR_OOM, "allocation of the density factors failed");
  if (pr->cell_rho_factor)
    CUDA_TRY(st, cudaMemcpyAsync(f.p, pr->cell_rho_factor, st->geo.cells * sizeof(double),
                                 cudaMemcpyHostToDevice, st->stream));
  LaunchArgs a{};
  a.op = OP_PROJECT;
  a.prob = pr;
  a.fac = pr->cell_rho_factor ? (const double*)f.p : nullptr;
  a.out = (double*)t.p;
  rc = launch(st, a, "initial projection");
  if (rc) return rc;
  return load_detect(st, (const double*)t.p);
}

int adg_load_full(adg_state* st, const double* dofs, const uint8_t* beta, const double* sub) {
  if (!st || !dofs || !beta || !sub) return ADG_ERR_ARG;
  int rc = begin_load(st);
  if (rc) return rc;
  const size_t nd = (size_t)st->geo.cells * st->nv * nodes_per_cell(st);
  const size_t ns = (size_t)st->geo.cells * st->nv * subcells_per_cell(st);
  CUDA_TRY(st, cudaMemcpyAsync(st->b.U[0], dofs, nd * sizeof(double), cudaMemcpyHostToDevice,
                               st->stream));
  Temp tb(st, st->geo.cells);
  Temp ts(st, ns * sizeof(double));
  if (!tb.p || !ts.p) return fail(st, ADG_ERR_OOM, "allocation of the load buffers failed");
  CUDA_TRY(st, cudaMemcpyAsync(tb.p, beta, st->geo.cells, cudaMemcpyHostToDevice, st->stream));
  CUDA_TRY(st, cudaMemcpyAsync(ts.p, sub, ns * sizeof(double), cudaMemcpyHostToDevice, st->stream));
  LaunchArgs a{};
  a.op = OP_LOAD_FULL;
  a.beta = (const uint8_t*)tb.p;
  a.sub = (const double*)ts.p;
  rc = launch(st, a, "full load");
  if (rc) return rc;
  rc = sync(st);
  if (rc) return rc;
  int status = 0;
  CUDA_TRY(st, cudaMemcpy(&status, st->b.counters + CNT_STATUS, sizeof(int), cudaMemcpyDeviceToHost));
  if (status & 1) return fail(st, ADG_ERR_CAPACITY, "more flagged cells than subcell slots");
  st->loaded = true;
  st->lam_valid = true;
  return ADG_OK;
}

int adg_read_full(adg_state* st, double* dofs, uint8_t* beta, double* sub) {
  if (!st || !dofs || !beta || !sub) return ADG_ERR_ARG;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  {
    const int rr = refresh(st);
    if (rr) return rr;
  }
  const size_t nd = (size_t)st->geo.cells * st->nv * nodes_per_cell(st);
  const size_t ns = (size_t)st->geo.cells * st->nv * subcells_per_cell(st);
  Temp ts(st, ns * sizeof(double));
  if (!ts.p) return fail(st, ADG_ERR_OOM, "allocation of the read buffer failed");
  LaunchArgs a{};
  a.op = OP_READ_FULL;
  a.out = (double*)ts.p;
  int rc = launch(st, a, "full read");
  if (rc) return rc;
  CUDA_TRY(st, cudaMemcpyAsync(dofs, st->b.U[st->cur], nd * sizeof(double), cudaMemcpyDeviceToHost,
                               st->stream));
  CUDA_TRY(st, cudaMemcpyAsync(beta, st->b.beta[st->cur], st->geo.cells, cudaMemcpyDeviceToHost,
                               st->stream));
  CUDA_TRY(st, cudaMemcpyAsync(sub, ts.p, ns * sizeof(double), cudaMemcpyDeviceToHost, st->stream));
  return sync(st);
}

int adg_step(adg_state* st, double dt) {
  if (!st) return ADG_ERR_ARG;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  if (!(dt > 0.0) || std::isinf(dt)) return fail(st, ADG_ERR_ARG, "dt must be positive and finite");
  CUDA_TRY(st, launch_set_scalar(st->d_dts1, dt, st->stream));
  st->launch_count += 1;
  return common_step(st, st->d_dts1, 0.0, 0.0);
}

int adg_step_cfl(adg_state* st, double cfl, double dt_max) {
  if (!st) return ADG_ERR_ARG;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  if (!(cfl > 0.0)) return fail(st, ADG_ERR_ARG, "cfl must be positive");
  int rc = ensure_lambda(st);
  if (rc) return rc;
  return common_step(st, nullptr, cfl, dt_max);
}

int adg_max_dt(adg_state* st, double cfl, double* dt_out) {
  if (!st || !dt_out) return ADG_ERR_ARG;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  if (!(cfl > 0.0)) return fail(st, ADG_ERR_ARG, "cfl must be positive");
  int rc0 = ensure_lambda(st);
  if (rc0) return rc0;
  rc0 = refresh(st);
  if (rc0) return rc0;
  Params p = make_params(st);
  CUDA_TRY(st, launch_dt(p, cfl, -1.0, st->stream));
  double dt = 0.0;
  CUDA_TRY(st, cudaMemcpyAsync(&dt, st->b.dt, sizeof(double), cudaMemcpyDeviceToHost, st->stream));
  int rc = sync(st);
  if (rc) return rc;
  *dt_out = dt;
  if (!(dt > 0.0) || std::isinf(dt)) {
    int zero = 0;
    CUDA_TRY(st, cudaMemcpy(st->b.counters + CNT_STATUS, &zero, sizeof(int), cudaMemcpyHostToDevice));
    return fail(st, ADG_ERR_STATE, "no admissible wave speed");
  }
  return ADG_OK;
}

int adg_flags(adg_state* st, uint8_t* beta) {
  if (!st || !beta) return ADG_ERR_ARG;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  {
    const int rr = refresh(st);
    if (rr) return rr;
  }
  CUDA_TRY(st, cudaMemcpyAsync(beta, st->b.beta[st->cur], st->geo.cells, cudaMemcpyDeviceToHost,
                               st->stream));
  return sync(st);
}

int adg_read(adg_state* st, double* dofs) {
  if (!st || !dofs) return ADG_ERR_ARG;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  {
    const int rr = refresh(st);
    if (rr) return rr;
  }
  const size_t nd = (size_t)st->geo.cells * st->nv * nodes_per_cell(st);
  CUDA_TRY(st, cudaMemcpyAsync(dofs, st->b.U[st->cur], nd * sizeof(double), cudaMemcpyDeviceToHost,
                               st->stream));
  return sync(st);
}

int adg_troubled_count(adg_state* st, int64_t* out) {
  if (!st || !out) return ADG_ERR_ARG;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  {
    const int rr = refresh(st);
    if (rr) return rr;
  }
  int c = 0;
  CUDA_TRY(st, cudaMemcpyAsync(&c, st->b.counters + CNT_TROUBLED0 + st->cur, sizeof(int),
                               cudaMemcpyDeviceToHost, st->stream));
  int rc = sync(st);
  if (rc) return rc;
  *out = c;
  return ADG_OK;
}

int adg_set_boundary_state(adg_state* st, int face, const double* q) {
  if (!st || !q) return ADG_ERR_ARG;
  if (face < 0 || face >= 2 * st->dim) return fail(st, ADG_ERR_ARG, "face out of range");
  if (st->geo.bc[face] != ADG_BC_INFLOW) return fail(st, ADG_ERR_ARG, "face is not an inflow face");
  const int d = st->dim;
  double kin = 0.0;
  for (int k = 0; k < d; ++k) kin += q[1 + k] * q[1 + k];
  if (!(q[0] > 0.0) || !(q[d + 1] * q[0] - 0.5 * kin > 0.0))
    return fail(st, ADG_ERR_ARG, "inflow state must have rho > 0 and p > 0");
  for (int v = 0; v < st->nv; ++v) st->geo.bstate[face][v] = q[v];
  st->bstate_set |= 1 << face;
  st->params_dirty = true;
  return ADG_OK;
}

int adg_set_boundary_front(adg_state* st, int face, int axis, double a, double b, int kind_before,
                           const double* q_before, int kind_after, const double* q_after) {
  if (!st) return ADG_ERR_ARG;
  if (face < 0 || face >= 2 * st->dim) return fail(st, ADG_ERR_ARG, "face out of range");
  if (st->geo.bc[face] != ADG_BC_FRONT) return fail(st, ADG_ERR_ARG, "face is not a front face");
  if (axis < 0 || axis >= st->dim || axis == face / 2)
    return fail(st, ADG_ERR_ARG, "the front moves along a tangential axis of its face");
  const int kinds[2] = {kind_before, kind_after};
  const double* qs[2] = {q_before, q_after};
  for (int part = 0; part < 2; ++part) {
    const int kd = kinds[part];
    if (kd != ADG_BC_TRANSMISSIVE && kd != ADG_BC_REFLECTIVE && kd != ADG_BC_INFLOW)
      return fail(st, ADG_ERR_ARG, "a front part is transmissive, reflective or inflow");
    for (int v = 0; v < 5; ++v) st->geo.front_state[face][part][v] = 0.0;
    if (kd == ADG_BC_INFLOW) {
      const double* q = qs[part];
      if (!q) return fail(st, ADG_ERR_ARG, "an inflow part needs its state");
      double kin = 0.0;
      for (int k = 0; k < st->dim; ++k) kin += q[1 + k] * q[1 + k];
      if (!(q[0] > 0.0) || !(q[st->dim + 1] * q[0] - 0.5 * kin > 0.0))
        return fail(st, ADG_ERR_ARG, "inflow state must have rho > 0 and p > 0");
      for (int v = 0; v < st->nv; ++v) st->geo.front_state[face][part][v] = q[v];
    }
    st->geo.front_kind[face][part] = kd;
  }
  if (!std::isfinite(a) || !std::isfinite(b)) return fail(st, ADG_ERR_ARG, "front position must be finite");
  st->geo.front_axis[face] = axis;
  st->geo.front_a[face] = a;
  st->geo.front_b[face] = b;
  st->front_set |= 1 << face;
  st->params_dirty = true;
  return ADG_OK;
}

int adg_set_time(adg_state* st, double t) {
  if (!st) return ADG_ERR_ARG;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  if (!std::isfinite(t)) return fail(st, ADG_ERR_ARG, "time must be finite");
  CUDA_TRY(st, cudaMemcpyAsync(st->b.clock, &t, sizeof(double), cudaMemcpyHostToDevice, st->stream));
  CUDA_TRY(st, cudaStreamSynchronize(st->stream));
  return ADG_OK;
}

int adg_fallback_count(adg_state* st, int64_t* last_step, int64_t* total) {
  if (!st) return ADG_ERR_ARG;
  int c[CNT_COUNT] = {};
  if (st->allocated) {
    CUDA_TRY(st, cudaMemcpyAsync(c, st->b.counters, sizeof(c), cudaMemcpyDeviceToHost, st->stream));
    int rc = sync(st);
    if (rc) return rc;
  }
  if (last_step) *last_step = c[CNT_FB];
  if (total) *total = c[CNT_FB_TOTAL];
  return ADG_OK;
}

int adg_status(adg_state* st) {
  if (!st) return ADG_ERR_ARG;
  if (!st->allocated) return ADG_OK;
  int c[CNT_COUNT];
  CUDA_TRY(st, cudaMemcpyAsync(c, st->b.counters, sizeof(c), cudaMemcpyDeviceToHost, st->stream));
  int rc = sync(st);
  if (rc) return rc;
  CUDA_TRY(st, cudaMemsetAsync(st->b.counters + CNT_STATUS, 0, 2 * sizeof(int), st->stream));
  if (c[CNT_STATUS] & 1) return fail(st, ADG_ERR_CAPACITY, "more troubled cells than subcell slots");
  if (c[CNT_STATUS] & 2) return fail(st, ADG_ERR_STATE, "no admissible wave speed");
  if (c[CNT_INADM] > 0)
    return fail(st, ADG_WARN_SUBCELL_INADMISSIBLE,
                std::to_string(c[CNT_INADM]) + " limited cells left inadmissible subcells");
  return ADG_OK;
}

int adg_sizes(const adg_state* st, int64_t* cells, int* nvar, int* nodes, int* subcells) {
  if (!st) return ADG_ERR_ARG;
  if (cells) *cells = st->geo.cells;
  if (nvar) *nvar = st->nv;
  if (nodes) *nodes = nodes_per_cell(st);
  if (subcells) *subcells = subcells_per_cell(st);
  return ADG_OK;
}

int adg_phase_times(adg_state* st, double* ms, int cap) {
  if (!st || !ms || cap < PHASE_END + 1) return ADG_ERR_ARG;
  if (!st->profile) return fail(st, ADG_ERR_ARG, "profiling is off");
  for (int k = 0; k < adg_state::kEventSets; ++k) {
    int rc = collect_phases(st, k);
    if (rc) return rc;
  }
  for (int i = 0; i < PHASE_END; ++i) {
    ms[i] = st->phase_ms[i];
    st->phase_ms[i] = 0.0;
  }
  ms[PHASE_END] = st->timed_steps;
  st->timed_steps = 0;
  return ADG_OK;
}

namespace {

// Validates a box [lo, hi) of cells of the state; its cell count.
int box_count(adg_state* st, const int* lo, const int* hi, long long* count) {
  if (!lo || !hi) return fail(st, ADG_ERR_ARG, "box bounds are null");
  long long c = 1;
  for (int k = 0; k < st->dim; ++k) {
    if (lo[k] < 0 || hi[k] > st->geo.n[k] || lo[k] >= hi[k])
      return fail(st, ADG_ERR_ARG, "box outside the grid or empty along axis " + std::to_string(k));
    c *= hi[k] - lo[k];
  }
  *count = c;
  return ADG_OK;
}

int pack_unpack(adg_state* st, const int* lo, const int* hi, void* buf, int op) {
  if (!st || !buf) return ADG_ERR_ARG;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  if ((reinterpret_cast<uintptr_t>(buf) & 7) != 0) return fail(st, ADG_ERR_ARG, "buffer not 8-byte aligned");
  long long count = 0;
  int rc = box_count(st, lo, hi, &count);
  if (rc) return rc;
  int box[6] = {0, 0, 0, 1, 1, 1};
  for (int k = 0; k < st->dim; ++k) {
    box[k] = lo[k];
    box[3 + k] = hi[k];
  }
  LaunchArgs a{};
  a.op = op;
  a.box = box;
  a.buf = buf;
  rc = launch(st, a, op == OP_PACK ? "pack cells" : "unpack cells");
  if (rc) return rc;
  if (op == OP_UNPACK) st->lam_valid = false;      // the box's wave speeds are not known
  return ADG_OK;
}

}  // namespace

int adg_halo_bytes(const adg_state* st, int64_t count, int64_t* bytes) {
  if (!st || !bytes || count < 0) return ADG_ERR_ARG;
  *bytes = (int64_t)packed_bytes(st->dim, st->N, count);
  return ADG_OK;
}

int adg_pack_cells(adg_state* st, const int* lo, const int* hi, void* buf) {
  return pack_unpack(st, lo, hi, buf, OP_PACK);
}

int adg_unpack_cells(adg_state* st, const int* lo, const int* hi, const void* buf) {
  return pack_unpack(st, lo, hi, const_cast<void*>(buf), OP_UNPACK);
}

int adg_troubled_history(adg_state* st, int64_t* out, int max, int* written) {
  if (!st || !written || max < 0 || (max > 0 && !out)) return ADG_ERR_ARG;
  *written = 0;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  double clk[3] = {0.0, 0.0, 0.0};
  std::vector<int> h(HIST_LEN);
  CUDA_TRY(st, cudaMemcpyAsync(clk, st->b.clock, sizeof(clk), cudaMemcpyDeviceToHost, st->stream));
  CUDA_TRY(st, cudaMemcpyAsync(h.data(), st->b.hist, sizeof(int) * HIST_LEN, cudaMemcpyDeviceToHost,
                               st->stream));
  int rc = sync(st);
  if (rc) return rc;
  const long long steps = (long long)clk[2];
  long long k = steps < HIST_LEN ? steps : HIST_LEN;
  if (k > max) k = max;
  for (long long i = 0; i < k; ++i) out[i] = h[(steps - k + i) % HIST_LEN];
  *written = (int)k;
  return ADG_OK;
}

int adg_autotune(adg_state* st, int reps, double* ms, int cap) {
  if (!st || reps < 1 || (cap > 0 && !ms)) return ADG_ERR_ARG;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  bool done = false;
  int rc = autotune_predictor(st, reps, &done);
  if (rc) return rc;
  if (!done) return fail(st, ADG_ERR_ARG, "autotune needs a state that has taken a step");
  for (int k = 0; k < cap && k < PRED_COUNT; ++k) ms[k] = st->tune_ms[k];
  for (int k = PRED_COUNT; k < cap; ++k) ms[k] = NAN;
  return ADG_OK;
}

int adg_info(const adg_state* st, int64_t* out, int cap) {
  if (!st || !out || cap < 4) return ADG_ERR_ARG;
  if (!st->allocated) return ADG_ERR_ARG;
  const int D = st->dim;
  const int nchunks = (st->cap + st->chunk - 1) / st->chunk;
  out[0] = st->cap;
  out[1] = st->chunk;
  out[2] = st->host_passes ? kernels_per_step(D, nchunks, st->cascade)
                           : kernels_per_loop_step(D, st->cascade) + (int64_t)nchunks * (2 * D + 5);
  out[3] = (int64_t)st->bytes_held;
  if (cap >= 5) {
    // host-counted kernels plus the passes that device-sized loops ran
    int passes = 0;
    if (cudaMemcpyAsync(&passes, st->b.counters + CNT_PASSES, sizeof(int), cudaMemcpyDeviceToHost,
                        st->stream) != cudaSuccess ||
        cudaStreamSynchronize(st->stream) != cudaSuccess)
      return ADG_ERR_CUDA;
    out[4] = st->launch_count + (int64_t)passes * (2 * D + 5);
  }
  if (cap >= 8) out[7] = effective_pred(st);
  if (cap >= 7) {
    out[5] = st->iters;
    out[6] = st->prec == ADG_PREC_MIXED_FP32 ? (st->fp64_sweeps < st->iters ? st->fp64_sweeps : st->iters)
                                             : st->iters;
  }
  return ADG_OK;
}

const char* adg_last_error(const adg_state* st) {
  if (!st) return "null state";
  return st->err.c_str();
}

void adg_destroy(adg_state* st) {
  if (!st) return;
  free_all(st);
  for (int k = 0; k < adg_state::kEventSets; ++k)
    for (int i = 0; i < PHASE_COUNT; ++i)
      if (st->ev[k][i]) cudaEventDestroy(st->ev[k][i]);
  if (st->cap_stream) cudaStreamDestroy(st->cap_stream);
  if (st->body_stream) cudaStreamDestroy(st->body_stream);
  delete st;
}

}  // extern "C"
