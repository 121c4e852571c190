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
  cudaEvent_t ev[PHASE_COUNT] = {};
  double phase_ms[PHASE_COUNT] = {};
  int timed_steps = 0;
  bool pending = false;     // events of the last step not yet read
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

void free_all(adg_state* st) {
  if (st->stream) cudaStreamSynchronize(st->stream);
  else cudaDeviceSynchronize();
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
  p.eps = st->eps;
  p.floor = st->floor;
  p.ops = st->ops_dev;
  p.b = st->b;
  p.cur = st->cur;
  p.stamp = st->stamp;
  p.lam_mode = st->lam_mode ? 1 : 0;
  p.fp64_sweeps = st->fp64_sweeps < st->iters ? st->fp64_sweeps : st->iters;
  return p;
}

cudaError_t dispatch(const adg_state* st, LaunchArgs& a) {
  if (st->dim == 2) return st->N <= 5 ? dispatch_2d_lo(st->N, a) : dispatch_2d_hi(st->N, a);
  return dispatch_3d(st->N, a);
}

int launch(adg_state* st, LaunchArgs& a, const char* what) {
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
    cap = cells / 8;
    if (cap < 4096) cap = 4096;
  }
  if (cap > cells) cap = cells;
  st->cap = (int)cap;
  size_t parts[6];
  const size_t per = limiter_scratch_doubles(st->dim, st->N, &parts[0], &parts[1], &parts[2],
                                             &parts[3], &parts[4], &parts[5]);
  const size_t budget = (size_t)2 << 30;   // bytes of limiter scratch
  long long chunk = (long long)(budget / (per * sizeof(double)));
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
  ALLOC(b.dt, double, 2);
  b.lamred = b.dt + 1;
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
  CUDA_TRY(st, cudaMemsetAsync(b.dt, 0, sizeof(double) * 2, st->stream));
  st->allocated = true;
  return ADG_OK;
}

int sync(adg_state* st) {
  CUDA_TRY(st, cudaStreamSynchronize(st->stream));
  return ADG_OK;
}

// Reset the current level's counters before a load
int begin_load(adg_state* st) {
  int rc = ensure_allocated(st);
  if (rc) return rc;
  st->cur = 0;
  CUDA_TRY(st, cudaMemsetAsync(st->b.counters, 0, sizeof(int) * CNT_COUNT, st->stream));
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

// Fold the events of the previous profiled step into the sums.
int collect_phases(adg_state* st) {
  if (!st->pending) return ADG_OK;
  CUDA_TRY(st, cudaEventSynchronize(st->ev[PHASE_END]));
  for (int i = 0; i < PHASE_END; ++i) {
    float ms = 0.f;
    CUDA_TRY(st, cudaEventElapsedTime(&ms, st->ev[i], st->ev[i + 1]));
    st->phase_ms[i] += ms;
  }
  st->timed_steps += 1;
  st->pending = false;
  return ADG_OK;
}

int common_step(adg_state* st) {
  const int nxt = 1 - st->cur;
  if (st->profile) {
    int rc = collect_phases(st);
    if (rc) return rc;
  }
  CUDA_TRY(st, cudaMemsetAsync(st->b.counters + CNT_TROUBLED0 + nxt, 0, sizeof(int), st->stream));
  CUDA_TRY(st, cudaMemsetAsync(st->b.counters + CNT_FIX, 0, sizeof(int), st->stream));
  st->stamp += 1;
  LaunchArgs a{};
  a.ev = st->profile ? st->ev : nullptr;
  a.op = OP_STEP_DG;
  int rc = launch(st, a, "DG step");
  if (rc) return rc;
  a.op = OP_STEP_LIMITER;
  rc = launch(st, a, "subcell limiter");
  if (rc) return rc;
  st->cur = nxt;
  st->pending = st->profile;
  st->lam_valid = st->lam_mode;
  return ADG_OK;
}

// Make b.lam describe the current level; later steps keep it current.
int ensure_lambda(adg_state* st) {
  st->lam_mode = true;
  if (st->lam_valid) return ADG_OK;
  LaunchArgs a{};
  a.op = OP_LAMBDA;
  int rc = launch(st, a, "wave speeds");
  if (rc) return rc;
  st->lam_valid = true;
  return ADG_OK;
}

}  // namespace

extern "C" {

int adg_create(const adg_grid* grid, int N, double gamma, const int* bc, int prec,
               adg_state** out) {
  if (!out) return ADG_ERR_ARG;
  *out = nullptr;
  if (!grid || !bc) return ADG_ERR_ARG;
  if (grid->dim != 2 && grid->dim != 3) return ADG_ERR_ARG;
  if (N < 1 || N > 9 || (grid->dim == 3 && N > 3)) return ADG_ERR_ARG;
  if (!(gamma > 1.0)) return ADG_ERR_ARG;
  if (prec != ADG_PREC_FP64 && prec != ADG_PREC_MIXED_FP32) return ADG_ERR_ARG;
  for (int k = 0; k < grid->dim; ++k) {
    if (grid->n[k] < 1 || !(grid->dx[k] > 0.0)) return ADG_ERR_ARG;
    const int lo = bc[2 * k], hi = bc[2 * k + 1];
    if ((lo != ADG_BC_PERIODIC && lo != ADG_BC_TRANSMISSIVE) ||
        (hi != ADG_BC_PERIODIC && hi != ADG_BC_TRANSMISSIVE))
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
  st->prec = prec;
  st->gamma = gamma;
  st->iters = N + 1;
  std::memset(&st->geo, 0, sizeof(Geo));
  st->geo.dim = grid->dim;
  for (int k = 0; k < 3; ++k) {
    st->geo.n[k] = (k < grid->dim) ? grid->n[k] : 1;
    st->geo.dx[k] = (k < grid->dim) ? grid->dx[k] : 1.0;
    st->geo.x0[k] = (k < grid->dim) ? grid->x0[k] : 0.0;
    st->geo.periodic[k] = (k < grid->dim) ? (bc[2 * k] == ADG_BC_PERIODIC) : 0;
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
      if (!(value >= 1.0 && value <= 64.0)) return fail(st, ADG_ERR_ARG, "FP64 sweeps in 1..64");
      st->fp64_sweeps = (int)value;
      return ADG_OK;
    case ADG_OPT_PROFILE:
      if (value != 0.0 && !st->ev[0])
        for (int i = 0; i < PHASE_COUNT; ++i) CUDA_TRY(st, cudaEventCreate(&st->ev[i]));
      st->profile = value != 0.0;
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
  if (pr->kind != ADG_IC_RADIAL && pr->kind != ADG_IC_QUADRANT)
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
  CUDA_TRY(st, launch_set_scalar(st->b.dt, dt, st->stream));
  return common_step(st);
}

int adg_step_cfl(adg_state* st, double cfl, double dt_max) {
  if (!st) return ADG_ERR_ARG;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  if (!(cfl > 0.0)) return fail(st, ADG_ERR_ARG, "cfl must be positive");
  int rc = ensure_lambda(st);
  if (rc) return rc;
  Params p = make_params(st);
  CUDA_TRY(st, launch_dt(p, cfl, dt_max, st->stream));
  return common_step(st);
}

int adg_max_dt(adg_state* st, double cfl, double* dt_out) {
  if (!st || !dt_out) return ADG_ERR_ARG;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  if (!(cfl > 0.0)) return fail(st, ADG_ERR_ARG, "cfl must be positive");
  int rc0 = ensure_lambda(st);
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
  CUDA_TRY(st, cudaMemcpyAsync(beta, st->b.beta[st->cur], st->geo.cells, cudaMemcpyDeviceToHost,
                               st->stream));
  return sync(st);
}

int adg_read(adg_state* st, double* dofs) {
  if (!st || !dofs) return ADG_ERR_ARG;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  const size_t nd = (size_t)st->geo.cells * st->nv * nodes_per_cell(st);
  CUDA_TRY(st, cudaMemcpyAsync(dofs, st->b.U[st->cur], nd * sizeof(double), cudaMemcpyDeviceToHost,
                               st->stream));
  return sync(st);
}

int adg_troubled_count(adg_state* st, int64_t* out) {
  if (!st || !out) return ADG_ERR_ARG;
  if (!st->loaded) return fail(st, ADG_ERR_ARG, "nothing loaded");
  int c = 0;
  CUDA_TRY(st, cudaMemcpyAsync(&c, st->b.counters + CNT_TROUBLED0 + st->cur, sizeof(int),
                               cudaMemcpyDeviceToHost, st->stream));
  int rc = sync(st);
  if (rc) return rc;
  *out = c;
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
  int rc = collect_phases(st);
  if (rc) return rc;
  for (int i = 0; i < PHASE_END; ++i) {
    ms[i] = st->phase_ms[i];
    st->phase_ms[i] = 0.0;
  }
  ms[PHASE_END] = st->timed_steps;
  st->timed_steps = 0;
  return ADG_OK;
}

int adg_info(const adg_state* st, int64_t* out, int cap) {
  if (!st || !out || cap < 4) return ADG_ERR_ARG;
  if (!st->allocated) return ADG_ERR_ARG;
  const int D = st->dim;
  const int nchunks = (st->cap + st->chunk - 1) / st->chunk;
  out[0] = st->cap;
  out[1] = st->chunk;
  out[2] = 1 + 1 + D + 1 + (int64_t)nchunks * (1 + D + 1 + D + 1) + 1;
  out[3] = (int64_t)st->bytes_held;
  return ADG_OK;
}

const char* adg_last_error(const adg_state* st) {
  if (!st) return "null state";
  return st->err.c_str();
}

void adg_destroy(adg_state* st) {
  if (!st) return;
  free_all(st);
  for (int i = 0; i < PHASE_COUNT; ++i)
    if (st->ev[i]) cudaEventDestroy(st->ev[i]);
  delete st;
}

}  // extern "C"
