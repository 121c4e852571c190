// Kernel instantiations for 3D grids, degrees N = 1..3, plus the
// dimension-independent helpers (time step, scalar upload, scratch sizes).
#include "launch.cuh"

namespace adg {

// dt = min(cfl * min_k dx_k / lambda_max, dt_max) from the per-cell wave
// speeds (Eq. cfl); one block.  A non-finite or non-positive result sets
// status bit 1 and is stored as is.
__global__ void k_dt(Params p, double cfl, double dt_max) {
  __shared__ double red[32];
  double l = 0.0;
  for (long long c = threadIdx.x; c < p.geo.cells; c += blockDim.x) l = nanmax(l, p.b.lam[c]);
  l = block_reduce_max(l, red);
  if (threadIdx.x == 0) {
    double h = p.geo.dx[0];
    for (int k = 1; k < p.dim; ++k) h = fmin(h, p.geo.dx[k]);
    double dt = cfl * h / l;
    if (!(dt > 0.0) || isinf(dt) || l != l) atomicOr(&p.b.counters[CNT_STATUS], 2);
    if (dt_max > 0.0 && dt > dt_max) dt = dt_max;
    *p.b.dt = dt;
    *p.b.lamred = l;
  }
}

__global__ void k_set_scalar(double* dst, double v) { *dst = v; }

// Largest per-cell wave speed of each state for a CFL step: blockIdx.y is the
// state, 64 blocks share its cells and combine their block maxima with an
// atomic max on the bits of the (non-negative) double; NaN is kept as the
// largest key.  k_step_begin reads the key and clears it.  Fixed steps skip.
__global__ void k_lam_max(StepLaunch sl) {
  __shared__ double red[32];
  if (sl.dts) return;
  Params& p = *sl.pps[blockIdx.y];
  double l = 0.0, l1 = 0.0;
  const long long nc = p.geo.cells;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long c0 = 0;
  if ((reinterpret_cast<uintptr_t>(p.b.lam) & 15) == 0) {
    const double2* L2 = reinterpret_cast<const double2*>(p.b.lam);
    const long long n2 = nc / 2;
    for (long long c = t; c < n2; c += stride) {
      const double2 x = L2[c];
      l = nanmax(l, x.x);
      l1 = nanmax(l1, x.y);
    }
    c0 = 2 * n2;
  }
  for (long long c = c0 + t; c < nc; c += stride) l = nanmax(l, p.b.lam[c]);
  l = block_reduce_max(nanmax(l, l1), red);
  if (threadIdx.x == 0) atomicMax(p.b.lamkey, l != l ? LLONG_MAX : __double_as_longlong(l));
}

// Start of a batched step, one block per state: the state's dt (fixed from
// sl.dts, or Eq. (cfl) from its largest wave speed, capped by sl.dt_max and
// by its end time), a new step stamp and cleared counters.  A state with
// dt = 0 idles through the step.
__global__ void k_step_begin(StepLaunch sl) {
  Params& p = *sl.pps[blockIdx.x];
  double dt = 0.0;
  if (sl.dts) {
    dt = sl.dts[blockIdx.x];
  } else {
    // the maximum k_lam_max left (the max is exact: any grouping gives it)
    const long long key = *p.b.lamkey;
    const double l = key == LLONG_MAX ? __longlong_as_double(0x7ff8000000000000LL) : __longlong_as_double(key);
    __syncthreads();
    if (threadIdx.x == 0) *p.b.lamkey = 0;
    double h = p.geo.dx[0];
    for (int k = 1; k < p.dim; ++k) h = fmin(h, p.geo.dx[k]);
    dt = (sl.cfl > 0.0 ? sl.cfl : p.cfl) * h / l;
    if (!(dt > 0.0) || isinf(dt) || l != l) {
      if (threadIdx.x == 0) atomicOr(&p.b.counters[CNT_STATUS], 2);
      dt = 0.0;
    }
    if (sl.dt_max > 0.0 && dt > sl.dt_max) dt = sl.dt_max;
  }
  if (threadIdx.x == 0) {
    const double t = p.b.clock[0], tend = p.b.clock[1];
    if (tend > 0.0) {
      const double rem = tend - t;
      if (dt > rem) dt = rem;
      if (!(rem > 1e-12 * tend)) dt = 0.0;
    }
    *p.b.dt = dt;
    *p.b.tstart = t;
    // the step's dt / dx_k and dt Ns / dx_k, evaluated once here instead of in
    // every thread of every kernel (FP64 divisions)
    const int Ns = 2 * p.N + 1;
    for (int k = 0; k < p.dim; ++k) {
      p.b.coef[k] = dt / p.geo.dx[k];
      p.b.coef[3 + k] = dt * Ns / p.geo.dx[k];
    }
    if (p.b.coef_f) {
      for (int k = 0; k < p.dim; ++k) {
        p.b.coef_f[k] = (float)p.b.coef[k];
        p.b.coef_f[3 + k] = (float)p.b.coef[3 + k];
      }
      p.b.coef_f[6] = (float)(p.gamma - 1.0);
      p.b.coef_f[7] = (float)p.gamma;
    }
    if (dt > 0.0) {
      p.b.counters[CNT_TROUBLED0 + (1 - p.cur)] = 0;
      p.b.counters[CNT_FIX] = 0;
      p.b.counters[CNT_FB] = 0;
      p.b.counters[CNT_REFIX] = 0;
      p.stamp += 1;
      p.b.clock[0] = t + dt;
      p.b.clock[2] += 1.0;
    }
  }
}

// End of a batched step: states that stepped swap levels.
__global__ void k_step_end(StepLaunch sl) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= sl.n) return;
  Params& p = *sl.pps[s];
  if (*p.b.dt > 0.0) {
    // the step's troubled count into the history, at the step's index
    const long long k = (long long)p.b.clock[2] - 1;
    if (p.b.hist && k >= 0) p.b.hist[k % HIST_LEN] = p.b.counters[CNT_TROUBLED0 + (1 - p.cur)];
    p.cur = 1 - p.cur;
  }
}

// Prefix of the troubled cells each state handles in limiter pass `pass`
// (pass < 0: the pass of a device-sized loop, pre_lim[n + 1]).
__global__ void k_lim_prefix(StepLaunch sl, int pass) {
  if (pass < 0) pass = (int)sl.pre_lim[sl.n + 1];
  long long acc = 0;
  for (int s = 0; s < sl.n; ++s) {
    sl.pre_lim[s] = acc;
    acc += pass_len(*sl.pps[s], pass);
  }
  sl.pre_lim[sl.n] = acc;
}

// Opens the device-sized pass loop: the passes this step needs are the most
// any state of the launch needs, ceil(min(n_T, capacity) / chunk), at most
// sl.max_passes, so the loop ends after a bounded number of iterations.
__global__ void k_lim_loop_begin(StepLaunch sl) {
  int need = 0;
  for (int s = 0; s < sl.n; ++s) {
    const Params& p = *sl.pps[s];
    if (!(*p.b.dt > 0.0)) continue;
    int nT = p.b.counters[CNT_TROUBLED0 + (1 - p.cur)];
    if (nT > p.cap) nT = p.cap;
    const int k = (nT + p.chunk - 1) / p.chunk;
    if (k > need) need = k;
  }
  if (need > sl.max_passes) need = sl.max_passes;
  sl.pre_lim[sl.n + 1] = 0;
  sl.pre_lim[sl.n + 2] = need;
  sl.pps[0]->b.counters[CNT_PASSES] += need;
  cudaGraphSetConditional(sl.cond, need > 0 ? 1u : 0u);
}

// Last node of the loop body: the next pass, or the end of the loop.
__global__ void k_lim_loop_next(StepLaunch sl) {
  const long long pass = sl.pre_lim[sl.n + 1] + 1;
  sl.pre_lim[sl.n + 1] = pass;
  cudaGraphSetConditional(sl.cond, pass < sl.pre_lim[sl.n + 2] ? 1u : 0u);
}

// Prefix of the entries of one per-step list counter (states idle this step
// contribute none).
__global__ void k_count_prefix(StepLaunch sl, long long* pre, int counter) {
  long long acc = 0;
  for (int s = 0; s < sl.n; ++s) {
    pre[s] = acc;
    const Params& p = *sl.pps[s];
    if (*p.b.dt > 0.0) acc += p.b.counters[counter];
  }
  pre[sl.n] = acc;
}

// Prefix of the neighbour-fix entries of every state.
__global__ void k_fix_prefix(StepLaunch sl) {
  long long acc = 0;
  for (int s = 0; s < sl.n; ++s) {
    sl.pre_fix[s] = acc;
    const Params& p = *sl.pps[s];
    if (*p.b.dt > 0.0) acc += p.b.counters[CNT_FIX];
  }
  sl.pre_fix[sl.n] = acc;
}


cudaError_t upload_constants_3d(int N, const Ops& o) { return upload_picard_constants_here(N, o); }

cudaError_t dispatch_3d(int N, const LaunchArgs& a) {
  switch (N) {
    case 1: return Launch<3, 1>::run(a);
    case 2: return Launch<3, 2>::run(a);
    case 3: return Launch<3, 3>::run(a);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_dt(const Params& p, double cfl, double dt_max, cudaStream_t s) {
  k_dt<<<1, 1024, 0, s>>>(p, cfl, dt_max);
  return cudaGetLastError();
}

cudaError_t launch_set_scalar(double* dst, double v, cudaStream_t s) {
  k_set_scalar<<<1, 1, 0, s>>>(dst, v);
  return cudaGetLastError();
}

cudaError_t launch_step_begin(const StepLaunch& sl, cudaStream_t s) {
  k_lam_max<<<dim3(64, sl.n), 256, 0, s>>>(sl);
  k_step_begin<<<sl.n, 32, 0, s>>>(sl);
  return cudaGetLastError();
}

cudaError_t launch_step_end(const StepLaunch& sl, cudaStream_t s) {
  k_step_end<<<(sl.n + 127) / 128, 128, 0, s>>>(sl);
  return cudaGetLastError();
}

cudaError_t launch_lim_prefix(const StepLaunch& sl, int pass, cudaStream_t s) {
  k_lim_prefix<<<1, 1, 0, s>>>(sl, pass);
  return cudaGetLastError();
}

cudaError_t launch_lim_loop_begin(const StepLaunch& sl, cudaStream_t s) {
  k_lim_loop_begin<<<1, 1, 0, s>>>(sl);
  return cudaGetLastError();
}

cudaError_t launch_lim_loop_next(const StepLaunch& sl, cudaStream_t s) {
  k_lim_loop_next<<<1, 1, 0, s>>>(sl);
  return cudaGetLastError();
}

cudaError_t add_loop_node(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body) {
  cudaStreamCaptureStatus status;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &status, nullptr, &graph, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) return e;
  if (status != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureUnmatched;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  e = cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &np);
  if (e != cudaSuccess) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

cudaError_t launch_fix_prefix(const StepLaunch& sl, cudaStream_t s) {
  k_fix_prefix<<<1, 1, 0, s>>>(sl);
  return cudaGetLastError();
}

cudaError_t launch_count_prefix(const StepLaunch& sl, long long* pre, int counter, cudaStream_t s) {
  k_count_prefix<<<1, 1, 0, s>>>(sl, pre, counter);
  return cudaGetLastError();
}

size_t packed_bytes(int dim, int N, long long count) {
  if (dim == 2) {
    switch (N) {
      case 1: return Packed<2, 1>::bytes(count);
      case 2: return Packed<2, 2>::bytes(count);
      case 3: return Packed<2, 3>::bytes(count);
      case 4: return Packed<2, 4>::bytes(count);
      case 5: return Packed<2, 5>::bytes(count);
      case 6: return Packed<2, 6>::bytes(count);
      case 7: return Packed<2, 7>::bytes(count);
      case 8: return Packed<2, 8>::bytes(count);
      case 9: return Packed<2, 9>::bytes(count);
    }
  } else {
    switch (N) {
      case 1: return Packed<3, 1>::bytes(count);
      case 2: return Packed<3, 2>::bytes(count);
      case 3: return Packed<3, 3>::bytes(count);
    }
  }
  return 0;
}

size_t limiter_scratch_doubles(int dim, int N, size_t* a, size_t* b, size_t* c, size_t* d,
                               size_t* e, size_t* f) {
  if (dim == 2) {
    switch (N) {
      case 1: return scratch_of<2, 1>(a, b, c, d, e, f);
      case 2: return scratch_of<2, 2>(a, b, c, d, e, f);
      case 3: return scratch_of<2, 3>(a, b, c, d, e, f);
      case 4: return scratch_of<2, 4>(a, b, c, d, e, f);
      case 5: return scratch_of<2, 5>(a, b, c, d, e, f);
      case 6: return scratch_of<2, 6>(a, b, c, d, e, f);
      case 7: return scratch_of<2, 7>(a, b, c, d, e, f);
      case 8: return scratch_of<2, 8>(a, b, c, d, e, f);
      case 9: return scratch_of<2, 9>(a, b, c, d, e, f);
    }
  } else {
    switch (N) {
      case 1: return scratch_of<3, 1>(a, b, c, d, e, f);
      case 2: return scratch_of<3, 2>(a, b, c, d, e, f);
      case 3: return scratch_of<3, 3>(a, b, c, d, e, f);
    }
  }
  return 0;
}

}  // namespace adg
