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
