// Kernel instantiations for 2D grids, degrees N = 1..5.
#include "launch.cuh"

namespace adg {

cudaError_t upload_constants_2d_lo(int N, const Ops& o) { return upload_picard_constants_here(N, o); }

cudaError_t dispatch_2d_lo(int N, const LaunchArgs& a) {
  switch (N) {
    case 1: return Launch<2, 1>::run(a);
    case 2: return Launch<2, 2>::run(a);
    case 3: return Launch<2, 3>::run(a);
    case 4: return Launch<2, 4>::run(a);
    case 5: return Launch<2, 5>::run(a);
  }
  return cudaErrorInvalidValue;
}

}  // namespace adg
