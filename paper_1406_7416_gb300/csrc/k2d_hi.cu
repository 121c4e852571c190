// Kernel instantiations for 2D grids, degrees N = 6..9.
#include "launch.cuh"

namespace adg {

cudaError_t upload_constants_2d_hi(int N, const Ops& o) { return upload_picard_constants_here(N, o); }

cudaError_t dispatch_2d_hi(int N, const LaunchArgs& a) {
  switch (N) {
    case 6: return Launch<2, 6>::run(a);
    case 7: return Launch<2, 7>::run(a);
    case 8: return Launch<2, 8>::run(a);
    case 9: return Launch<2, 9>::run(a);
  }
  return cudaErrorInvalidValue;
}

}  // namespace adg
