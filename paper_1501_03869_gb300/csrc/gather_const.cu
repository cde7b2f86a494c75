// gather_const.cu -- instantiations of the gather kernel with constant-speed
// delays computed in the kernel (the conventional back projection that
// Sec. III compares against; the kernel itself is in gather.cuh).
#include "gather.cuh"

namespace patbp {

cudaError_t gather_dispatch_const(const GatherConfig& c, int fmt, const StreamParams& p, int grid,
                                  cudaStream_t st, int* resident, int n_sm) {
  return gather_dispatch_t<1>(c, fmt, p, grid, st, resident, n_sm);
}

const void* gather_func_const(const GatherConfig& c, int fmt) { return gather_func_t<1>(c, fmt); }

}  // namespace patbp
