// gather_wgt_const.cu -- instantiations of the gather kernel with solid-angle
// weights per (pixel, sensor) and constant-speed delays computed in the kernel
// (mode 3).  The kernel is in gather.cuh.
#include "gather.cuh"

namespace patbp {

cudaError_t gather_dispatch_wgt_const(const GatherConfig& c, int fmt, const StreamParams& p, int grid,
                                      cudaStream_t st, int* resident, int n_sm) {
  return gather_dispatch_t<3>(c, fmt, p, grid, st, resident, n_sm);
}

const void* gather_func_wgt_const(const GatherConfig& c, int fmt) { return gather_func_t<3>(c, fmt); }

}  // namespace patbp
