// gather_wgt.cu -- instantiations of the gather kernel with solid-angle weights
// per (pixel, sensor) and delays from the stored table (mode 2): the exact back
// projection that Eq. (BP) approximates (Sec. II-C).  The kernel is in gather.cuh.
#include "gather.cuh"

namespace patbp {

cudaError_t gather_dispatch_wgt(const GatherConfig& c, int fmt, const StreamParams& p, int grid,
                                cudaStream_t st, int* resident, int n_sm) {
  return gather_dispatch_t<2>(c, fmt, p, grid, st, resident, n_sm);
}

const void* gather_func_wgt(const GatherConfig& c, int fmt) { return gather_func_t<2>(c, fmt); }

}  // namespace patbp
