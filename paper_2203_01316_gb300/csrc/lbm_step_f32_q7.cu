// Kernel instantiations for FP32 storage, D3Q7 h.
#define LBM_KERNEL_TU
#include "lbm_kernels.cuh"

namespace lbmd {
template cudaError_t launch_step<float, 7>(const Buffers&, const DevParams&, cudaStream_t, bool);
template cudaError_t launch_objective<float, 7>(const Buffers&, const DevParams&, AdjObjective, double*, double*,
                                              cudaStream_t);
template cudaError_t launch_init<float, 7>(const Buffers&, const DevParams&, const double*, const double*,
                                         const double*, cudaStream_t);
template cudaError_t launch_macros<float, 7>(const Buffers&, const DevParams&, double*, double*, double*,
                                           cudaStream_t);
template cudaError_t launch_populations<float, 7>(const Buffers&, const DevParams&, double*, double*, cudaStream_t);
template cudaError_t launch_record_h<float, 7>(const Buffers&, const DevParams&, void*, cudaStream_t);
template cudaError_t launch_mirror<float, 7>(const Buffers&, const DevParams&, cudaStream_t);
template cudaError_t launch_inlet<float, 7>(const Buffers&, const DevParams&, cudaStream_t, bool);
template cudaError_t launch_balances<float, 7>(const Buffers&, const DevParams&, double*, double*, cudaStream_t);
template cudaError_t launch_surface_flux<float, 7>(const Buffers&, const DevParams&, int, double*, double*,
                                                 cudaStream_t);
template cudaError_t launch_wall_force<float, 7>(const Buffers&, const DevParams&, int, double*, double*,
                                               cudaStream_t);
}  // namespace lbmd
