// Kernel instantiations for FP64 storage, D3Q7 h.
#define LBM_KERNEL_TU
#include "lbm_kernels.cuh"

namespace lbmd {
template cudaError_t launch_step<double, 7>(const Buffers&, const DevParams&, cudaStream_t, bool);
template cudaError_t launch_objective<double, 7>(const Buffers&, const DevParams&, AdjObjective, double*, double*,
                                              cudaStream_t);
template cudaError_t launch_init<double, 7>(const Buffers&, const DevParams&, const double*, const double*,
                                         const double*, cudaStream_t);
template cudaError_t launch_macros<double, 7>(const Buffers&, const DevParams&, double*, double*, double*,
                                           cudaStream_t);
template cudaError_t launch_populations<double, 7>(const Buffers&, const DevParams&, double*, double*, cudaStream_t);
template cudaError_t launch_record_h<double, 7>(const Buffers&, const DevParams&, void*, cudaStream_t);
template cudaError_t launch_mirror<double, 7>(const Buffers&, const DevParams&, cudaStream_t);
template cudaError_t launch_inlet<double, 7>(const Buffers&, const DevParams&, cudaStream_t, bool);
template cudaError_t launch_balances<double, 7>(const Buffers&, const DevParams&, double*, double*, cudaStream_t);
template cudaError_t launch_surface_flux<double, 7>(const Buffers&, const DevParams&, int, double*, double*,
                                                 cudaStream_t);
template cudaError_t launch_wall_force<double, 7>(const Buffers&, const DevParams&, int, double*, double*,
                                               cudaStream_t);
}  // namespace lbmd
