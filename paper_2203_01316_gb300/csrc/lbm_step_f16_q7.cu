// Kernel instantiations for FP16 (shifted) storage, D3Q7 h.
#define LBM_KERNEL_TU
#include "lbm_kernels.cuh"

namespace lbmd {
template cudaError_t launch_step<__half, 7>(const Buffers&, const DevParams&, cudaStream_t, bool);
template cudaError_t launch_objective<__half, 7>(const Buffers&, const DevParams&, AdjObjective, double*, double*,
                                              cudaStream_t);
template cudaError_t launch_init<__half, 7>(const Buffers&, const DevParams&, const double*, const double*,
                                         const double*, cudaStream_t);
template cudaError_t launch_macros<__half, 7>(const Buffers&, const DevParams&, double*, double*, double*,
                                           cudaStream_t);
template cudaError_t launch_populations<__half, 7>(const Buffers&, const DevParams&, double*, double*, cudaStream_t);
template cudaError_t launch_record_h<__half, 7>(const Buffers&, const DevParams&, void*, cudaStream_t);
template cudaError_t launch_mirror<__half, 7>(const Buffers&, const DevParams&, cudaStream_t);
template cudaError_t launch_inlet<__half, 7>(const Buffers&, const DevParams&, cudaStream_t, bool);
template cudaError_t launch_balances<__half, 7>(const Buffers&, const DevParams&, double*, double*, cudaStream_t);
template cudaError_t launch_surface_flux<__half, 7>(const Buffers&, const DevParams&, int, double*, double*,
                                                 cudaStream_t);
template cudaError_t launch_wall_force<__half, 7>(const Buffers&, const DevParams&, int, double*, double*,
                                               cudaStream_t);
}  // namespace lbmd
