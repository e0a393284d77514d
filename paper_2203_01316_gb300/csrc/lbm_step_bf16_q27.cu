// Kernel instantiations for BF16 (shifted) storage, D3Q27 h.
#define LBM_KERNEL_TU
#include "lbm_kernels.cuh"

namespace lbmd {
template cudaError_t launch_step<__nv_bfloat16, 27>(const Buffers&, const DevParams&, cudaStream_t, bool);
template cudaError_t launch_objective<__nv_bfloat16, 27>(const Buffers&, const DevParams&, AdjObjective, double*, double*,
                                              cudaStream_t);
template cudaError_t launch_init<__nv_bfloat16, 27>(const Buffers&, const DevParams&, const double*, const double*,
                                         const double*, cudaStream_t);
template cudaError_t launch_macros<__nv_bfloat16, 27>(const Buffers&, const DevParams&, double*, double*, double*,
                                           cudaStream_t);
template cudaError_t launch_populations<__nv_bfloat16, 27>(const Buffers&, const DevParams&, double*, double*, cudaStream_t);
template cudaError_t launch_record_h<__nv_bfloat16, 27>(const Buffers&, const DevParams&, void*, cudaStream_t);
template cudaError_t launch_mirror<__nv_bfloat16, 27>(const Buffers&, const DevParams&, cudaStream_t);
template cudaError_t launch_inlet<__nv_bfloat16, 27>(const Buffers&, const DevParams&, cudaStream_t, bool);
template cudaError_t launch_balances<__nv_bfloat16, 27>(const Buffers&, const DevParams&, double*, double*, cudaStream_t);
template cudaError_t launch_surface_flux<__nv_bfloat16, 27>(const Buffers&, const DevParams&, int, double*, double*,
                                                 cudaStream_t);
template cudaError_t launch_wall_force<__nv_bfloat16, 27>(const Buffers&, const DevParams&, int, double*, double*,
                                               cudaStream_t);
}  // namespace lbmd
