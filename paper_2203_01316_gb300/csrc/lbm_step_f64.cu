// Kernel instantiations for FP64 storage.
#define LBM_KERNEL_TU
#include "lbm_kernels.cuh"

namespace lbmd {
#define LBM_INST(Q)                                                                                              \
    template cudaError_t launch_step<double, Q>(const Buffers&, const DevParams&, cudaStream_t, bool);              \
    template cudaError_t launch_objective<double, Q>(const Buffers&, const DevParams&, AdjObjective, double*, double*, \
                                                  cudaStream_t);                                                 \
    template cudaError_t launch_init<double, Q>(const Buffers&, const DevParams&, const double*, const double*,     \
                                             const double*, cudaStream_t);                                       \
    template cudaError_t launch_macros<double, Q>(const Buffers&, const DevParams&, double*, double*, double*,      \
                                               cudaStream_t);                                                    \
    template cudaError_t launch_populations<double, Q>(const Buffers&, const DevParams&, double*, double*,          \
                                                    cudaStream_t);                                               \
    template cudaError_t launch_balances<double, Q>(const Buffers&, const DevParams&, double*, double*,             \
                                                 cudaStream_t);                                                  \
    template cudaError_t launch_surface_flux<double, Q>(const Buffers&, const DevParams&, int, double*, double*,    \
                                                     cudaStream_t);
LBM_INST(27)
LBM_INST(7)
template cudaError_t launch_adjoint<double, 27>(const Buffers&, const DevParams&, const double*, const double*, double*,
                                            AdjObjective, double*, cudaStream_t);
template cudaError_t launch_adjoint<double, 7>(const Buffers&, const DevParams&, const double*, const double*, double*,
                                           AdjObjective, double*, cudaStream_t);
}  // namespace lbmd
