// Adjoint kernel instantiations for FP64 storage, D3Q27 h (a translation
// unit of their own so that they compile in parallel with the step kernels).
#define LBM_KERNEL_TU
#include "lbm_kernels.cuh"

namespace lbmd {
template cudaError_t launch_adjoint<double, 27>(const Buffers&, const DevParams&, const double*, const double*,
                                           const double*, double*, AdjObjective, double*, cudaStream_t);
template cudaError_t launch_adjoint_flow<double, 27>(const Buffers&, const DevParams&, const double*, const double*,
                                                const double*, const double*, double*, double*, AdjObjective, double*,
                                                double*, const double*, double*, cudaStream_t);
}  // namespace lbmd
