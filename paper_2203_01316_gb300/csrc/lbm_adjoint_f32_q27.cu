// Adjoint kernel instantiations for FP32 storage, D3Q27 h (a translation
// unit of their own so that they compile in parallel with the step kernels).
#define LBM_KERNEL_TU
#include "lbm_kernels.cuh"

namespace lbmd {
template cudaError_t launch_adjoint<float, 27>(const Buffers&, const DevParams&, const float*, const float*,
                                           const float*, float*, AdjObjective, double*, cudaStream_t);
template cudaError_t launch_adjoint_flow<float, 27>(const Buffers&, const DevParams&, const float*, const float*,
                                                const float*, const float*, float*, float*, AdjObjective, double*,
                                                double*, const float*, float*, cudaStream_t);
}  // namespace lbmd
