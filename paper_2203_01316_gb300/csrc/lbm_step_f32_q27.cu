// Kernel instantiations for FP32 storage, D3Q27 h.
#define LBM_KERNEL_TU
#include "lbm_kernels.cuh"

namespace lbmd {
template cudaError_t launch_step<float, 27>(const Buffers&, const DevParams&, cudaStream_t, bool);
template cudaError_t launch_objective<float, 27>(const Buffers&, const DevParams&, AdjObjective, double*, double*,
                                              cudaStream_t);
template cudaError_t launch_init<float, 27>(const Buffers&, const DevParams&, const double*, const double*,
                                         const double*, cudaStream_t);
template cudaError_t launch_macros<float, 27>(const Buffers&, const DevParams&, double*, double*, double*,
                                           cudaStream_t);
template cudaError_t launch_populations<float, 27>(const Buffers&, const DevParams&, double*, double*, cudaStream_t);
template cudaError_t launch_record_h<float, 27>(const Buffers&, const DevParams&, void*, cudaStream_t);
template cudaError_t launch_mirror<float, 27>(const Buffers&, const DevParams&, cudaStream_t);
template cudaError_t launch_inlet<float, 27>(const Buffers&, const DevParams&, cudaStream_t, bool);
template cudaError_t launch_balances<float, 27>(const Buffers&, const DevParams&, double*, double*, cudaStream_t);
template cudaError_t launch_surface_flux<float, 27>(const Buffers&, const DevParams&, int, double*, double*,
                                                 cudaStream_t);
template cudaError_t launch_wall_force<float, 27>(const Buffers&, const DevParams&, int, double*, double*,
                                               cudaStream_t);

// streaming map of the step kernels (storage independent)
__global__ void k_stream_map(const uint8_t* __restrict__ flags, const int32_t* __restrict__ wnode,
                             const uint32_t* __restrict__ wmask, int nw, int32_t* __restrict__ src,
                             const DevParams p) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const size_t N = (size_t)p.N;
    const int type = flags[n] & 3;
    if (type == T_SOLID || type == T_INLET) {
        for (int a = 0; a < 27; ++a) src[a * N + n] = -2;
        return;
    }
    uint32_t mask = 0;
    if (flags[n] & F_WALL) {
        int lo = 0, hi = nw - 1;
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            const int v = wnode[mid];
            if (v == n) { mask = wmask[mid]; break; }
            if (v < n) lo = mid + 1; else hi = mid - 1;
        }
    }
    int x, y, z;
    node_xyz(n, p, x, y, z);
    const Nbr nb = make_nbr(x, y, z, p);
#pragma unroll
    for (int a = 0; a < 27; ++a) src[a * N + n] = (mask & (1u << OPP(a))) ? -1 : src_of(nb, a);
}

cudaError_t launch_stream_map(const Buffers& b, const DevParams& p, int qh, int32_t* src, cudaStream_t s) {
    (void)qh;
    const int grid = (p.N + kBlock - 1) / kBlock;
    k_stream_map<<<grid, kBlock, 0, s>>>(b.flags, b.wnode, b.wmask, b.nw, src, p);
    return cudaGetLastError();
}

cudaError_t launch_reduce6(const double* acc, int n, double* out, cudaStream_t s) {
    k_reduce_partials<6><<<1, 1024, 0, s>>>(acc, n, out);
    return cudaGetLastError();
}
}  // namespace lbmd
