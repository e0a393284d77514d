// lbm_balances_noalloc: FP64 mass and energy totals of caller-owned FP32
// population arrays, computed without allocating any device memory.
//
// Who needs it: code that hands this library device buffers owned by a host
// framework (a plugin or custom-call interface that passes in its inputs and
// outputs and offers no allocator), or an application that fixes its device
// memory budget at start-up and must not call cudaMalloc afterwards.  The
// ordinary lbm_balances needs a context, whose creation allocates.
//
// How: the per-block partial sums live in a file-scope __device__ array of
// fixed size (kMaxBlocks x 4 doubles = 64 KiB).  Every GPU that loads this
// library holds that array until the process exits.  Host code cannot use
// the array's name as an address (on the host it names a stand-in, not
// device memory), so the device address is looked up with
// cudaGetSymbolAddress with the caller's device current.  The address
// belongs to the module instance of the current CUDA context, so it is
// looked up again on every call whose stream is not capturing (a context
// reset or another context on the same device can move the module); a call
// made while its stream is being captured into a graph uses the address the
// last uncaptured call on that device found, so the first call on a device
// must come before any stream capture, and a context reset between that
// call and a capture leaves a stale address in the graph.
//
// Every call shares the array.  Each call writes every partial slot it later
// reads, so nothing has to be cleared between calls; but two calls whose
// kernels overlap on the GPU (different streams, or different host threads)
// race on the array and may return wrong totals.  Serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/lbm.h"

void lbm_internal_set_global_error(const std::string& msg);  // lbm_api.cu

namespace {

constexpr int kThreads = 256;
constexpr int kNodesPerThread = 64;
constexpr int kMaxBlocks = 2048;
constexpr int64_t kMaxNodes = (int64_t)kMaxBlocks * kThreads * kNodesPerThread;  // 33,554,432
constexpr int kMaxDevices = 64;

// public node flags that hold no state of their own (lbm_set_geometry)
constexpr uint8_t kFlagSolid = 1, kFlagSymmetry = 4;

// partial sums per block: (sum f, sum h, non-finite count, counted nodes)
static __device__ __align__(256) double g_partials[kMaxBlocks * 4];

std::mutex g_mutex;
double* g_addr[kMaxDevices] = {};

__device__ __forceinline__ void warp_block_sum(double (&v)[4], double* sh) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) sh[wid * 4 + k] = v[k];
    __syncthreads();
    if (wid == 0) {
        const int nwarps = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (lane < nwarps) ? sh[lane * 4 + k] : 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
}

// theta: the per-node App. D source Q or NULL.  The arrays hold the
// post-collision state, which already carries the level's source, so a
// node's energy is H = sum(h*) - Q/2 (App. D), the same correction as the
// context's lbm_balances and lbm_macros
__global__ void __launch_bounds__(kThreads) k_partials(const float* __restrict__ f, const float* __restrict__ h,
                                                       int qh, int n_nodes, const uint8_t* __restrict__ flags,
                                                       const float* __restrict__ theta,
                                                       double* __restrict__ part) {
    __shared__ double sh[32 * 4];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const size_t N = (size_t)n_nodes;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x) {
        if (flags && (flags[n] == kFlagSolid || flags[n] == kFlagSymmetry)) continue;
        bool bad = false;
        for (int a = 0; a < 27; ++a) {
            const float x = f[a * N + n];
            bad |= !isfinite(x);
            v[0] += (double)x;
        }
        for (int i = 0; i < qh; ++i) {
            const float x = h[i * N + n];
            bad |= !isfinite(x);
            v[1] += (double)x;
        }
        if (theta) v[1] -= 0.5 * (double)theta[n];
        v[2] += bad ? 1.0 : 0.0;
        v[3] += 1.0;
    }
    warp_block_sum(v, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) part[blockIdx.x * 4 + k] = v[k];
}

__global__ void k_final(const double* __restrict__ part, int nparts, double rho0, double T_ref,
                        double* __restrict__ totals) {
    __shared__ double sh[32 * 4];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += part[i * 4 + k];
    warp_block_sum(v, sh);
    if (threadIdx.x == 0) {
        totals[0] = v[0] + rho0 * v[3];
        totals[1] = v[1] + T_ref * v[3];
        totals[2] = v[2];
    }
}

lbm_status fail(lbm_status s, const std::string& msg) {
    lbm_internal_set_global_error(msg);
    return s;
}

// device address of g_partials in the current context (see the file header)
lbm_status scratch_address(int dev, cudaStream_t s, double** out) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("lbm_balances_noalloc: ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess)
            return fail(LBM_ERR_CUDA, std::string("lbm_balances_noalloc: scratch address: ") + cudaGetErrorString(e));
        g_addr[dev] = static_cast<double*>(p);
    } else if (!g_addr[dev]) {
        return fail(LBM_ERR_STATE,
                    "lbm_balances_noalloc: the first call on a device must come before any stream capture");
    }
    *out = g_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_balances_noalloc(const float* f, const float* h, int q_h, int64_t n_nodes,
                                           const uint8_t* flags, const float* theta, double rho0, double T_ref,
                                           double* totals, void* cuda_stream) {
    if (!f || !h || !totals) return fail(LBM_ERR_INVALID, "lbm_balances_noalloc: null pointer");
    if (q_h != 27 && q_h != 7) return fail(LBM_ERR_INVALID, "lbm_balances_noalloc: q_h must be 27 or 7");
    if (n_nodes < 1) return fail(LBM_ERR_INVALID, "lbm_balances_noalloc: n_nodes must be >= 1");
    if (n_nodes > kMaxNodes)
        return fail(LBM_ERR_INVALID, "lbm_balances_noalloc: n_nodes = " + std::to_string((long long)n_nodes) +
                                         " exceeds the static scratch capacity of " +
                                         std::to_string((long long)kMaxNodes) + " nodes");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("lbm_balances_noalloc: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(LBM_ERR_INVALID, "lbm_balances_noalloc: device index too large");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double* part = nullptr;
    const lbm_status st = scratch_address(dev, s, &part);
    if (st != LBM_OK) return st;
    const int per_block = kThreads * kNodesPerThread;
    const int blocks = (int)((n_nodes + per_block - 1) / per_block);
    k_partials<<<blocks, kThreads, 0, s>>>(f, h, q_h, (int)n_nodes, flags, theta, part);
    k_final<<<1, 1024, 0, s>>>(part, blocks, rho0, T_ref, totals);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("lbm_balances_noalloc: ") + cudaGetErrorString(e));
    return LBM_OK;
}
