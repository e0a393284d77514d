// Geometry of a channel with spherical obstacles, built on the device: the
// node flags and the wall-link list (node, direction, q, wall) that
// lbm_set_geometry takes (Sec. 3: q is the fraction of the link at which the
// wall lies).  A node is solid when it lies in a closed ball |x - c|^2 <= R^2,
// periodic images in y and z included; a fluid node's link a is a wall link
// when its target x + e_a (inside the box in x) is in a ball, and q is the
// smallest t in (0, 1] with |x + t e_a - c| = R, in FP64, stored as float.
// Every FP64 operation is one correctly rounded IEEE operation in a fixed
// order (no contraction into FMAs), so that the result is reproducible
// bit for bit by any FP64 implementation that follows the same order.
#include <cstdint>
#include <cuda_runtime.h>

#include "lbm_kernels.cuh"

namespace lbmd {
namespace {

using Sphere = GeoSphere;

// squared distance of integer point (x, y, z) from the centre, in the order
// ((dx*dx + dy*dy) + dz*dz), each operation rounded once
__device__ __forceinline__ double dist2(double x, double y, double z, const Sphere& s) {
    const double dx = __dsub_rn(x, s.cx), dy = __dsub_rn(y, s.cy), dz = __dsub_rn(z, s.cz);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// the sphere and the image shifts (ky, kz) whose ball holds the point
// (x, y + ky ny, z + kz nz) for a point given in [0, nx) x [0, ny) x [0, nz)
// plus a step; -1 if none
__device__ int ball_of(int x, int y, int z, const Sphere* sp, int ns, int ny, int nz, int& ky, int& kz) {
    for (int i = 0; i < ns; ++i) {
        // x has no images: a point more than R + 1 away along x is outside by a
        // margin no rounding can close, so the exact test below is skipped
        if (fabs((double)x - sp[i].cx) > sp[i].R + 1.0) continue;
        const double RR = __dmul_rn(sp[i].R, sp[i].R);
        for (int a = -1; a <= 1; ++a)
            for (int b = -1; b <= 1; ++b) {
                if (dist2((double)x, (double)(y + a * ny), (double)(z + b * nz), sp[i]) <= RR) {
                    ky = a;
                    kz = b;
                    return i;
                }
            }
    }
    return -1;
}

__global__ void k_sphere_flags(uint8_t* __restrict__ flags, int nx, int ny, int nz, int periodic_x,
                               const Sphere* __restrict__ sp, int ns) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = (int64_t)nx * ny * nz;
    if (n >= N) return;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
    int ky, kz;
    uint8_t f = 0;
    if (!periodic_x) f = (x == 0) ? 2 : (x == nx - 1 ? 3 : 0);
    if (ball_of(x, y, z, sp, ns, ny, nz, ky, kz) >= 0) f = 1;
    flags[n] = f;
}

// bit a of mask[n]: link a of fluid node n ends in a ball
__global__ void k_sphere_link_masks(const uint8_t* __restrict__ flags, uint32_t* __restrict__ mask, int nx, int ny,
                                    int nz, const Sphere* __restrict__ sp, int ns) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = (int64_t)nx * ny * nz;
    if (n >= N) return;
    uint32_t m = 0;
    if (flags[n] == 0) {
        const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
        for (int a = 1; a < 27; ++a) {
            const int xt = x + EX(a);
            if (xt < 0 || xt >= nx) continue;
            int ky, kz;
            if (ball_of(xt, y + EY(a), z + EZ(a), sp, ns, ny, nz, ky, kz) >= 0) m |= 1u << a;
        }
    }
    mask[n] = m;
}

// links per block of kGeoBlock nodes
__global__ void k_block_link_counts(const uint32_t* __restrict__ mask, int64_t N, int* __restrict__ bsum) {
    __shared__ int warp_sum[kGeoBlock / 32];
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int c = (n < N) ? __popc(mask[n]) : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kGeoBlock / 32; ++w) s += warp_sum[w];
        bsum[blockIdx.x] = s;
    }
}

// exclusive prefix sums of the block counts, one block; total at boff[nb]
__global__ void k_scan_block_counts(const int* __restrict__ bsum, int nb, int64_t* __restrict__ boff) {
    __shared__ int64_t part[kGeoBlock];
    const int t = threadIdx.x;
    const int per = (nb + kGeoBlock - 1) / kGeoBlock;  // consecutive blocks per thread
    int64_t s = 0;
    for (int i = t * per; i < min(nb, (t + 1) * per); ++i) s += bsum[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int i = 0; i < kGeoBlock; ++i) {
            const int64_t v = part[i];
            part[i] = run;
            run += v;
        }
        boff[nb] = run;
    }
    __syncthreads();
    int64_t run = part[t];
    for (int i = t * per; i < min(nb, (t + 1) * per); ++i) {
        boff[i] = run;
        run += bsum[i];
    }
}

// q of link a of node (x, y, z), whose target lies in ball i at image shifts
// (ky, kz): the node in the same image frame, then the smaller root of
// |d + t e|^2 = R^2, clipped to (0, 1]
__device__ float link_q(int x, int y, int z, int a, const Sphere& s, int ky, int kz, int ny, int nz) {
    const double dx = __dsub_rn((double)x, s.cx);
    const double dy = __dsub_rn((double)(y + ky * ny), s.cy);
    const double dz = __dsub_rn((double)(z + kz * nz), s.cz);
    const double ex = EX(a), ey = EY(a), ez = EZ(a);
    const double ee = (double)(EX(a) * EX(a) + EY(a) * EY(a) + EZ(a) * EZ(a));
    const double de = __dadd_rn(__dadd_rn(__dmul_rn(dx, ex), __dmul_rn(dy, ey)), __dmul_rn(dz, ez));
    const double dd = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    double disc = __dsub_rn(__dmul_rn(de, de), __dmul_rn(ee, __dsub_rn(dd, __dmul_rn(s.R, s.R))));
    disc = disc > 0.0 ? disc : 0.0;
    double t = __ddiv_rn(__dsub_rn(-de, __dsqrt_rn(disc)), ee);
    const double tmin = 4.9406564584124654e-324;  // the smallest positive double
    t = t < tmin ? tmin : (t > 1.0 ? 1.0 : t);
    float q = __double2float_rn(t);
    if (q <= 0.0f) q = 1.17549435e-38f;  // the smallest normal float
    return q;
}

__global__ void k_sphere_links_write(const uint32_t* __restrict__ mask, int nx, int ny, int nz,
                                     const Sphere* __restrict__ sp, int ns, const int64_t* __restrict__ boff,
                                     int32_t* __restrict__ lnode, int32_t* __restrict__ ldir,
                                     float* __restrict__ lq, int32_t* __restrict__ lwall) {
    __shared__ int warp_sum[kGeoBlock / 32];
    const int64_t N = (int64_t)nx * ny * nz;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t m = (n < N) ? mask[n] : 0u;
    const int c = __popc(m);
    // exclusive scan of c over the block: within the warp, then across warps
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = c;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) warp_sum[wid] = inc;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < wid; ++w) before += warp_sum[w];
    if (!m) return;
    int64_t k = boff[blockIdx.x] + before + inc - c;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
    for (int a = 1; a < 27; ++a) {
        if (!((m >> a) & 1u)) continue;
        int ky = 0, kz = 0;
        const int i = ball_of(x + EX(a), y + EY(a), z + EZ(a), sp, ns, ny, nz, ky, kz);
        lnode[k] = (int32_t)n;
        ldir[k] = a;
        lq[k] = link_q(x, y, z, a, sp[i], ky, kz, ny, nz);
        lwall[k] = sp[i].wall;
        ++k;
    }
}

}  // namespace

cudaError_t launch_sphere_flags(uint8_t* flags, uint32_t* mask, int nx, int ny, int nz, int periodic_x,
                                const GeoSphere* sp, int ns, int* bsum, int64_t* boff, cudaStream_t s) {
    const int64_t N = (int64_t)nx * ny * nz;
    const int nb = (int)((N + kGeoBlock - 1) / kGeoBlock);
    k_sphere_flags<<<nb, kGeoBlock, 0, s>>>(flags, nx, ny, nz, periodic_x, sp, ns);
    k_sphere_link_masks<<<nb, kGeoBlock, 0, s>>>(flags, mask, nx, ny, nz, sp, ns);
    k_block_link_counts<<<nb, kGeoBlock, 0, s>>>(mask, N, bsum);
    k_scan_block_counts<<<1, kGeoBlock, 0, s>>>(bsum, nb, boff);
    return cudaGetLastError();
}

cudaError_t launch_sphere_links(const uint32_t* mask, int nx, int ny, int nz, const GeoSphere* sp, int ns,
                                const int64_t* boff, int32_t* lnode, int32_t* ldir, float* lq, int32_t* lwall,
                                cudaStream_t s) {
    const int64_t N = (int64_t)nx * ny * nz;
    const int nb = (int)((N + kGeoBlock - 1) / kGeoBlock);
    k_sphere_links_write<<<nb, kGeoBlock, 0, s>>>(mask, nx, ny, nz, sp, ns, boff, lnode, ldir, lq, lwall);
    return cudaGetLastError();
}

}  // namespace lbmd
