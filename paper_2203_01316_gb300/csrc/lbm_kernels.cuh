// Kernel templates and their launchers.  The launchers are declared for every
// translation unit; their bodies (and the kernels) are compiled only where
// LBM_KERNEL_TU is defined, one translation unit per storage type.
#pragma once

#include "lbm_device.cuh"

namespace lbmd {

// internal node flags: bits 0-1 type, bit 2 = has at least one wall link,
// bit 3 = is x_f (= x - e_a) of a wall link (x, a) with q <= 1/2
enum : uint8_t { T_FLUID = 0, T_SOLID = 1, T_INLET = 2, T_OUTLET = 3, F_WALL = 4, F_RWALL = 8 };

struct Buffers {
    const void* fA;  // post-collision state, time t
    void* fB;        // post-collision state, time t+1
    const void* hA;
    void* hB;
    const uint8_t* flags;
    const float* theta;       // per-node source or nullptr
    const void* inlet_post;   // R[27 + QH]: inlet post-collision deviations
    const int32_t* wnode;     // wall nodes (sorted)
    const int32_t* seg_base;  // wall nodes before each 32-node segment
    const uint32_t* wmask;    // bit a set: node + e_a is solid
    const int32_t* woff;      // first link of the wall node
    const float* lq;          // per link q, sorted by (node, dir)
    const int32_t* lwall;     // per link wall id
    const float* Twall;       // per wall temperature
    int nw;                   // number of wall nodes
    // adjoint: nodes y that are x_f = x - e_a of a link (x, a) with q <= 1/2
    const int32_t* rseg_base; // such nodes before each 32-node segment
    const uint32_t* rmask;    // bit a set: y + e_a has link a with q <= 1/2
    const int32_t* roff;      // first entry in rlink
    const int32_t* rlink;     // link index (into lq / lwall) of each entry
    double* dlink;            // per link accumulator of dJ/dT_w terms
    void* urec;               // recorded velocities of a step (3N, R) or nullptr
    void* frec;               // coupled adjoint record of a level (R): the ten raw moments of the
                              // pre-collision f arrivals [10][N], then, with the Zou-He inlet, the
                              // inlet nodes' full arrivals [27][ny nz]; or nullptr
    void* hrec;               // recorded pre-collision h arrivals (Q_h N, R) or nullptr
};

// objective of the adjoint: a linear function of the post-collision state
struct AdjObjective {
    int kind;       // 0: surface heat flux of `wall`; 1: sum e_x h over the plane x = plane;
                    // 2: component `comp` of the momentum-exchange force on `wall` (f only)
    int wall, plane, comp;
    double weight;  // 0: no objective term at this level
};

constexpr int kBlock = 128;
constexpr int kRedBlocks = 1216;  // 8 x 152 SMs, partial sums of the reductions
constexpr int kRedThreads = 256;

// advance_h = false advances f only (velocity recomputation for the adjoint);
// b.urec non-null records the velocity u used by each node's collision
template <typename S, int QH>
cudaError_t launch_step(const Buffers& b, const DevParams& p, cudaStream_t s, bool advance_h = true);
// adjoint of one level of the h evolution (R = float, or double for FP64
// storage); h_level: the level's post-collision h record (Cumulants-1st only)
template <typename R, int QH>
cudaError_t launch_adjoint(const Buffers& b, const DevParams& p, const R* u_level, const R* h_level,
                           const R* mu_next, R* mu_out, AdjObjective obj, double* dtheta, cudaStream_t s);
// Zou-He inlet plane, after a step (advance_h = false: f only)
template <typename S, int QH>
cudaError_t launch_inlet(const Buffers& b, const DevParams& p, cudaStream_t s, bool advance_h);
// symmetry rows: fill them in the post-collision arrays before a step
template <typename S, int QH>
cudaError_t launch_mirror(const Buffers& b, const DevParams& p, cudaStream_t s);
// out[0..5] = sum over the n nodes of acc[n * 6 + k] (the coupled adjoint's
// per-node dJ/dF, dJ/du_in accumulators)
cudaError_t launch_reduce6(const double* acc, int n, double* out, cudaStream_t s);
// adjoint of one level of the coupled f + h evolution (records of the level's
// pre-collision arrivals; f_level NULL at the initial level); wbuf: R[3][N]
// scratch for the velocity derivative passed from the h to the f kernel
template <typename R, int QH>
cudaError_t launch_adjoint_flow(const Buffers& b, const DevParams& p, const R* f_level, const R* h_level,
                                const R* muf_next, const R* muh_next, R* muf_out, R* muh_out, AdjObjective obj,
                                double* dtheta, double* acc6, const R* din, R* wbuf, cudaStream_t s);
// rec[i * N + n] = post-collision h deviation of population i at node n (type R)
template <typename S, int QH>
cudaError_t launch_record_h(const Buffers& b, const DevParams& p, void* rec, cudaStream_t s);
// *acc += weight * F(current level) (F: surface flux of a wall, section flux of a plane or one
// component of a wall's force)
template <typename S, int QH>
cudaError_t launch_objective(const Buffers& b, const DevParams& p, AdjObjective obj, double* scratch, double* acc,
                             cudaStream_t s);
template <typename S, int QH>
cudaError_t launch_init(const Buffers& b, const DevParams& p, const double* rho, const double* u, const double* T,
                        cudaStream_t s);
template <typename S, int QH>
cudaError_t launch_macros(const Buffers& b, const DevParams& p, double* rho, double* u, double* T, cudaStream_t s);
template <typename S, int QH>
cudaError_t launch_populations(const Buffers& b, const DevParams& p, double* f, double* h, cudaStream_t s);
// partial sums: scratch[3*kRedBlocks] -> out[3] = (sum of rho, sum of H, non-finite count)
template <typename S, int QH>
cudaError_t launch_balances(const Buffers& b, const DevParams& p, double* scratch, double* out, cudaStream_t s);
template <typename S, int QH>
cudaError_t launch_surface_flux(const Buffers& b, const DevParams& p, int wall, double* scratch, double* out,
                                cudaStream_t s);
// partial sums: scratch[3*kRedBlocks] -> out[3] = momentum-exchange force on the wall
template <typename S, int QH>
cudaError_t launch_wall_force(const Buffers& b, const DevParams& p, int wall, double* scratch, double* out,
                              cudaStream_t s);
cudaError_t launch_stream_map(const Buffers& b, const DevParams& p, int qh, int32_t* src, cudaStream_t s);

// ---- geometry of spheres built on the device (lbm_geometry.cu) ----
struct GeoSphere {
    double cx, cy, cz, R;
    int wall;
};
constexpr int kGeoBlock = 256;
// flags[N] (0 fluid, 1 solid, 2 inlet, 3 outlet), the link masks of the fluid
// nodes, per-block link counts bsum[nb] and their exclusive sums boff[nb + 1]
// (boff[nb] = total), nb = ceil(N / kGeoBlock)
cudaError_t launch_sphere_flags(uint8_t* flags, uint32_t* mask, int nx, int ny, int nz, int periodic_x,
                                const GeoSphere* sp, int ns, int* bsum, int64_t* boff, cudaStream_t s);
// the links, sorted by (node, direction), into arrays of boff[nb] entries
cudaError_t launch_sphere_links(const uint32_t* mask, int nx, int ny, int nz, const GeoSphere* sp, int ns,
                                const int64_t* boff, int32_t* lnode, int32_t* ldir, float* lq, int32_t* lwall,
                                cudaStream_t s);

#ifdef LBM_KERNEL_TU

// ---- pull addressing -------------------------------------------------------
struct Nbr {
    int xs[3];  // source x for e_x = -1, 0, +1 (the source is x - e_x)
    int ys[3];  // ny*nx * ... offsets
    int zs[3];
};

__device__ __forceinline__ void node_xyz(int n, const DevParams& p, int& x, int& y, int& z) {
    const uint32_t r = p.mx ? __umulhi((uint32_t)n, p.mx) >> p.sx : (uint32_t)n;  // n / nx
    const uint32_t q = p.my ? __umulhi(r, p.my) >> p.sy : r;                      // r / ny
    x = n - (int)r * p.nx;
    y = (int)r - (int)q * p.ny;
    z = (int)q;
}

__device__ __forceinline__ Nbr make_nbr(int x, int y, int z, const DevParams& p) {
    Nbr b;
    int xm = x - 1, xp = x + 1;
    if (p.periodic_x) {
        if (xm < 0) xm += p.nx;
        if (xp >= p.nx) xp -= p.nx;
    } else {
        // only the outlet plane reaches past the box: zero normal gradient
        xm = max(xm, 0);
        xp = min(xp, p.nx - 1);
    }
    const int ym = (y == 0) ? p.ny - 1 : y - 1, yp = (y == p.ny - 1) ? 0 : y + 1;
    const int zm = (z == 0) ? p.nz - 1 : z - 1, zp = (z == p.nz - 1) ? 0 : z + 1;
    // index 0 <-> e = -1 (source +1), 2 <-> e = +1 (source -1)
    b.xs[0] = xp; b.xs[1] = x; b.xs[2] = xm;
    b.ys[0] = yp * p.nx; b.ys[1] = y * p.nx; b.ys[2] = ym * p.nx;
    const int pl = p.nx * p.ny;
    b.zs[0] = zp * pl; b.zs[1] = z * pl; b.zs[2] = zm * pl;
    return b;
}

// node from which population a is pulled
__device__ __forceinline__ int src_of(const Nbr& b, int a) {
    return b.xs[EX(a) + 1] + b.ys[EY(a) + 1] + b.zs[EZ(a) + 1];
}

// ---- collision + store shared by the bulk and the wall kernels ----------------
// element (i, node) of an SoA array [Q][N] as a 32-bit unsigned index
// (lbm_create keeps 27 N below 2^31), so that each address is one widening
// multiply-add instead of sign extensions and 64-bit adds
__device__ __forceinline__ uint32_t soa(int i, int N, int node) {
    return (uint32_t)i * (uint32_t)N + (uint32_t)node;
}

// ---- 16-bit stores ------------------------------------------------------------
// Two values of one node (populations a and a + 1) are converted with one
// packed conversion and stored as two 16-bit halves.  Stochastic rounding
// uses the conversion's own random-bits operand (FP16: bits 0-12 round the
// low value, bits 16-28 the high one; BF16: bits 0-15 and 16-31): the value
// rounds up in magnitude with probability equal to the discarded fraction,
// so rounding errors have zero mean.  The 32 bits are one draw of the node's
// stream, which starts at a hash of (node, time level) and serves the f stores
// and then the h stores.
template <bool SR> __device__ __forceinline__ uint32_t cvt_pair(__half*, float hi, float lo, uint32_t r) {
    uint32_t d;
    if constexpr (SR) asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    else asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
template <bool SR> __device__ __forceinline__ uint32_t cvt_pair(__nv_bfloat16*, float hi, float lo, uint32_t r) {
    uint32_t d;
    if constexpr (SR) asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    else asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
// v[0..Q) of node n into X[i * N + n] (16-bit storage)
template <bool SR, typename S, int Q>
__device__ __forceinline__ void store16(S* __restrict__ X, const float* v, int n, int N, SrStream& rs) {
#pragma unroll
    for (int i = 0; i < Q; i += 2) {
        const float hi = (i + 1 < Q) ? v[i + 1] : 0.0f;
        const uint32_t d = cvt_pair<SR>(X, hi, v[i], SR ? rs.next() : 0u);
        *(unsigned short*)(X + soa(i, N, n)) = (unsigned short)(d & 0xffffu);
        if (i + 1 < Q) *(unsigned short*)(X + soa(i + 1, N, n)) = (unsigned short)(d >> 16);
    }
}

template <typename S, int QH>
__device__ __forceinline__ void collide_store_f(typename Acc<S>::R* fd, S* __restrict__ fB, int n,
                                                const DevParams& p, typename Acc<S>::R& ux,
                                                typename Acc<S>::R& uy, typename Acc<S>::R& uz, SrStream& rs) {
    using R = typename Acc<S>::R;
    R rho;
    collide_f<R>(fd, p, ux, uy, uz, rho);
    if constexpr (sizeof(S) == 2) {
        if (p.stochastic) store16<true, S, 27>(fB, fd, n, p.N, rs);
        else store16<false, S, 27>(fB, fd, n, p.N, rs);
    } else {
#pragma unroll
        for (int a = 0; a < 27; ++a) st(fB + soa(a, p.N, n), fd[a]);
    }
}

template <typename S, int QH, bool CUM = false, bool TRT = false>
__device__ __forceinline__ void collide_store_h(typename Acc<S>::R* hd, S* __restrict__ hB, int n,
                                                const DevParams& p, typename Acc<S>::R ux,
                                                typename Acc<S>::R uy, typename Acc<S>::R uz,
                                                typename Acc<S>::R Q, SrStream& rs) {
    using R = typename Acc<S>::R;
    if constexpr (sizeof(R) == 4) {
        // FP32 arithmetic: the transforms' roundings bias the zeroth moment of
        // the result (a steady energy drift over long runs at small k), so
        // the rest population takes exactly what the others leave of the
        // pre-collision zeroth moment plus the source
        R pre;
        collide_h<R, QH, CUM, TRT>(hd, ux, uy, uz, Q, p, &pre);
        R others = R(0);
#pragma unroll
        for (int i = 1; i < QH; ++i) others += hd[i];
        hd[0] = (pre + Q) - others;
    } else {
        collide_h<R, QH, CUM, TRT>(hd, ux, uy, uz, Q, p);
    }
    if constexpr (sizeof(S) == 2) {
        if (p.stochastic) store16<true, S, QH>(hB, hd, n, p.N, rs);
        else store16<false, S, QH>(hB, hd, n, p.N, rs);
    } else {
#pragma unroll
        for (int i = 0; i < QH; ++i) st(hB + soa(i, p.N, n), hd[i]);
    }
}

// the division of the q > 1/2 link rule: the denominator 2q lies in [1, 2],
// where the fast FP32 division is within 2 ulp and needs no range checks
// (porous bed: +2% with the wall nodes' warps serialised on these bodies);
// FP64 keeps the correctly rounded division
template <typename R> __device__ __forceinline__ R wdiv(R a, R b) {
    if constexpr (sizeof(R) == 4) return __fdividef(a, b);
    else return a / b;
}

// ---- the step: pull streaming, Eq. IBB / Eq. IABB on wall links, planes,
// collision of f and h; one thread per node --------------------------------
// Wall nodes find their entry in the wall table without a search: the nodes
// of one warp are 32 consecutive node indices, so the entry is the number of
// wall nodes before the warp (seg_base[n/32]) plus the wall nodes of lower
// lanes (ballot + popc).
// 5 resident blocks of 128 threads per SM caps the step kernel at 96
// registers; measured on the 384x128x128 workload this beats the unbounded
// 171-register build by 1.6x (more warps keep more loads in flight).
#ifndef LBM_STEP_MIN_BLOCKS
#define LBM_STEP_MIN_BLOCKS 5
#endif
// D3Q7 h carries fewer registers: 8 blocks (64 registers) measured 18.3k
// MLUPS on the 512x256x256 porous bed against 15.4k at 5 blocks
#ifndef LBM_STEP_MIN_BLOCKS_Q7
#define LBM_STEP_MIN_BLOCKS_Q7 8
#endif
// 16-bit storage with D3Q27 h: 7 blocks (72 registers) measured 15.38k MLUPS
// (FP16) against 15.30k at 6 and 15.25k at 8
#ifndef LBM_STEP_MIN_BLOCKS_16
#define LBM_STEP_MIN_BLOCKS_16 7
#endif
// FP64 arithmetic needs twice the registers: 2 blocks per SM
template <typename S, int QH> constexpr int step_min_blocks() {
    return sizeof(typename Acc<S>::R) == 8
               ? 2
               : (QH == 7 ? LBM_STEP_MIN_BLOCKS_Q7 : (sizeof(S) == 2 ? LBM_STEP_MIN_BLOCKS_16 : LBM_STEP_MIN_BLOCKS));
}

// EQ: the BB + EQ wall rule (compile time, so the default rules keep their
// register allocation); CUM: the Cumulants-1st h kind; TRT: the CM-TRT kind
// with its rates fixed at compile time.  WM (wall mode): 0 every node; 1
// every node but the wall nodes; 2 the wall nodes only, one thread per entry
// of the wall table (modes 1 and 2 together make one step; see launch_step)
template <typename S, int QH, bool DO_H, bool REC, bool CUM = false, bool EQ = false, bool PRE = false,
          bool TRT = false, int WM = 0>
__global__ void __launch_bounds__(kBlock, step_min_blocks<S, QH>()) k_step(const S* __restrict__ fA, S* __restrict__ fB,
                                                  const S* __restrict__ hA, S* __restrict__ hB,
                                                  const uint8_t* __restrict__ flags,
                                                  const float* __restrict__ theta,
                                                  const typename Acc<S>::R* __restrict__ inlet,
                                                  const int32_t* __restrict__ seg_base,
                                                  const uint32_t* __restrict__ wmask,
                                                  const int32_t* __restrict__ woff,
                                                  const float* __restrict__ lq,
                                                  const int32_t* __restrict__ lwall,
                                                  const float* __restrict__ Twall,
                                                  typename Acc<S>::R* __restrict__ urec,
                                                  void* __restrict__ frec, void* __restrict__ hrec,
                                                  const int32_t* __restrict__ wnode, const DevParams p) {
    using R = typename Acc<S>::R;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in_range = (WM == 2) ? t < p.nwall : t < p.N;
    const int n = (WM == 2) ? (in_range ? __ldg(wnode + t) : 0) : t;
    const uint8_t fl = in_range ? flags[n] : (uint8_t)T_SOLID;
    const bool is_wall = (fl & F_WALL) != 0;
    const uint32_t ballot = (WM == 0) ? __ballot_sync(0xffffffffu, is_wall) : 0u;
    if (!in_range) return;
    if (WM == 1 && is_wall) return;
    const int type = fl & 3;
    if (type == T_SOLID) return;
    const int N = p.N;
    if (type == T_INLET) {
#pragma unroll
        for (int a = 0; a < 27; ++a) st(fB + soa(a, N, n), inlet[a]);
        if (DO_H) {
#pragma unroll
            for (int i = 0; i < QH; ++i) st(hB + soa(i, N, n), inlet[27 + i]);
        }
        if (REC) {
            urec[n] = par<R>(p.uin[0], p.pf.uin[0]);
            urec[N + n] = par<R>(p.uin[1], p.pf.uin[1]);
            urec[2 * N + n] = par<R>(p.uin[2], p.pf.uin[2]);
        }
        return;
    }
    uint32_t mask = 0;
    int off = 0;
    if (is_wall) {
        const int lane = threadIdx.x & 31;
        const int idx = (WM == 2) ? t : __ldg(seg_base + (n >> 5)) + __popc(ballot & ((1u << lane) - 1u));
        mask = __ldg(wmask + idx);
        off = __ldg(woff + idx);
    }
    int x, y, z;
    node_xyz(n, p, x, y, z);
    const Nbr nb = make_nbr(x, y, z, p);
    SrStream rs{sr_bits((uint32_t)n, p.step_ctr ? *p.step_ctr : p.step)};  // 16-bit stochastic rounding: f stores, then h
    R fd[27];
#pragma unroll
    for (int a = 0; a < 27; ++a) fd[a] = ld<R>(fA + soa(a, N, src_of(nb, a)));
    if (WM == 2) {
        // wall nodes alone, so every lane has links: the link bodies without
        // branches (loads predicated on the mask bit, the result selected),
        // so that their loads are in flight together
#pragma unroll
        for (int b = 0; b < 27; ++b) {
            const int a = OPP(b);
            const bool has = (mask >> a) & 1u;
            const float q = has ? __ldg(lq + off + __popc(mask & ((1u << a) - 1u))) : 0.5f;
            const bool thin = (mask >> b) & 1u;
            const R fa_b = has ? ld<R>(fA + soa(a, N, n)) : R(0);
            const R fb_b = has ? ld<R>(fA + soa(b, N, n)) : R(0);
            const R qq = (R)fmaxf(q, 0.5f);
            const R v_lin = R(2) * (R)q * fa_b + (R(1) - R(2) * (R)q) * fd[a];
            const R v_far = wdiv<R>(fa_b + (R(2) * qq - R(1)) * fb_b, R(2) * qq);
            const R v = (q <= 0.5f && !thin) ? v_lin : v_far;
            fd[b] = has ? v : fd[b];
        }
    } else if (mask) {
        // the arrival b whose source x_b - e_b = x_b + e_a (a = opp b) is solid
#pragma unroll
        for (int b = 0; b < 27; ++b) {
            const int a = OPP(b);
            if (!(mask & (1u << a))) continue;
            const float q = __ldg(lq + off + __popc(mask & ((1u << a) - 1u)));
            const bool thin = (mask >> b) & 1u;  // x_f = x_b - e_a is solid too
            const R fa_b = ld<R>(fA + soa(a, N, n));
            if (q <= 0.5f && !thin) {
                fd[b] = R(2) * (R)q * fa_b + (R(1) - R(2) * (R)q) * fd[a];  // fd[a] = f*_a(x_f)
            } else {
                const R qq = (R)fmaxf(q, 0.5f);
                const R fb_b = ld<R>(fA + soa(b, N, n));
                fd[b] = wdiv<R>(fa_b + (R(2) * qq - R(1)) * fb_b, R(2) * qq);
            }
        }
    }
    R ux, uy, uz;
    if constexpr (PRE) {  // the coupled adjoint needs f only through these ten moments
        R m[10];
        raw_moments_f<R>(fd, m[0], m[1], m[2], m[3], m[4], m[5], m[6], m[7], m[8], m[9]);
#pragma unroll
        for (int k = 0; k < 10; ++k) ((R*)frec)[soa(k, N, n)] = m[k];
    }
    collide_store_f<S, QH>(fd, fB, n, p, ux, uy, uz, rs);
    if (REC) {
        urec[n] = ux;
        urec[N + n] = uy;
        urec[2 * N + n] = uz;
    }
    if constexpr (DO_H) {
    R hd[QH];
#pragma unroll
    for (int i = 0; i < QH; ++i) hd[i] = ld<R>(hA + soa(i, N, src_of(nb, HDIR<QH>(i))));
    if (WM == 2) {  // as for f: no branches in the link bodies
        const R Tref = par<R>(p.Tref, p.pf.Tref);
#pragma unroll
        for (int ib = 0; ib < QH; ++ib) {
            const int b = HDIR<QH>(ib);
            const int ia = HOPP<QH>(ib);
            const int a = HDIR<QH>(ia);
            const bool has = (mask >> a) & 1u;
            const int l = off + __popc(mask & ((1u << a) - 1u));
            const float q = has ? __ldg(lq + l) : 0.5f;
            const R heq2 = has ? R(2) * (R)HW<QH>(ia) * ((R)__ldg(Twall + __ldg(lwall + l)) - Tref) : R(0);
            const bool thin = (mask >> b) & 1u;
            R v;
            if constexpr (EQ) {
                v = R(0.5) * heq2;
            } else {
                const R ha_b = has ? ld<R>(hA + soa(ia, N, n)) : R(0);
                const R hb_b = has ? ld<R>(hA + soa(ib, N, n)) : R(0);
                const R qq = (R)fmaxf(q, 0.5f);
                const R v_lin = -(R(2) * (R)q * ha_b + (R(1) - R(2) * (R)q) * hd[ia]) + heq2;
                const R v_far = wdiv<R>(-ha_b + (R(2) * qq - R(1)) * hb_b + heq2, R(2) * qq);
                v = (q <= 0.5f && !thin) ? v_lin : v_far;
            }
            hd[ib] = has ? v : hd[ib];
        }
    } else if (mask) {
        const R Tref = par<R>(p.Tref, p.pf.Tref);
#pragma unroll
        for (int ib = 0; ib < QH; ++ib) {
            const int b = HDIR<QH>(ib);
            const int ia = HOPP<QH>(ib);
            const int a = HDIR<QH>(ia);
            if (!(mask & (1u << a))) continue;
            const int l = off + __popc(mask & ((1u << a) - 1u));
            const float q = __ldg(lq + l);
            const R heq2 = R(2) * (R)HW<QH>(ia) * ((R)__ldg(Twall + __ldg(lwall + l)) - Tref);
            const bool thin = (mask >> b) & 1u;
            if constexpr (EQ) {  // EQ: the wall equilibrium w T_w itself
                hd[ib] = R(0.5) * heq2;
                continue;
            }
            const R ha_b = ld<R>(hA + soa(ia, N, n));
            if (q <= 0.5f && !thin) {
                hd[ib] = -(R(2) * (R)q * ha_b + (R(1) - R(2) * (R)q) * hd[ia]) + heq2;
            } else {
                const R qq = (R)fmaxf(q, 0.5f);
                const R hb_b = ld<R>(hA + soa(ib, N, n));
                hd[ib] = wdiv<R>(-ha_b + (R(2) * qq - R(1)) * hb_b + heq2, R(2) * qq);
            }
        }
    }
    const R Q = theta ? (R)__ldg(theta + n) : R(0);
    if constexpr (PRE) {
#pragma unroll
        for (int i = 0; i < QH; ++i) ((R*)hrec)[soa(i, N, n)] = hd[i];
    }
    collide_store_h<S, QH, CUM, TRT>(hd, hB, n, p, ux, uy, uz, Q, rs);
    }
}

// With many wall nodes the plain 16-bit step runs as two launches: every
// node but the wall nodes, then the wall nodes alone, one thread per entry of
// the wall table, with branch-free link bodies.  A warp that holds wall nodes
// runs the link bodies of the union of its lanes' link directions, each with
// a load round trip behind its branch; packed into warps of their own (the
// porous bed: 11k full warps instead of 94k mixed ones) they cost less, though
// their pulls no longer coalesce.  Measured on the 512x256x256 porous bed
// (D3Q7 h): FP16 22.3k -> 23.6k MLUPS; FP32 20.2k -> 20.1k, so FP32 and FP64
// keep one launch.  Results are those of the single launch bit for bit.
// Threshold: a wall node per LBM_WALL_SPLIT_NODES nodes or more.
#ifndef LBM_WALL_SPLIT_NODES
#define LBM_WALL_SPLIT_NODES 400
#endif
template <typename S, int QH, bool CUM, bool EQ, bool TRT>
void launch_plain_step(const Buffers& b, const DevParams& p, cudaStream_t s) {
    using R = typename Acc<S>::R;
    const int grid = (p.N + kBlock - 1) / kBlock;
#define LBM_PLAIN_ARGS                                                                                           \
    (const S*)b.fA, (S*)b.fB, (const S*)b.hA, (S*)b.hB, b.flags, b.theta, (const R*)b.inlet_post, b.seg_base, \
        b.wmask, b.woff, b.lq, b.lwall, b.Twall, nullptr, nullptr, nullptr, b.wnode, p
    if constexpr (sizeof(S) == 2) {
        if (p.nwall > 0 && (int64_t)p.nwall * LBM_WALL_SPLIT_NODES >= (int64_t)p.N) {
            k_step<S, QH, true, false, CUM, EQ, false, TRT, 1><<<grid, kBlock, 0, s>>>(LBM_PLAIN_ARGS);
            k_step<S, QH, true, false, CUM, EQ, false, TRT, 2>
                <<<(p.nwall + kBlock - 1) / kBlock, kBlock, 0, s>>>(LBM_PLAIN_ARGS);
            return;
        }
    }
    k_step<S, QH, true, false, CUM, EQ, false, TRT, 0><<<grid, kBlock, 0, s>>>(LBM_PLAIN_ARGS);
#undef LBM_PLAIN_ARGS
}

template <typename S, int QH>
cudaError_t launch_step(const Buffers& b, const DevParams& p, cudaStream_t s, bool advance_h) {
    using R = typename Acc<S>::R;
    const int grid = (p.N + kBlock - 1) / kBlock;
    R* urec = (R*)b.urec;
#define LBM_STEP_ARGS                                                                                            \
    (const S*)b.fA, (S*)b.fB, (const S*)b.hA, (S*)b.hB, b.flags, b.theta, (const R*)b.inlet_post, b.seg_base, \
        b.wmask, b.woff, b.lq, b.lwall, b.Twall, urec, b.frec, b.hrec, b.wnode, p
    const bool cum = p.hkind == 3, eq = p.wall_bc == 1;
    if (b.frec) {  // pre-collision records for the coupled adjoint (R-typed storage only)
        if constexpr (sizeof(S) == sizeof(R)) {
            const int v = (cum ? 2 : 0) | (eq ? 1 : 0);
            switch (v) {
                case 0:  // CM-TRT: the same compile-time-rate collision as the plain step, so
                         // recorded levels and plain steps give the same bits
                    if (p.hkind == 0)
                        k_step<S, QH, true, false, false, false, true, true><<<grid, kBlock, 0, s>>>(LBM_STEP_ARGS);
                    else
                        k_step<S, QH, true, false, false, false, true><<<grid, kBlock, 0, s>>>(LBM_STEP_ARGS);
                    break;
                case 1: k_step<S, QH, true, false, false, true, true><<<grid, kBlock, 0, s>>>(LBM_STEP_ARGS); break;
                case 2: k_step<S, QH, true, false, true, false, true><<<grid, kBlock, 0, s>>>(LBM_STEP_ARGS); break;
                default: k_step<S, QH, true, false, true, true, true><<<grid, kBlock, 0, s>>>(LBM_STEP_ARGS); break;
            }
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;
        }
    }
    if (advance_h) {
        const int v = (urec ? 4 : 0) | (cum ? 2 : 0) | (eq ? 1 : 0);
        switch (v) {
            case 0:
                if (p.hkind == 0) launch_plain_step<S, QH, false, false, true>(b, p, s);
                else launch_plain_step<S, QH, false, false, false>(b, p, s);
                break;
            case 1: launch_plain_step<S, QH, false, true, false>(b, p, s); break;
            case 2: launch_plain_step<S, QH, true, false, false>(b, p, s); break;
            case 3: launch_plain_step<S, QH, true, true, false>(b, p, s); break;
            case 4: k_step<S, QH, true, true, false, false><<<grid, kBlock, 0, s>>>(LBM_STEP_ARGS); break;
            case 5: k_step<S, QH, true, true, false, true><<<grid, kBlock, 0, s>>>(LBM_STEP_ARGS); break;
            case 6: k_step<S, QH, true, true, true, false><<<grid, kBlock, 0, s>>>(LBM_STEP_ARGS); break;
            default: k_step<S, QH, true, true, true, true><<<grid, kBlock, 0, s>>>(LBM_STEP_ARGS); break;
        }
    }
    else if (urec) k_step<S, QH, false, true><<<grid, kBlock, 0, s>>>(LBM_STEP_ARGS);
    else k_step<S, QH, false, false><<<grid, kBlock, 0, s>>>(LBM_STEP_ARGS);
#undef LBM_STEP_ARGS
    return cudaGetLastError();
}

// ---- initialisation: equilibria, App. D shift, one collision -------------
template <typename S, int QH, bool CUM = false>
__global__ void __launch_bounds__(kBlock) k_init(S* __restrict__ fB, S* __restrict__ hB,
                                                  const uint8_t* __restrict__ flags, const float* __restrict__ theta,
                                                  const typename Acc<S>::R* __restrict__ inlet,
                                                  const double* __restrict__ rho, const double* __restrict__ u,
                                                  const double* __restrict__ T, const DevParams p) {
    using R = typename Acc<S>::R;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const int type = flags[n] & 3;
    if (type == T_SOLID) {
#pragma unroll
        for (int a = 0; a < 27; ++a) st(fB + (size_t)a * p.N + n, R(0));
#pragma unroll
        for (int i = 0; i < QH; ++i) st(hB + (size_t)i * p.N + n, R(0));
        return;
    }
    if (type == T_INLET) {
#pragma unroll
        for (int a = 0; a < 27; ++a) st(fB + (size_t)a * p.N + n, inlet[a]);
#pragma unroll
        for (int i = 0; i < QH; ++i) st(hB + (size_t)i * p.N + n, inlet[27 + i]);
        return;
    }
    const R vx = (R)u[n], vy = (R)u[(size_t)p.N + n], vz = (R)u[2 * (size_t)p.N + n];
    const R Q = theta ? (R)theta[n] : R(0);
    R fd[27];
    feq_dev<R>(fd, (R)(rho[n] - p.rho0), vx, vy, vz, p);
    // h = h^eq(rho T, u) - q/2 with q = h^eq(Q, u): one equilibrium at rho T - Q/2
    R hd[QH];
    heq_dev<R, QH>(hd, (R)(rho[n] * T[n] - p.Tref) - R(0.5) * Q, vx, vy, vz, p);
    R ux, uy, uz;
    SrStream rs{sr_bits((uint32_t)n, p.step_ctr ? *p.step_ctr : p.step)};
    collide_store_f<S, QH>(fd, fB, n, p, ux, uy, uz, rs);
    collide_store_h<S, QH, CUM>(hd, hB, n, p, ux, uy, uz, Q, rs);
}

template <typename S, int QH>
cudaError_t launch_init(const Buffers& b, const DevParams& p, const double* rho, const double* u, const double* T,
                        cudaStream_t s) {
    using R = typename Acc<S>::R;
    const int grid = (p.N + kBlock - 1) / kBlock;
    if (p.hkind == 3)
        k_init<S, QH, true><<<grid, kBlock, 0, s>>>((S*)b.fB, (S*)b.hB, b.flags, b.theta, (const R*)b.inlet_post, rho,
                                                    u, T, p);
    else
        k_init<S, QH><<<grid, kBlock, 0, s>>>((S*)b.fB, (S*)b.hB, b.flags, b.theta, (const R*)b.inlet_post, rho, u, T,
                                              p);
    return cudaGetLastError();
}

// ---- macroscopic fields from the post-collision state --------------------
// conservation gives rho = sum f*, u = (sum e f* - F/2)/rho,
// H = sum h* - Q/2 (App. D), T = H / rho
template <typename S, int QH>
__global__ void k_macros(const S* __restrict__ fA, const S* __restrict__ hA, const uint8_t* __restrict__ flags,
                         const float* __restrict__ theta, double* __restrict__ rho, double* __restrict__ u,
                         double* __restrict__ T, const DevParams p) {
    using R = typename Acc<S>::R;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const int type = flags[n] & 3;
    const size_t N = (size_t)p.N;
    if (type == T_SOLID) {
        rho[n] = 0.0; u[n] = 0.0; u[N + n] = 0.0; u[2 * N + n] = 0.0; T[n] = 0.0;
        return;
    }
    if (type == T_INLET) {
        rho[n] = 1.0; u[n] = p.uin[0]; u[N + n] = p.uin[1]; u[2 * N + n] = p.uin[2]; T[n] = p.Tin;
        return;
    }
    R dr = 0, jx = 0, jy = 0, jz = 0, dh = 0;
#pragma unroll
    for (int a = 0; a < 27; ++a) {
        const R v = ld<R>(fA + a * N + n);
        dr += v;
        jx += EX(a) * v;
        jy += EY(a) * v;
        jz += EZ(a) * v;
    }
#pragma unroll
    for (int i = 0; i < QH; ++i) dh += ld<R>(hA + i * N + n);
    const R r = par<R>(p.rho0, p.pf.rho0) + dr;
    const R Q = theta ? (R)theta[n] : R(0);
    rho[n] = (double)r;
    u[n] = (double)((jx - R(0.5) * par<R>(p.F[0], p.pf.F[0])) / r);
    u[N + n] = (double)((jy - R(0.5) * par<R>(p.F[1], p.pf.F[1])) / r);
    u[2 * N + n] = (double)((jz - R(0.5) * par<R>(p.F[2], p.pf.F[2])) / r);
    T[n] = (double)((par<R>(p.Tref, p.pf.Tref) + dh - R(0.5) * Q) / r);
}

template <typename S, int QH>
cudaError_t launch_macros(const Buffers& b, const DevParams& p, double* rho, double* u, double* T, cudaStream_t s) {
    const int grid = (p.N + kBlock - 1) / kBlock;
    k_macros<S, QH><<<grid, kBlock, 0, s>>>((const S*)b.fA, (const S*)b.hA, b.flags, b.theta, rho, u, T, p);
    return cudaGetLastError();
}

template <typename S, int QH>
__global__ void k_populations(const S* __restrict__ fA, const S* __restrict__ hA, const uint8_t* __restrict__ flags,
                              double* __restrict__ f, double* __restrict__ h, const DevParams p) {
    using R = typename Acc<S>::R;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const bool solid = (flags[n] & 3) == T_SOLID;
    const size_t N = (size_t)p.N;
    if (f) {
#pragma unroll
        for (int a = 0; a < 27; ++a)
            f[a * N + n] = solid ? 0.0 : (double)ld<R>(fA + a * N + n) + W27(a) * p.rho0;
    }
    if (h) {
#pragma unroll
        for (int i = 0; i < QH; ++i)
            h[i * N + n] = solid ? 0.0 : (double)ld<R>(hA + i * N + n) + HW<QH>(i) * p.Tref;
    }
}

template <typename S, int QH>
cudaError_t launch_populations(const Buffers& b, const DevParams& p, double* f, double* h, cudaStream_t s) {
    const int grid = (p.N + kBlock - 1) / kBlock;
    k_populations<S, QH><<<grid, kBlock, 0, s>>>((const S*)b.fA, (const S*)b.hA, b.flags, f, h, p);
    return cudaGetLastError();
}

// ---- reductions: warp shuffle -> block -> per-block partials -> one block --
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[wid * NV + k] = v[k];
    __syncthreads();
    if (wid == 0) {
        const int nwarps = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = (lane < nwarps) ? sh[lane * NV + k] : 0.0;
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
}

template <int NV>
__global__ void k_reduce_partials(const double* __restrict__ part, int nparts, double* __restrict__ out) {
    __shared__ double sh[32 * NV];
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += part[i * NV + k];
    block_sum<NV>(v, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = v[k];
}

// sums of the deviations (rho - rho0, H - Tref) and of non-finite values over
// non-solid nodes; the host adds rho0 and Tref times the node count
template <typename S, int QH>
__global__ void __launch_bounds__(kRedThreads) k_balances(const S* __restrict__ fA, const S* __restrict__ hA,
                                                          const uint8_t* __restrict__ flags,
                                                          const float* __restrict__ theta,
                                                          double* __restrict__ part, const DevParams p) {
    using R = typename Acc<S>::R;
    __shared__ double sh[32 * 3];
    double v[3] = {0.0, 0.0, 0.0};
    const size_t N = (size_t)p.N;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < p.N; n += gridDim.x * blockDim.x) {
        if ((flags[n] & 3) == T_SOLID) continue;
        // every stored value is added in FP64 (no FP32 partial sums)
        bool bad = false;
#pragma unroll
        for (int a = 0; a < 27; ++a) {
            const R x = ld<R>(fA + a * N + n);
            bad |= !isfinite(x);
            v[0] += (double)x;
        }
#pragma unroll
        for (int i = 0; i < QH; ++i) {
            const R x = ld<R>(hA + i * N + n);
            bad |= !isfinite(x);
            v[1] += (double)x;
        }
        if (theta) v[1] -= 0.5 * (double)theta[n];
        v[2] += bad ? 1.0 : 0.0;
    }
    block_sum<3>(v, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) part[blockIdx.x * 3 + k] = v[k];
}

template <typename S, int QH>
cudaError_t launch_balances(const Buffers& b, const DevParams& p, double* scratch, double* out, cudaStream_t s) {
    k_balances<S, QH><<<kRedBlocks, kRedThreads, 0, s>>>((const S*)b.fA, (const S*)b.hA, b.flags, b.theta, scratch, p);
    k_reduce_partials<3><<<1, 1024, 0, s>>>(scratch, kRedBlocks, out);
    return cudaGetLastError();
}

// surface heat flux of one wall (Sec. 4.4): for every IABB link of the wall,
// h_ibar(x_b, t+1) from Eq. IABB minus h*_i(x_b, t); the shifts cancel
template <typename S, int QH>
__global__ void __launch_bounds__(kRedThreads) k_surface_flux(const S* __restrict__ hA,
                                                              const int32_t* __restrict__ wnode,
                                                              const uint32_t* __restrict__ wmask,
                                                              const int32_t* __restrict__ woff,
                                                              const float* __restrict__ lq,
                                                              const int32_t* __restrict__ lwall,
                                                              const float* __restrict__ Twall, int nw, int wall,
                                                              double* __restrict__ part, const DevParams p) {
    using R = typename Acc<S>::R;
    __shared__ double sh[32];
    double v[1] = {0.0};
    const size_t N = (size_t)p.N;
    const R Tref = par<R>(p.Tref, p.pf.Tref);
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
        const int n = wnode[w];
        const uint32_t mask = wmask[w];
        const int off = woff[w];
        int x, y, z;
        node_xyz(n, p, x, y, z);
        const Nbr nb = make_nbr(x, y, z, p);
#pragma unroll
        for (int ia = 0; ia < QH; ++ia) {
            const int a = HDIR<QH>(ia);
            if (!(mask & (1u << a))) continue;
            const int l = off + __popc(mask & ((1u << a) - 1u));
            if (lwall[l] != wall) continue;
            const int ib = HOPP<QH>(ia);
            const int b = HDIR<QH>(ib);
            const float q = lq[l];
            const R heq2 = R(2) * (R)HW<QH>(ia) * ((R)Twall[wall] - Tref);
            const bool thin = (mask >> b) & 1u;
            const R ha_b = ld<R>(hA + ia * N + n);
            R hin;
            if (p.wall_bc == 1) {
                hin = R(0.5) * heq2;
            } else if (q <= 0.5f && !thin) {
                const R ha_f = ld<R>(hA + ia * N + src_of(nb, a));
                hin = -(R(2) * (R)q * ha_b + (R(1) - R(2) * (R)q) * ha_f) + heq2;
            } else {
                const R qq = (R)fmaxf(q, 0.5f);
                const R hb_b = ld<R>(hA + ib * N + n);
                hin = (-ha_b + (R(2) * qq - R(1)) * hb_b + heq2) / (R(2) * qq);
            }
            v[0] += (double)hin - (double)ha_b;
        }
    }
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

template <typename S, int QH>
cudaError_t launch_surface_flux(const Buffers& b, const DevParams& p, int wall, double* scratch, double* out,
                                cudaStream_t s) {
    k_surface_flux<S, QH><<<kRedBlocks, kRedThreads, 0, s>>>((const S*)b.hA, b.wnode, b.wmask, b.woff, b.lq, b.lwall,
                                                            b.Twall, b.nw, wall, scratch, p);
    k_reduce_partials<1><<<1, 1024, 0, s>>>(scratch, kRedBlocks, out);
    return cudaGetLastError();
}

// force on one wall by momentum exchange (Ladd 1994, Mei et al. 2002; not in
// the paper): every link (x_b, a) of the wall carries e_a f*_a(x_b, t) into
// the wall and takes back e_a f_abar(x_b, t+1) from Eq. IBB, exactly as the
// step applies it; the stored deviations add 2 w_a rho0 per link
template <typename S>
__global__ void __launch_bounds__(kRedThreads) k_wall_force(const S* __restrict__ fA,
                                                            const int32_t* __restrict__ wnode,
                                                            const uint32_t* __restrict__ wmask,
                                                            const int32_t* __restrict__ woff,
                                                            const float* __restrict__ lq,
                                                            const int32_t* __restrict__ lwall, int nw, int wall,
                                                            double* __restrict__ part, const DevParams p) {
    using R = typename Acc<S>::R;
    __shared__ double sh[3 * 32];
    double v[3] = {0.0, 0.0, 0.0};
    const size_t N = (size_t)p.N;
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
        const int n = wnode[w];
        const uint32_t mask = wmask[w];
        const int off = woff[w];
        int x, y, z;
        node_xyz(n, p, x, y, z);
        const Nbr nb = make_nbr(x, y, z, p);
#pragma unroll
        for (int a = 1; a < 27; ++a) {
            if (!(mask & (1u << a))) continue;
            const int l = off + __popc(mask & ((1u << a) - 1u));
            if (lwall[l] != wall) continue;
            const int b = OPP(a);
            const float q = lq[l];
            const bool thin = (mask >> b) & 1u;  // x_f = x_b - e_a is solid
            const R fa_b = ld<R>(fA + a * N + n);
            R fin;
            if (q <= 0.5f && !thin) {
                fin = R(2) * (R)q * fa_b + (R(1) - R(2) * (R)q) * ld<R>(fA + a * N + src_of(nb, a));
            } else {
                const R qq = (R)fmaxf(q, 0.5f);
                fin = (fa_b + (R(2) * qq - R(1)) * ld<R>(fA + b * N + n)) / (R(2) * qq);
            }
            const double carried = (double)fa_b + (double)fin + 2.0 * W27(a) * p.rho0;
            v[0] += EX(a) * carried;
            v[1] += EY(a) * carried;
            v[2] += EZ(a) * carried;
        }
    }
    block_sum<3>(v, sh);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = v[0];
        part[3 * blockIdx.x + 1] = v[1];
        part[3 * blockIdx.x + 2] = v[2];
    }
}

template <typename S, int QH>
cudaError_t launch_wall_force(const Buffers& b, const DevParams& p, int wall, double* scratch, double* out,
                              cudaStream_t s) {
    k_wall_force<S><<<kRedBlocks, kRedThreads, 0, s>>>((const S*)b.fA, b.wnode, b.wmask, b.woff, b.lq, b.lwall,
                                                      b.nw, wall, scratch, p);
    k_reduce_partials<3><<<1, 1024, 0, s>>>(scratch, kRedBlocks, out);
    return cudaGetLastError();
}

// ---- adjoint of the h evolution --------------------------------------------
// With u fixed (one-way coupling), one step is g^{k+1} = P s^k + b(T_w) and
// s^{k+1} = L(u^{k+1}) g^{k+1} + e(u^{k+1}) theta, with
// L = T^-1 (1 - S) T + T^-1 S E 1^T and e = T^-1 E (Eq. H_cm_collision and
// the App. D source).  One call computes, per node y,
//   lambda^k(y) = (P^T mu^{k+1})(y) + dJ_k/ds^k(y)           (gather)
//   mu^k(y)     = L(u^k)^T lambda^k = T^T (1-S) z + 1 (E^T S z),  z = T^-T lambda
//   dJ/dtheta(y) += E^T z,   dJ/dT_w(link) += (db/dT_w) mu^{k+1}
// P^T is a pull from y + e_a (the transpose of the forward pull), plus the
// Eq. IABB partials of the wall links that read y.

// transposes of the 3-point maps fwd3 / inv3 (same slot conventions)
template <typename R> __device__ __forceinline__ void fwd3T(R& a, R& b, R& c, R v) {
    const R m0 = a - v * b + v * v * c;
    const R m1 = b - R(2) * v * c;
    const R m2 = c;
    a = m0 - m1 + m2;
    b = m0;
    c = m0 + m1 + m2;
}
template <typename R> __device__ __forceinline__ void inv3T(R& a, R& b, R& c, R v) {
    const R m2 = R(0.5) * (a + c) - b;
    const R m1 = R(0.5) * (c - a);
    const R m0 = b;
    a = m0 + v * m1 + v * v * m2;
    b = m1 + R(2) * v * m2;
    c = m2;
}

// partial derivatives of one Eq. IABB arrival with respect to h*_a(x_b),
// h*_abar(x_b) and T_w (the latter per unit weight w_a)
template <typename R>
__device__ __forceinline__ void iabb_partials(float q, bool thin, int wall_bc, R& d_ab, R& d_abb, R& d_T) {
    if (wall_bc == 1) {  // EQ: the arrival is w T_w
        d_ab = R(0); d_abb = R(0); d_T = R(1);
    } else if (q <= 0.5f && !thin) {
        d_ab = -R(2) * (R)q; d_abb = R(0); d_T = R(2);
    } else {
        const R qq = (R)fmaxf(q, 0.5f);
        d_ab = -R(1) / (R(2) * qq); d_abb = (R(2) * qq - R(1)) / (R(2) * qq); d_T = R(2) / (R(2) * qq);
    }
}

// Pieces of the D3Q27 central-moment transposes, shared by the h-only and
// the coupled adjoint: cube slots of z = T(u)^-T lambda (from the cube of
// lambda) and mu = L(u)^T lambda from z (Eq. H_cm_collision transposed: the
// per-order relaxation, the rank-one equilibrium term, then T(u)^T).
template <typename R> __device__ __forceinline__ void z_from_lambda27(R* cb, R ux, R uy, R uz) {
#pragma unroll
    for (int j = 0; j < 9; ++j) inv3T<R>(cb[3 * j], cb[3 * j + 1], cb[3 * j + 2], ux);
#pragma unroll
    for (int zz = 0; zz < 3; ++zz)
#pragma unroll
        for (int xx = 0; xx < 3; ++xx) inv3T<R>(cb[9 * zz + xx], cb[9 * zz + 3 + xx], cb[9 * zz + 6 + xx], uy);
#pragma unroll
    for (int j = 0; j < 9; ++j) inv3T<R>(cb[j], cb[9 + j], cb[18 + j], uz);
}
template <typename R>
__device__ __forceinline__ void transpose_from_z27(R* cb, R ux, R uy, R uz, const DevParams& p, R* mu,
                                                   double& dth) {
    R rank = R(0);
#pragma unroll
    for (int o = 0; o < 3; ++o)
#pragma unroll
        for (int nn = 0; nn < 3; ++nn)
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const R E = Eq<R>(m, nn, o);
                const R sr = par<R>(p.sh[m + nn + o], p.pf.sh[m + nn + o]);
                R& v = cb[MIDX(m, nn, o)];
                if (E != R(0)) {
                    dth += (double)(E * v);
                    rank += E * sr * v;
                }
                v *= (R(1) - sr);
            }
#pragma unroll
    for (int j = 0; j < 9; ++j) fwd3T<R>(cb[3 * j], cb[3 * j + 1], cb[3 * j + 2], ux);
#pragma unroll
    for (int zz = 0; zz < 3; ++zz)
#pragma unroll
        for (int xx = 0; xx < 3; ++xx) fwd3T<R>(cb[9 * zz + xx], cb[9 * zz + 3 + xx], cb[9 * zz + 6 + xx], uy);
#pragma unroll
    for (int j = 0; j < 9; ++j) fwd3T<R>(cb[j], cb[9 + j], cb[18 + j], uz);
#pragma unroll
    for (int a = 0; a < 27; ++a) mu[a] = cb[CUBE(a)] + rank;
}

// The transposed Jacobian of one node's h collision at velocity u (fixed):
// mu = (dC_h/dg)^T lambda and dth = (dC_h/dQ)^T lambda.  Central-moment kinds:
// C_h = L(u) g + e(u) Q (Eq. H_cm_collision, App. D source), transposed
// exactly; Cumulants-1st: the Jacobian of (H + Q) M(v) at the state whose
// post-collision deviations are hpost (Eq. H_cu_collision).
template <typename R, int QH, bool CUM>
__device__ __forceinline__ void h_collision_transpose(const R* lam, const R* hpost, const R ux, const R uy,
                                                      const R uz, const R Q, const DevParams& p, R* mu,
                                                      double& dth) {
    dth = 0.0;
    if constexpr (CUM) {
        // Cumulants-1st (Eq. H_cu_collision): s^k = (H + Q) M(v), M the unit
        // equilibrium at v = (1 - s) m + s u, m = sum e g / H, H = sum g of the
        // arrivals g.  From the recorded s^k: A = H + Q = sum s^k and
        // v = sum e s^k / A, and (1 - s) m = v - s u.  The transposed Jacobian
        //   mu_b = L0 + A/H sum_d ((1 - s) e_bd - (v_d - s u_d)) G_d,
        //   L0 = sum_a lambda_a M_a(v),  G_d = sum_a lambda_a dM_a/dv_d,
        // and dJ/dQ += L0.
        R A = par<R>(p.Tref, p.pf.Tref), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
        for (int i = 0; i < QH; ++i) {
            const int a = HDIR<QH>(i);
            const R g = hpost[i];
            A += g;
            if (EX(a) != 0) jx += EX(a) * g;
            if (EY(a) != 0) jy += EY(a) * g;
            if (EZ(a) != 0) jz += EZ(a) * g;
        }
        const R iA = R(1) / A;
        const R v[3] = {jx * iA, jy * iA, jz * iA};
        const R u[3] = {ux, uy, uz};
        const R c = cs2<R>();
        // per axis: unit-equilibrium factors and their v-derivatives at c = -1, 0, +1
        R W[3][3], D[3][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const R a2 = c + v[d] * v[d];
            W[d][0] = R(0.5) * (a2 - v[d]);
            W[d][1] = R(1) - a2;
            W[d][2] = R(0.5) * (a2 + v[d]);
            D[d][0] = v[d] - R(0.5);
            D[d][1] = R(-2) * v[d];
            D[d][2] = v[d] + R(0.5);
        }
        R L0 = R(0), G[3] = {R(0), R(0), R(0)};
        if constexpr (QH == 27) {
#pragma unroll
            for (int a = 0; a < 27; ++a) {
                const int cx = EX(a) + 1, cy = EY(a) + 1, cz = EZ(a) + 1;
                const R l = lam[a];
                L0 += l * W[0][cx] * W[1][cy] * W[2][cz];
                G[0] += l * D[0][cx] * W[1][cy] * W[2][cz];
                G[1] += l * W[0][cx] * D[1][cy] * W[2][cz];
                G[2] += l * W[0][cx] * W[1][cy] * D[2][cz];
            }
        } else {
            // D3Q7 unit equilibrium: rest 1 - sum_d a2_d, arms (a2_d +- v_d) / 2
            R rest = R(1);
#pragma unroll
            for (int d = 0; d < 3; ++d) rest -= c + v[d] * v[d];
            L0 = lam[0] * rest;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                L0 += lam[1 + d] * W[d][2] + lam[4 + d] * W[d][0];
                G[d] = lam[0] * D[d][1] + lam[1 + d] * D[d][2] + lam[4 + d] * D[d][0];
            }
        }
        const R s = par<R>(p.sh[1], p.pf.sh[1]);
        const R kap = A / (A - Q);
        R base = L0;
#pragma unroll
        for (int d = 0; d < 3; ++d) base -= kap * (v[d] - s * u[d]) * G[d];
        const R c1 = kap * (R(1) - s);
#pragma unroll
        for (int i = 0; i < QH; ++i) {
            const int a = HDIR<QH>(i);
            mu[i] = base + c1 * (EX(a) * G[0] + EY(a) * G[1] + EZ(a) * G[2]);
        }
        dth = (double)L0;
    } else if constexpr (QH == 27) {
        R cb[27];
#pragma unroll
        for (int a = 0; a < 27; ++a) cb[CUBE(a)] = lam[a];
        z_from_lambda27<R>(cb, ux, uy, uz);
        transpose_from_z27<R>(cb, ux, uy, uz, p, mu, dth);
    } else {
        // D3Q7: moments 000, 100/010/001, 200/020/002
        const R u[3] = {ux, uy, uz};
        const R c = cs2<R>();
        // z = T^-T lambda (transpose of the D3Q7 inverse transform of collide_h7)
        R z0 = lam[0], z1[3], z2[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const R mb2 = R(0.5) * (lam[1 + d] + lam[4 + d]) - lam[0];
            const R mb1 = R(0.5) * (lam[1 + d] - lam[4 + d]);
            z2[d] = mb2;
            z1[d] = mb1 + R(2) * u[d] * mb2;
            z0 += u[d] * mb1 + u[d] * u[d] * mb2;
        }
        const R s0 = par<R>(p.sh[0], p.pf.sh[0]), s1 = par<R>(p.sh[1], p.pf.sh[1]), s2 = par<R>(p.sh[2], p.pf.sh[2]);
        dth = (double)z0 + (double)(c * (z2[0] + z2[1] + z2[2]));
        const R rank = s0 * z0 + s2 * c * (z2[0] + z2[1] + z2[2]);
        z0 *= (R(1) - s0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            z1[d] *= (R(1) - s1);
            z2[d] *= (R(1) - s2);
        }
        // T^T z: population i gets z0 + sum_d (e_id - u_d) z1_d + (e_id - u_d)^2 z2_d
        R base = z0;
#pragma unroll
        for (int d = 0; d < 3; ++d) base += -u[d] * z1[d] + u[d] * u[d] * z2[d];
        mu[0] = base + rank;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const R rest_d = -u[d] * z1[d] + u[d] * u[d] * z2[d];
            const R plus = (R(1) - u[d]) * z1[d] + (R(1) - u[d]) * (R(1) - u[d]) * z2[d];
            const R minus = (R(-1) - u[d]) * z1[d] + (R(1) + u[d]) * (R(1) + u[d]) * z2[d];
            mu[1 + d] = base - rest_d + plus + rank;
            mu[4 + d] = base - rest_d + minus + rank;
        }
    }
}

// Transpose of the Zou-He rule for h at an inlet node (k_inlet), the density
// (from f) held fixed: an unknown arrival j (e_x = +1) is the equilibrium at
// u_in with the amplitude that closes sum h = rho T_in, so it depends on the
// known arrivals k (e_x <= 0) through -M_j(u_in) / M_+(u_in) per unit, M the
// unit equilibrium and M_+ the sum of M over the unknowns; in product form
// that ratio is w(e_y, u_y) w(e_z, u_z) (D3Q7: 1).  mu holds the adjoint of
// the node's full arrival vector and becomes that of its known arrivals (the
// unknown ones are pulled from nowhere and get 0).
template <typename R>
__device__ __forceinline__ R w1_unit(int e, R u) {
    return e == 0 ? R(1) - u * u - cs2<R>() : R(0.5) * (u * u + R(e) * u + cs2<R>());
}
template <typename R, int QH>
__device__ __forceinline__ void zou_he_h_transpose(R* mu, const DevParams& p) {
    const R uy = par<R>(p.uin[1], p.pf.uin[1]), uz = par<R>(p.uin[2], p.pf.uin[2]);
    R sum = R(0);
#pragma unroll
    for (int i = 0; i < QH; ++i) {
        const int a = HDIR<QH>(i);
        if (EX(a) != 1) continue;
        sum += (QH == 27 ? w1_unit<R>(EY(a), uy) * w1_unit<R>(EZ(a), uz) : R(1)) * mu[i];
    }
#pragma unroll
    for (int i = 0; i < QH; ++i) mu[i] = (EX(HDIR<QH>(i)) == 1) ? R(0) : mu[i] - sum;
}

template <typename R, int QH, bool CUM = false>
__global__ void __launch_bounds__(kBlock) k_adjoint(const R* __restrict__ mu_next, R* __restrict__ out,
                                                     const R* __restrict__ uk, const R* __restrict__ hk,
                                                     const float* __restrict__ theta, double* __restrict__ dtheta,
                                                     const uint8_t* __restrict__ flags,
                                                     const int32_t* __restrict__ seg_base,
                                                     const uint32_t* __restrict__ wmask,
                                                     const int32_t* __restrict__ woff, const float* __restrict__ lq,
                                                     const int32_t* __restrict__ lwall,
                                                     const int32_t* __restrict__ rseg_base,
                                                     const uint32_t* __restrict__ rmask,
                                                     const int32_t* __restrict__ roff,
                                                     const int32_t* __restrict__ rlink, double* __restrict__ dlink,
                                                     const AdjObjective obj, const DevParams p) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in_range = n < p.N;
    const uint8_t fl = in_range ? flags[n] : (uint8_t)T_SOLID;
    const bool is_wall = (fl & F_WALL) != 0, is_rw = (fl & F_RWALL) != 0;
    const uint32_t bal_w = __ballot_sync(0xffffffffu, is_wall);
    const uint32_t bal_r = __ballot_sync(0xffffffffu, is_rw);
    if (!in_range) return;
    const int N = p.N;
    const int type = fl & 3;
    // a Zou-He inlet node streams and collides like a fluid node
    if (type == T_SOLID || (type == T_INLET && !p.zou_he)) {
#pragma unroll
        for (int i = 0; i < QH; ++i) out[soa(i, N, n)] = R(0);
        return;
    }
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    int x, y, z;
    node_xyz(n, p, x, y, z);
    // symmetry rows: the row beside a symmetry row reads its own populations,
    // e_y reversed, through the row's copies (k_mirror), so a push into a
    // symmetry row lands on this row with the mirrored velocity
    const bool rlo = p.mirror_lo && y == 1, rhi = p.mirror_hi && y == p.ny - 2;
    // push neighbours: index 0 <-> e = -1, 2 <-> e = +1; -1 when outside a bounded x
    int xt[3] = {x - 1, x, x + 1};
    if (p.periodic_x) {
        if (xt[0] < 0) xt[0] += p.nx;
        if (xt[2] >= p.nx) xt[2] -= p.nx;
    } else {
        if (xt[0] < 0) xt[0] = -1;
        if (xt[2] >= p.nx) xt[2] = -1;
    }
    const int yt[3] = {((y == 0) ? p.ny - 1 : y - 1) * p.nx, y * p.nx, ((y == p.ny - 1) ? 0 : y + 1) * p.nx};
    const int pl = p.nx * p.ny;
    const int zt[3] = {((z == 0) ? p.nz - 1 : z - 1) * pl, z * pl, ((z == p.nz - 1) ? 0 : z + 1) * pl};
    const R wsurf = (obj.kind == 0) ? (R)obj.weight : R(0);
    // mu_next is zero at solid and inlet nodes (this kernel writes zeros
    // there), which are exactly the nodes that pull nothing: no flag test
    R lam[QH];
#pragma unroll
    for (int i = 0; i < QH; ++i) {
        const int a = HDIR<QH>(i);
        const int xx = xt[EX(a) + 1];
        const bool refl = (EY(a) == -1 && rlo) || (EY(a) == 1 && rhi);
        const int row = refl ? y * p.nx : yt[EY(a) + 1];
        const int ii = refl ? HFLIPY<QH>(i) : i;
        lam[i] = (xx < 0) ? R(0) : __ldg(mu_next + soa(ii, N, xx + row + zt[EZ(a) + 1]));
    }
    if (!p.periodic_x && x == p.nx - 1) {
        // outlet plane: its incoming e_x < 0 populations copy this node's value
#pragma unroll
        for (int i = 0; i < QH; ++i) {
            const int a = HDIR<QH>(i);
            if (EX(a) != -1) continue;
            const bool refl = (EY(a) == -1 && rlo) || (EY(a) == 1 && rhi);
            const int t = x + (refl ? y * p.nx : yt[EY(a) + 1]) + zt[EZ(a) + 1];
            lam[i] += mu_next[(refl ? HFLIPY<QH>(i) : i) * N + t];
        }
    }
    if (is_rw) {
        // this node is x_f of links (t = y + e_a, a) with q <= 1/2
        const int idx = __ldg(rseg_base + (n >> 5)) + __popc(bal_r & lt);
        const uint32_t rm = __ldg(rmask + idx);
        const int ro = __ldg(roff + idx);
#pragma unroll
        for (int i = 0; i < QH; ++i) {
            const int a = HDIR<QH>(i);
            if (!(rm & (1u << a))) continue;
            const int l = __ldg(rlink + ro + __popc(rm & ((1u << a) - 1u)));
            const float q = __ldg(lq + l);
            const R cw = (__ldg(lwall + l) == obj.wall) ? wsurf : R(0);
            const int t = xt[EX(a) + 1] + yt[EY(a) + 1] + zt[EZ(a) + 1];
            lam[i] -= (R(1) - R(2) * (R)q) * (mu_next[HOPP<QH>(i) * N + t] + cw);
        }
    }
    if (is_wall) {
        const int idx = __ldg(seg_base + (n >> 5)) + __popc(bal_w & lt);
        const uint32_t mask = __ldg(wmask + idx);
        const int off = __ldg(woff + idx);
#pragma unroll
        for (int i = 0; i < QH; ++i) {
            const int b = HDIR<QH>(i);
            if (!(mask & (1u << b))) continue;
            const int ib = HOPP<QH>(i);
            const int l = off + __popc(mask & ((1u << b) - 1u));
            const float q = __ldg(lq + l);
            const R cw = (__ldg(lwall + l) == obj.wall) ? wsurf : R(0);
            const bool thin = (mask >> HDIR<QH>(ib)) & 1u;
            R d_ab, d_abb, d_T;
            iabb_partials<R>(q, thin, p.wall_bc, d_ab, d_abb, d_T);
            const R m = mu_next[ib * N + n] + cw;
            lam[i] += d_ab * m - cw;
            lam[ib] += d_abb * m;
            dlink[l] += (double)d_T * HW<QH>(i) * (double)m;
        }
    }
    if (obj.kind == 1 && x == obj.plane) {
#pragma unroll
        for (int i = 0; i < QH; ++i) lam[i] += (R)obj.weight * (R)EX(HDIR<QH>(i));
    }
    if (!uk) {
#pragma unroll
        for (int i = 0; i < QH; ++i) out[soa(i, N, n)] = lam[i];
        return;
    }
    const R ux = uk[n], uy = uk[N + n], uz = uk[2 * N + n];
    double dth = 0.0;
    {
        R mu[QH], hp[QH];
        if constexpr (CUM) {
#pragma unroll
            for (int i = 0; i < QH; ++i) hp[i] = hk[soa(i, N, n)];
        }
        const R Q = theta ? (R)__ldg(theta + n) : R(0);
        h_collision_transpose<R, QH, CUM>(lam, hp, ux, uy, uz, Q, p, mu, dth);
        if (type == T_INLET) zou_he_h_transpose<R, QH>(mu, p);
#pragma unroll
        for (int i = 0; i < QH; ++i) out[soa(i, N, n)] = mu[i];
    }
    if (dtheta) dtheta[n] += dth;
}

template <typename R, int QH>
cudaError_t launch_adjoint(const Buffers& b, const DevParams& p, const R* u_level, const R* h_level,
                           const R* mu_next, R* mu_out, AdjObjective obj, double* dtheta, cudaStream_t s) {
    const int grid = (p.N + kBlock - 1) / kBlock;
#define LBM_ADJ_ARGS                                                                                             \
    mu_next, mu_out, u_level, h_level, b.theta, dtheta, b.flags, b.seg_base, b.wmask, b.woff, b.lq, b.lwall,    \
        b.rseg_base, b.rmask, b.roff, b.rlink, b.dlink, obj, p
    if (p.hkind == 3) k_adjoint<R, QH, true><<<grid, kBlock, 0, s>>>(LBM_ADJ_ARGS);
    else k_adjoint<R, QH, false><<<grid, kBlock, 0, s>>>(LBM_ADJ_ARGS);
#undef LBM_ADJ_ARGS
    return cudaGetLastError();
}

// ---- Zou-He inlet (Sec. 4.4) ------------------------------------------------
// Runs after the step over the inlet plane x = 0 and replaces what the step
// stored there.  Arrivals with e_x <= 0 are pulled from the post-collision
// state A as in the step.  The unknown f (e_x = +1) follow from
// non-equilibrium bounce-back at u_in: f_a = f_abar + f^eq_a - f^eq_abar with
// rho from mass and x-momentum, rho (1 - u_x) = sum_{e_x=0} f + 2 sum_{e_x=-1} f,
// less e_ya N_y + e_za N_z, N_d = sum_{e_x=0} e_d (f - f^eq) / 6, which makes
// the transverse momentum rho u_d exactly.  The unknown h take the shape of the
// equilibrium at u_in with the amplitude that makes sum h = rho T_in.  The
// node then collides and stores like a fluid node.  Everything is in deviation
// form (f - w rho0, h - w T_ref).
// The rule on one node's arrivals (deviation form), with the known ones
// (e_x <= 0) in place: fills the unknown f and returns the density deviation
// (zou_he_fill_f), then the unknown h (zou_he_fill_h).  T is the arithmetic
// type (a dual number differentiates the rule with respect to u_in).
template <typename T>
__device__ __forceinline__ T zou_he_fill_f(T* fd, T ux, T uy, T uz, const DevParams& p) {
    T s0 = T(0), sm = T(0);
#pragma unroll
    for (int a = 0; a < 27; ++a) {
        if (EX(a) == 0) s0 += fd[a];
        if (EX(a) == -1) sm += fd[a];
    }
    // the e_x = 0 and e_x = -1 weights sum to 2/3 and 1/6
    const T drho = (s0 + T(2) * sm + par<T>(p.rho0, p.pf.rho0) * ux) / (T(1) - ux);
    T fe[27];
    feq_dev<T>(fe, drho, ux, uy, uz, p);
    T Ny = T(0), Nz = T(0);
#pragma unroll
    for (int a = 0; a < 27; ++a) {
        if (EX(a) != 0) continue;
        if (EY(a) != 0) Ny += EY(a) * (fd[a] - fe[a]);
        if (EZ(a) != 0) Nz += EZ(a) * (fd[a] - fe[a]);
    }
    Ny *= T(1) / T(6);
    Nz *= T(1) / T(6);
#pragma unroll
    for (int a = 0; a < 27; ++a) {
        if (EX(a) != 1) continue;
        const int b = OPP(a);
        fd[a] = fd[b] + fe[a] - fe[b] - EY(a) * Ny - EZ(a) * Nz;
    }
    return drho;
}
template <typename T, int QH>
__device__ __forceinline__ void zou_he_fill_h(T* hd, T drho, T ux, T uy, T uz, const DevParams& p) {
    T K = T(0);
#pragma unroll
    for (int k = 0; k < QH; ++k)
        if (EX(HDIR<QH>(k)) != 1) K += hd[k];
    // unknown deviations = h^eq(amp, u_in) - w T_ref; with damp = amp - T_ref:
    // damp (c_s^2 + u_x^2 + u_x)/2 = rho T_in - T_ref - K - T_ref (u_x^2 + u_x)/2
    const T Tref = par<T>(p.Tref, p.pf.Tref);
    const T mU = T(0.5) * (cs2<T>() + ux * ux + ux);
    const T target = drho * par<T>(p.Tin, p.pf.Tin) + (T)(p.rho0 * p.Tin - p.Tref);
    const T damp = (target - K - Tref * T(0.5) * (ux * ux + ux)) / mU;
    T he[QH];
    heq_dev<T, QH>(he, damp, ux, uy, uz, p);
#pragma unroll
    for (int k = 0; k < QH; ++k)
        if (EX(HDIR<QH>(k)) == 1) hd[k] = he[k];
}

// frec, hrec: pre-collision records of the coupled adjoint (the f moments and,
// after them, the inlet node's full arrival vector after the rule; the h
// arrivals), or nullptr
template <typename S, int QH, bool CUM, bool DO_H>
__global__ void __launch_bounds__(kBlock) k_inlet(const S* __restrict__ fA, S* __restrict__ fB,
                                                   const S* __restrict__ hA, S* __restrict__ hB,
                                                   const uint8_t* __restrict__ flags,
                                                   const float* __restrict__ theta,
                                                   typename Acc<S>::R* __restrict__ urec, void* __restrict__ frec,
                                                   void* __restrict__ hrec, const DevParams p) {
    using R = typename Acc<S>::R;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.ny * p.nz) return;
    const int y = i % p.ny, z = i / p.ny;
    const int n = p.nx * (y + p.ny * z);  // x = 0
    if ((flags[n] & 3) != T_INLET) return;  // symmetry rows are solid on the device
    const int N = p.N;
    const Nbr nb = make_nbr(0, y, z, p);
    const R ux = par<R>(p.uin[0], p.pf.uin[0]), uy = par<R>(p.uin[1], p.pf.uin[1]), uz = par<R>(p.uin[2], p.pf.uin[2]);
    R fd[27];
#pragma unroll
    for (int a = 0; a < 27; ++a) fd[a] = (EX(a) == 1) ? R(0) : ld<R>(fA + a * N + src_of(nb, a));
    const R drho = zou_he_fill_f<R>(fd, ux, uy, uz, p);
    if (frec) {
        R m[10];
        raw_moments_f<R>(fd, m[0], m[1], m[2], m[3], m[4], m[5], m[6], m[7], m[8], m[9]);
#pragma unroll
        for (int k = 0; k < 10; ++k) ((R*)frec)[k * N + n] = m[k];
        R* inl = (R*)frec + (size_t)10 * N;  // [27][ny nz], row i = y + ny z
#pragma unroll
        for (int a = 0; a < 27; ++a) inl[(size_t)a * p.ny * p.nz + i] = fd[a];
    }
    R vx, vy, vz;
    SrStream rs{sr_bits((uint32_t)n, p.step_ctr ? *p.step_ctr : p.step)};
    collide_store_f<S, QH>(fd, fB, n, p, vx, vy, vz, rs);
    if (urec) {
        urec[n] = vx;
        urec[N + n] = vy;
        urec[2 * N + n] = vz;
    }
    if constexpr (DO_H) {
        R hd[QH];
#pragma unroll
        for (int k = 0; k < QH; ++k) {
            const int a = HDIR<QH>(k);
            hd[k] = (EX(a) == 1) ? R(0) : ld<R>(hA + k * N + src_of(nb, a));
        }
        zou_he_fill_h<R, QH>(hd, drho, ux, uy, uz, p);
        if (hrec) {
#pragma unroll
            for (int k = 0; k < QH; ++k) ((R*)hrec)[k * N + n] = hd[k];
        }
        const R Q = theta ? (R)__ldg(theta + n) : R(0);
        collide_store_h<S, QH, CUM>(hd, hB, n, p, vx, vy, vz, Q, rs);
    }
}

template <typename S, int QH>
cudaError_t launch_inlet(const Buffers& b, const DevParams& p, cudaStream_t s, bool advance_h) {
    using R = typename Acc<S>::R;
    const int total = p.ny * p.nz;
    const int grid = (total + kBlock - 1) / kBlock;
#define LBM_INLET_ARGS                                                                                   \
    (const S*)b.fA, (S*)b.fB, (const S*)b.hA, (S*)b.hB, b.flags, b.theta, (R*)b.urec, b.frec, b.hrec, p
    if (!advance_h) k_inlet<S, QH, false, false><<<grid, kBlock, 0, s>>>(LBM_INLET_ARGS);
    else if (p.hkind == 3) k_inlet<S, QH, true, true><<<grid, kBlock, 0, s>>>(LBM_INLET_ARGS);
    else k_inlet<S, QH, false, true><<<grid, kBlock, 0, s>>>(LBM_INLET_ARGS);
#undef LBM_INLET_ARGS
    return cudaGetLastError();
}

// ---- symmetry rows (top and bottom symmetry planes, Sec. 4.4) -------------
// Specular reflection at the plane halfway between a symmetry row and its
// neighbour row: before each step every node of the rows y = 0 / y = ny-1
// takes the post-collision populations of the node beside it (y = 1 /
// y = ny-2) with e_y reversed; the step pulls from it like from any node and
// never writes it (it is flagged solid and has no wall links).
template <typename S, int QH>
__global__ void k_mirror(S* __restrict__ fA, S* __restrict__ hA, const DevParams p) {
    const int per = p.nx * p.nz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * per) return;
    const int side = i / per, r = i - side * per;
    if (side == 0 ? !p.mirror_lo : !p.mirror_hi) return;
    const int x = r % p.nx, z = r / p.nx;
    const int yg = side == 0 ? 0 : p.ny - 1, ys = side == 0 ? 1 : p.ny - 2;
    const size_t N = (size_t)p.N;
    const size_t g = x + (size_t)p.nx * (yg + (size_t)p.ny * z);
    const size_t src = x + (size_t)p.nx * (ys + (size_t)p.ny * z);
#pragma unroll
    for (int a = 0; a < 27; ++a) fA[a * N + g] = fA[FLIPY(a) * N + src];
#pragma unroll
    for (int k = 0; k < QH; ++k) hA[k * N + g] = hA[HFLIPY<QH>(k) * N + src];
}

template <typename S, int QH>
cudaError_t launch_mirror(const Buffers& b, const DevParams& p, cudaStream_t s) {
    const int total = 2 * p.nx * p.nz;
    k_mirror<S, QH><<<(total + kBlock - 1) / kBlock, kBlock, 0, s>>>((S*)b.fA, (S*)b.hA, p);
    return cudaGetLastError();
}

// ---- adjoint of the coupled f + h evolution -------------------------------
// The h step depends on the flow through u = U(g_f; F), so gradients with
// respect to flow parameters (the body force F, the inlet velocity u_in) need
// the adjoint of f as well.  Per node and level, from the recorded
// pre-collision arrivals g_f, g_h (Eq. hydro_cu_collision, Eq. H_cm_collision
// or H_cu_collision):
//   lambda = P^T mu^{k+1} + dJ/ds^k            (f: Eq. IBB; h: Eq. IABB)
//   w      = (dC_h/du)^T lambda_h
//   mu_h   = (dC_h/dg_h)^T lambda_h,   dJ/dQ += (dC_h/dQ)^T lambda_h
//   mu_f   = (dC_f/dg_f)^T lambda_f + (dU/dg_f)^T w
//   dJ/dF += (dC_f/dF)^T lambda_f + (dU/dF)^T w
// and at inlet nodes (equilibria at u_in) dJ/du_in += (ds_in/du_in)^T lambda.
// mu_h and dJ/dQ use the h-only adjoint's exact transpose, the u derivative
// of the h collision three forward-mode passes in dual numbers.  The f
// collision reads g_f only through its mass, momentum and second moments
// (m = P g_f, ten numbers), so (dC_f/dg_f)^T lambda_f = P^T G with
// G_k = lambda_f . (dC_f/dg_f) d_k for perturbations d_k with P d_k = unit_k
// (collide_f_adjoint: reverse mode through the synthesis, forward mode
// through the front part).

// Eq. IBB: derivative of the arrival f_abar(x_b) with respect to f*_a(x_b)
// and f*_abar(x_b) (the x_f term goes through the reverse-link table)
// component d of e_a
__device__ __forceinline__ int ecomp(int a, int d) { return d == 0 ? EX(a) : (d == 1 ? EY(a) : EZ(a)); }

template <typename R>
__device__ __forceinline__ void ibb_partials(float q, bool thin, R& d_ab, R& d_abb) {
    if (q <= 0.5f && !thin) {
        d_ab = R(2) * (R)q;
        d_abb = R(0);
    } else {
        const R qq = (R)fmaxf(q, 0.5f);
        d_ab = R(1) / (R(2) * qq);
        d_abb = (R(2) * qq - R(1)) / (R(2) * qq);
    }
}

// front part of the f collision (Eq. hydro_cu_collision, collide_f_force):
// from the ten moments m = (drho, j, second moments) and F to the relaxed
// second central moments s (diagonal) and k (off-diagonal), 1/rho, the mean
// after collision v and the velocity u for h
template <typename T> struct FFront {
    T drho, irho, sxx, syy, szz, kxy, kxz, kyz, v[3], u[3];
};
template <typename T>
__device__ __forceinline__ FFront<T> f_front(const T* m, const T Fx, const T Fy, const T Fz, const DevParams& p) {
    FFront<T> o;
    const T c = cs2<T>();
    const T drho = m[0], jx = m[1], jy = m[2], jz = m[3];
    const T rho = par<T>(p.rho0, p.pf.rho0) + drho;
    const T irho = T(1) / rho;
    const T mux = jx * irho, muy = jy * irho, muz = jz * irho;
    const T axx = m[4] - drho * c - jx * mux;
    const T ayy = m[5] - drho * c - jy * muy;
    const T azz = m[6] - drho * c - jz * muz;
    const T om1 = T(1) - par<T>(p.omega1, p.pf.omega1);
    const T omb = T(1) - par<T>(p.omega_bulk, p.pf.omega_bulk);
    const T dxy = (axx - ayy) * om1, dxz = (axx - azz) * om1, tr = (axx + ayy + azz) * omb;
    o.kxy = (m[7] - jx * muy) * om1;
    o.kxz = (m[8] - jx * muz) * om1;
    o.kyz = (m[9] - jy * muz) * om1;
    o.sxx = (tr + dxy + dxz) * (T(1) / T(3));
    o.syy = o.sxx - dxy;
    o.szz = o.sxx - dxz;
    o.drho = drho;
    o.irho = irho;
    o.v[0] = mux + Fx * irho;
    o.v[1] = muy + Fy * irho;
    o.v[2] = muz + Fz * irho;
    o.u[0] = mux + T(0.5) * Fx * irho;
    o.u[1] = muy + T(0.5) * Fy * irho;
    o.u[2] = muz + T(0.5) * Fz * irho;
    return o;
}

// Reverse mode through f_front: from the adjoints of its outputs (bs = s
// diagonal, bk = k off-diagonal, birho, bdrho_out, bv, bu) to those of the
// ten moments m and of F, written out step by step backwards through f_front.
template <typename R>
__device__ __forceinline__ void f_front_adjoint(const R* m, const DevParams& p, R bsxx, R bsyy, R bszz, R bkxy,
                                                R bkxz, R bkyz, R birho, R bdrho, const R* bv, const R* bu, R* G) {
    const R c = cs2<R>();
    const R drho = m[0], jx = m[1], jy = m[2], jz = m[3];
    const R rho = par<R>(p.rho0, p.pf.rho0) + drho;
    const R irho = R(1) / rho;
    const R mux = jx * irho, muy = jy * irho, muz = jz * irho;
    const R om1 = R(1) - par<R>(p.omega1, p.pf.omega1);
    const R omb = R(1) - par<R>(p.omega_bulk, p.pf.omega_bulk);
    const R F[3] = {par<R>(p.F[0], p.pf.F[0]), par<R>(p.F[1], p.pf.F[1]), par<R>(p.F[2], p.pf.F[2])};
    // sxx = (tr + dxy + dxz)/3, syy = sxx - dxy, szz = sxx - dxz
    const R bst = bsxx + bsyy + bszz;
    const R bdxy = bst * (R(1) / R(3)) - bsyy;
    const R bdxz = bst * (R(1) / R(3)) - bszz;
    const R btr = bst * (R(1) / R(3));
    // dxy = (axx - ayy) om1, dxz = (axx - azz) om1, tr = (axx + ayy + azz) omb
    const R baxx = om1 * (bdxy + bdxz) + omb * btr;
    const R bayy = -om1 * bdxy + omb * btr;
    const R bazz = -om1 * bdxz + omb * btr;
    R bj[3] = {R(0), R(0), R(0)}, bmu[3] = {R(0), R(0), R(0)};
    // kxy = (m7 - jx muy) om1, kxz = (m8 - jx muz) om1, kyz = (m9 - jy muz) om1
    G[7] = om1 * bkxy;
    G[8] = om1 * bkxz;
    G[9] = om1 * bkyz;
    bj[0] -= om1 * (bkxy * muy + bkxz * muz);
    bmu[1] -= om1 * bkxy * jx;
    bmu[2] -= om1 * (bkxz * jx + bkyz * jy);
    bj[1] -= om1 * bkyz * muz;
    // a_dd = m_(4+d) - drho c - j_d mu_d
    const R ba[3] = {baxx, bayy, bazz};
    const R mu[3] = {mux, muy, muz}, j[3] = {jx, jy, jz};
    R bdr = bdrho;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        G[4 + d] = ba[d];
        bdr -= c * ba[d];
        bj[d] -= mu[d] * ba[d];
        bmu[d] -= j[d] * ba[d];
    }
    // v_d = mu_d + F_d irho, u_d = mu_d + F_d irho / 2
    R bir = birho;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        bmu[d] += bv[d] + bu[d];
        G[10 + d] = irho * (bv[d] + R(0.5) * bu[d]);
        bir += F[d] * (bv[d] + R(0.5) * bu[d]);
    }
    // mu_d = j_d irho
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        bj[d] += irho * bmu[d];
        bir += j[d] * bmu[d];
    }
    // irho = 1 / (rho0 + drho)
    bdr -= irho * irho * bir;
    G[0] = bdr;
    G[1] = bj[0];
    G[2] = bj[1];
    G[3] = bj[2];
}

// w_d = lambda_h . dC_h/du_d for the central-moment kinds (Eq.
// H_cm_collision, App. D source), in reverse mode.  With Y = T(u) g the
// central moments of the arrivals g (deviations), Y* their relaxed values and
// z = T(u)^-T lambda: dT/du_d = -S_d T exactly on the three-point stencil,
// (S_d Y)_mno = m_d Y_(m - e_d)no lowering the d-th order by one, and the
// stored shift T_ref K(u) of the central moments gives S_d K, so
//   dC_h/du_d = T^-1 (S_d Y* - (1 - S) S_d Y + S T_ref S_d K)
// and w_d = z . (S_d Y* - (1 - S) S_d Y + S T_ref S_d K).
// w from z = T(u)^-T lambda in cube slots (D3Q27)
template <typename R>
__device__ __forceinline__ void velocity_from_z27(const R* Z, const R* g, R ux, R uy, R uz, R Q, const DevParams& p,
                                                  R* w) {
    const R Tref = par<R>(p.Tref, p.pf.Tref);
    {
        R Y[27];
#pragma unroll
        for (int a = 0; a < 27; ++a) Y[CUBE(a)] = g[a];
        forward_cube<R>(Y, ux, uy, uz);
        const R dH = Y[0] + R(0.5) * Q;
        const R tx = ux * ux, ty = uy * uy, tz = uz * uz;
        R Ys[27];
#pragma unroll
        for (int o = 0; o < 3; ++o)
#pragma unroll
            for (int n = 0; n < 3; ++n)
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const R sr = par<R>(p.sh[m + n + o], p.pf.sh[m + n + o]);
                    const R E = Eq<R>(m, n, o);
                    const R D = Dm<R>(m, n, o, ux, uy, uz, tx, ty, tz);
                    const int i = MIDX(m, n, o);
                    Ys[i] = (R(1) - sr) * Y[i] + sr * (dH * E + Tref * D) + (R(1) - R(0.5) * sr) * Q * E;
                }
        R acc[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int o = 0; o < 3; ++o)
#pragma unroll
            for (int n = 0; n < 3; ++n)
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const R sr = par<R>(p.sh[m + n + o], p.pf.sh[m + n + o]);
                    const R zz = Z[MIDX(m, n, o)];
                    if (m >= 1) {
                        const int lo = MIDX(m - 1, n, o);
                        const R K = Kd<R>(m - 1, ux) * Kd<R>(n, uy) * Kd<R>(o, uz);
                        acc[0] += zz * R(m) * (Ys[lo] - (R(1) - sr) * Y[lo] + sr * Tref * K);
                    }
                    if (n >= 1) {
                        const int lo = MIDX(m, n - 1, o);
                        const R K = Kd<R>(m, ux) * Kd<R>(n - 1, uy) * Kd<R>(o, uz);
                        acc[1] += zz * R(n) * (Ys[lo] - (R(1) - sr) * Y[lo] + sr * Tref * K);
                    }
                    if (o >= 1) {
                        const int lo = MIDX(m, n, o - 1);
                        const R K = Kd<R>(m, ux) * Kd<R>(n, uy) * Kd<R>(o - 1, uz);
                        acc[2] += zz * R(o) * (Ys[lo] - (R(1) - sr) * Y[lo] + sr * Tref * K);
                    }
                }
        w[0] = acc[0];
        w[1] = acc[1];
        w[2] = acc[2];
    }
}

template <typename R, int QH>
__device__ __forceinline__ void h_velocity_adjoint(const R* lam, const R* g, R ux, R uy, R uz, R Q,
                                                   const DevParams& p, R* w) {
    const R Tref = par<R>(p.Tref, p.pf.Tref);
    if constexpr (QH == 27) {
        R Z[27];
#pragma unroll
        for (int a = 0; a < 27; ++a) Z[CUBE(a)] = lam[a];
        z_from_lambda27<R>(Z, ux, uy, uz);
        velocity_from_z27<R>(Z, g, ux, uy, uz, Q, p, w);
    } else {
        // D3Q7: moments 0, 1d, 2d about u; S_d takes 0 -> 1d and 1d -> 2d (x2)
        const R u[3] = {ux, uy, uz};
        const R c = cs2<R>();
        R z0 = lam[0];
        R z1[3], z2[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const R mb2 = R(0.5) * (lam[1 + d] + lam[4 + d]) - lam[0];
            const R mb1 = R(0.5) * (lam[1 + d] - lam[4 + d]);
            z2[d] = mb2;
            z1[d] = mb1 + R(2) * u[d] * mb2;
            z0 += u[d] * mb1 + u[d] * u[d] * mb2;
        }
        (void)z0;
        const R m0 = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6];
        const R dH = m0 + R(0.5) * Q;
        const R s0 = par<R>(p.sh[0], p.pf.sh[0]), s1 = par<R>(p.sh[1], p.pf.sh[1]), s2 = par<R>(p.sh[2], p.pf.sh[2]);
        const R y0 = m0, ys0 = (R(1) - s0) * m0 + s0 * dH + (R(1) - R(0.5) * s0) * Q;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const R k1 = (g[1 + d] - g[4 + d]) - u[d] * m0;
            const R ys1 = (R(1) - s1) * k1 + s1 * (Tref * u[d]);
            // S_d K: 1 at the first order, 2 K_1 = -2 u_d at the second
            w[d] = z1[d] * (ys0 - (R(1) - s1) * y0 + s1 * Tref) +
                   z2[d] * R(2) * (ys1 - (R(1) - s2) * k1 - s2 * Tref * u[d]);
        }
        (void)c;
    }
}

// mu_h, dJ/dQ and w of a central-moment kind, z = T(u)^-T lambda computed
// once for both (D3Q27; D3Q7 forms z in a few operations and calls the two
// functions)
template <typename R, int QH>
__device__ __forceinline__ void h_transpose_and_velocity(const R* lam, const R* g, R ux, R uy, R uz, R Q,
                                                         const DevParams& p, R* mu, double& dth, R* w) {
    if constexpr (QH == 27) {
        R Z[27];
#pragma unroll
        for (int a = 0; a < 27; ++a) Z[CUBE(a)] = lam[a];
        z_from_lambda27<R>(Z, ux, uy, uz);
        velocity_from_z27<R>(Z, g, ux, uy, uz, Q, p, w);
        dth = 0.0;
        transpose_from_z27<R>(Z, ux, uy, uz, p, mu, dth);
    } else {
        h_velocity_adjoint<R, QH>(lam, g, ux, uy, uz, Q, p, w);
        h_collision_transpose<R, QH, false>(lam, nullptr, ux, uy, uz, Q, p, mu, dth);
    }
}

// Adjoint of the f collision of one node, given the ten raw moments m of its
// pre-collision arrivals (raw_moments_f order; the collision reads f only
// through them): G[k] = lambda . (dC_f/dg) d_k + w . (dU/dg) d_k for the ten unit-moment
// perturbations d_k (k < 10) and the same for the three components of F
// (k = 10..12).  The synthesis (central moments -> populations through the
// inverse transform at the mean v) is differentiated in reverse mode once:
// z = T(v)^-T lambda, the adjoints of s, k, 1/rho, drho by hand, and of v
// through both the equilibrium part of the moments and the transform, whose
// derivative is d/dv_x T(v)^-1 kappa = T(v)^-1 (S_x kappa), (S_x kappa)_mno =
// m kappa_(m-1)no (exact on the three-point lattice).  The front part (ten
// moments and F -> s, k, 1/rho, v, u) is reversed by hand (f_front_adjoint).
template <typename R>
__device__ __forceinline__ void collide_f_adjoint(const R* m, const DevParams& p, const R* lam, const R* w, R* G) {
    const FFront<R> S = f_front<R>(m, par<R>(p.F[0], p.pf.F[0]), par<R>(p.F[1], p.pf.F[1]), par<R>(p.F[2], p.pf.F[2]), p);
    const R c = cs2<R>();
    const R sxx = S.sxx, syy = S.syy, szz = S.szz, kxy = S.kxy, kxz = S.kxz, kyz = S.kyz, irho = S.irho;
    const R vx = S.v[0], vy = S.v[1], vz = S.v[2];
    const R rho0 = par<R>(p.rho0, p.pf.rho0);
    // post-collision central moments kappa (as in collide_f_force)
    R K[27];
    {
        const R n220 = c * (sxx + syy) + (sxx * syy + R(2) * kxy * kxy) * irho;
        const R n202 = c * (sxx + szz) + (sxx * szz + R(2) * kxz * kxz) * irho;
        const R n022 = c * (syy + szz) + (syy * szz + R(2) * kyz * kyz) * irho;
        const R n211 = c * kyz + (sxx * kyz + R(2) * kxy * kxz) * irho;
        const R n121 = c * kxz + (syy * kxz + R(2) * kxy * kyz) * irho;
        const R n112 = c * kxy + (szz * kxy + R(2) * kxz * kyz) * irho;
        const R n222 = c * c * (sxx + syy + szz) +
                       (c * (sxx * syy + sxx * szz + syy * szz) + R(2) * c * (kxy * kxy + kxz * kxz + kyz * kyz)) * irho +
                       (sxx * syy * szz + R(2) * (sxx * kyz * kyz + syy * kxz * kxz + szz * kxy * kxy) +
                        R(8) * kxy * kxz * kyz) * irho * irho;
        const R tx = vx * vx, ty = vy * vy, tz = vz * vz;
#pragma unroll
        for (int o = 0; o < 3; ++o)
#pragma unroll
            for (int n = 0; n < 3; ++n)
#pragma unroll
                for (int mm = 0; mm < 3; ++mm) {
                    R neq = R(0);
                    if (mm == 1 && n == 1 && o == 0) neq = kxy;
                    if (mm == 1 && n == 0 && o == 1) neq = kxz;
                    if (mm == 0 && n == 1 && o == 1) neq = kyz;
                    if (mm == 2 && n == 0 && o == 0) neq = sxx;
                    if (mm == 0 && n == 2 && o == 0) neq = syy;
                    if (mm == 0 && n == 0 && o == 2) neq = szz;
                    if (mm == 2 && n == 2 && o == 0) neq = n220;
                    if (mm == 2 && n == 0 && o == 2) neq = n202;
                    if (mm == 0 && n == 2 && o == 2) neq = n022;
                    if (mm == 2 && n == 1 && o == 1) neq = n211;
                    if (mm == 1 && n == 2 && o == 1) neq = n121;
                    if (mm == 1 && n == 1 && o == 2) neq = n112;
                    if (mm == 2 && n == 2 && o == 2) neq = n222;
                    K[MIDX(mm, n, o)] = neq + S.drho * Eq<R>(mm, n, o) + rho0 * Dm<R>(mm, n, o, vx, vy, vz, tx, ty, tz);
                }
    }
    // z = T(v)^-T lambda (the transposed passes in reverse order)
    R Z[27];
#pragma unroll
    for (int a = 0; a < 27; ++a) Z[CUBE(a)] = lam[a];
#pragma unroll
    for (int j = 0; j < 9; ++j) inv3T<R>(Z[3 * j], Z[3 * j + 1], Z[3 * j + 2], vx);
#pragma unroll
    for (int zz = 0; zz < 3; ++zz)
#pragma unroll
        for (int xx = 0; xx < 3; ++xx) inv3T<R>(Z[9 * zz + xx], Z[9 * zz + 3 + xx], Z[9 * zz + 6 + xx], vy);
#pragma unroll
    for (int j = 0; j < 9; ++j) inv3T<R>(Z[j], Z[9 + j], Z[18 + j], vz);
    // adjoints of the synthesis inputs
    R bsxx = Z[MIDX(2, 0, 0)], bsyy = Z[MIDX(0, 2, 0)], bszz = Z[MIDX(0, 0, 2)];
    R bkxy = Z[MIDX(1, 1, 0)], bkxz = Z[MIDX(1, 0, 1)], bkyz = Z[MIDX(0, 1, 1)];
    R birho = R(0), bdrho = R(0);
    {
        R t = Z[MIDX(2, 2, 0)];
        bsxx += t * (c + syy * irho); bsyy += t * (c + sxx * irho); bkxy += t * R(4) * kxy * irho;
        birho += t * (sxx * syy + R(2) * kxy * kxy);
        t = Z[MIDX(2, 0, 2)];
        bsxx += t * (c + szz * irho); bszz += t * (c + sxx * irho); bkxz += t * R(4) * kxz * irho;
        birho += t * (sxx * szz + R(2) * kxz * kxz);
        t = Z[MIDX(0, 2, 2)];
        bsyy += t * (c + szz * irho); bszz += t * (c + syy * irho); bkyz += t * R(4) * kyz * irho;
        birho += t * (syy * szz + R(2) * kyz * kyz);
        t = Z[MIDX(2, 1, 1)];
        bkyz += t * (c + sxx * irho); bsxx += t * kyz * irho; bkxy += t * R(2) * kxz * irho;
        bkxz += t * R(2) * kxy * irho; birho += t * (sxx * kyz + R(2) * kxy * kxz);
        t = Z[MIDX(1, 2, 1)];
        bkxz += t * (c + syy * irho); bsyy += t * kxz * irho; bkxy += t * R(2) * kyz * irho;
        bkyz += t * R(2) * kxy * irho; birho += t * (syy * kxz + R(2) * kxy * kyz);
        t = Z[MIDX(1, 1, 2)];
        bkxy += t * (c + szz * irho); bszz += t * kxy * irho; bkxz += t * R(2) * kyz * irho;
        bkyz += t * R(2) * kxz * irho; birho += t * (szz * kxy + R(2) * kxz * kyz);
        t = Z[MIDX(2, 2, 2)];
        const R P2 = sxx * syy + sxx * szz + syy * szz, Q2 = kxy * kxy + kxz * kxz + kyz * kyz;
        const R P3 = sxx * syy * szz + R(2) * (sxx * kyz * kyz + syy * kxz * kxz + szz * kxy * kxy) +
                     R(8) * kxy * kxz * kyz;
        const R i2 = irho * irho;
        bsxx += t * (c * c + c * (syy + szz) * irho + (syy * szz + R(2) * kyz * kyz) * i2);
        bsyy += t * (c * c + c * (sxx + szz) * irho + (sxx * szz + R(2) * kxz * kxz) * i2);
        bszz += t * (c * c + c * (sxx + syy) * irho + (sxx * syy + R(2) * kxy * kxy) * i2);
        bkxy += t * (R(4) * c * kxy * irho + (R(4) * szz * kxy + R(8) * kxz * kyz) * i2);
        bkxz += t * (R(4) * c * kxz * irho + (R(4) * syy * kxz + R(8) * kxy * kyz) * i2);
        bkyz += t * (R(4) * c * kyz * irho + (R(4) * sxx * kyz + R(8) * kxy * kxz) * i2);
        birho += t * ((c * P2 + R(2) * c * Q2) + R(2) * P3 * irho);
    }
    R bv[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int o = 0; o < 3; ++o)
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
            for (int mm = 0; mm < 3; ++mm) {
                const R zz = Z[MIDX(mm, n, o)];
                bdrho += zz * Eq<R>(mm, n, o);
                // the equilibrium part rho0 (E - K(v)) of the moments
                const R kx = Kd<R>(mm, vx), ky = Kd<R>(n, vy), kz = Kd<R>(o, vz);
                const R dkx = mm == 0 ? R(0) : (mm == 1 ? R(-1) : R(2) * vx);
                const R dky = n == 0 ? R(0) : (n == 1 ? R(-1) : R(2) * vy);
                const R dkz = o == 0 ? R(0) : (o == 1 ? R(-1) : R(2) * vz);
                bv[0] -= zz * rho0 * dkx * ky * kz;
                bv[1] -= zz * rho0 * kx * dky * kz;
                bv[2] -= zz * rho0 * kx * ky * dkz;
                // the transform: d/dv T(v)^-1 kappa = T(v)^-1 (S kappa)
                if (mm >= 1) bv[0] += zz * R(mm) * K[MIDX(mm - 1, n, o)];
                if (n >= 1) bv[1] += zz * R(n) * K[MIDX(mm, n - 1, o)];
                if (o >= 1) bv[2] += zz * R(o) * K[MIDX(mm, n, o - 1)];
            }
    // reverse mode through the front part
    f_front_adjoint<R>(m, p, bsxx, bsyy, bszz, bkxy, bkxz, bkyz, birho, bdrho, bv, w, G);
}

// Adjoint of the Zou-He rule at an inlet node for the coupled sweep (the
// rule: zou_he_fill_f, zou_he_fill_h).  g, gh: the node's recorded full
// arrival vectors (the known ones, e_x <= 0, as pulled); muf, muh: the
// adjoints of the full arrival vectors, replaced by those of the known ones
// (the unknown ones are pulled from nowhere: 0).  For fixed u_in the rule is
// affine in the known arrivals, and its transpose follows the rule backwards:
// the h amplitude damp = (rho T_in - T_ref - K - T_ref (u_x^2 + u_x)/2) / M+
// (M+ = (c_s^2 + u_x^2 + u_x)/2, K the sum of the known h), the unknown f
// f_a = f_abar + fe_a - fe_abar - e_ya N_y - e_za N_z with fe the equilibrium
// at (drho, u_in) and N_d = sum_{e_x = 0} e_d (f - fe) / 6, and drho =
// (s_0 + 2 s_- + rho0 u_x) / (1 - u_x) from the known f.  dJ/du_in
// (accumulated into duin[3]) comes from three forward-mode passes through the
// rule itself.
template <typename R, int QH>
__device__ __forceinline__ void zou_he_transpose_coupled(const R* g, const R* gh, R* muf, R* muh,
                                                         const DevParams& p, double* duin) {
    const R ux = par<R>(p.uin[0], p.pf.uin[0]), uy = par<R>(p.uin[1], p.pf.uin[1]), uz = par<R>(p.uin[2], p.pf.uin[2]);
    using D = Dual<R>;
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
        D fd[27], hd[QH];
#pragma unroll
        for (int a = 0; a < 27; ++a) fd[a] = D(EX(a) == 1 ? R(0) : g[a], R(0), 0);
#pragma unroll
        for (int k = 0; k < QH; ++k) hd[k] = D(EX(HDIR<QH>(k)) == 1 ? R(0) : gh[k], R(0), 0);
        const D vx(ux, d == 0 ? R(1) : R(0), 0), vy(uy, d == 1 ? R(1) : R(0), 0), vz(uz, d == 2 ? R(1) : R(0), 0);
        const D drho = zou_he_fill_f<D>(fd, vx, vy, vz, p);
        zou_he_fill_h<D, QH>(hd, drho, vx, vy, vz, p);
        R acc = R(0);
#pragma unroll
        for (int a = 0; a < 27; ++a)
            if (EX(a) == 1) acc += muf[a] * fd[a].d;
#pragma unroll
        for (int k = 0; k < QH; ++k)
            if (EX(HDIR<QH>(k)) == 1) acc += muh[k] * hd[k].d;
        duin[d] += (double)acc;
    }
    // per-axis unit equilibrium weights at u_in (index e + 1)
    R M[3][3];
#pragma unroll
    for (int e = -1; e <= 1; ++e) {
        M[0][e + 1] = w1_unit<R>(e, ux);
        M[1][e + 1] = w1_unit<R>(e, uy);
        M[2][e + 1] = w1_unit<R>(e, uz);
    }
    const R mU = M[0][2];
    // h: the unknown arrivals are damp M_j (+ a constant)
    R bdamp = R(0);
#pragma unroll
    for (int k = 0; k < QH; ++k) {
        const int a = HDIR<QH>(k);
        if (EX(a) != 1) continue;
        bdamp += muh[k] * (QH == 27 ? M[0][2] * M[1][EY(a) + 1] * M[2][EZ(a) + 1] : mU);
    }
    const R bK = -bdamp / mU;
    R bdrho = par<R>(p.Tin, p.pf.Tin) * bdamp / mU;
#pragma unroll
    for (int k = 0; k < QH; ++k) muh[k] = (EX(HDIR<QH>(k)) == 1) ? R(0) : muh[k] + bK;
    // f: the unknown arrivals through fe (drho) and N_y, N_z
    R bfe[27];
#pragma unroll
    for (int a = 0; a < 27; ++a) bfe[a] = R(0);
    R bNy = R(0), bNz = R(0);
#pragma unroll
    for (int a = 0; a < 27; ++a) {
        if (EX(a) != 1) continue;
        const int b = OPP(a);
        const R m = muf[a];
        muf[b] += m;
        bfe[a] += m;
        bfe[b] -= m;
        bNy -= R(EY(a)) * m;
        bNz -= R(EZ(a)) * m;
    }
#pragma unroll
    for (int c = 0; c < 27; ++c) {
        if (EX(c) != 0) continue;
        const R t = (R(EY(c)) * bNy + R(EZ(c)) * bNz) * (R(1) / R(6));
        muf[c] += t;
        bfe[c] -= t;
    }
#pragma unroll
    for (int a = 0; a < 27; ++a) bdrho += bfe[a] * M[0][EX(a) + 1] * M[1][EY(a) + 1] * M[2][EZ(a) + 1];
    const R q = bdrho / (R(1) - ux);
#pragma unroll
    for (int c = 0; c < 27; ++c) {
        if (EX(c) == 0) muf[c] += q;
        else if (EX(c) == -1) muf[c] += R(2) * q;
        else muf[c] = R(0);
    }
}

// mu_f = P^T G: for each population b, G_0 + e_b . (G_1, G_2, G_3) +
// (e_bx^2, e_by^2, e_bz^2) . (G_4, G_5, G_6) + e_bx e_by G_7 + e_bx e_bz G_8 +
// e_by e_bz G_9 (the transpose of raw_moments_f), built along the x lines:
// per (e_y, e_z) a base and a slope, then base, base + (G_4 +- slope)
template <typename R> __device__ __forceinline__ void moments_transpose_f(const R* G, R* out) {
    R Z[3], SZ[3], Y[3];
#pragma unroll
    for (int e = -1; e <= 1; ++e) {
        Z[e + 1] = (e == 0) ? G[0] : G[0] + (G[6] + R(e) * G[3]);
        SZ[e + 1] = (e == 0) ? G[1] : G[1] + R(e) * G[8];
        Y[e + 1] = (e == 0) ? R(0) : G[5] + R(e) * G[2];
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const int ey = j % 3 - 1, ez = j / 3 - 1;
        R base = (ey == 0) ? Z[ez + 1] : Z[ez + 1] + Y[ey + 1];
        if (ey != 0 && ez != 0) base += R(ey * ez) * G[9];
        const R slope = (ey == 0) ? SZ[ez + 1] : SZ[ez + 1] + R(ey) * G[7];
        out[DIR(0, ey, ez)] = base;
        out[DIR(1, ey, ez)] = base + (G[4] + slope);
        out[DIR(-1, ey, ez)] = base + (G[4] - slope);
    }
}

// velocity u of the h collision from the raw moments of a node's pre-collision
// f arrivals (m[0] = density deviation, m[1..3] = momentum), as
// collide_f_force computes it: u = (sum e f + F/2) / rho
template <typename R>
__device__ __forceinline__ void flow_velocity(const R* m, const DevParams& p, R& ux, R& uy, R& uz) {
    const R drho = m[0], jx = m[1], jy = m[2], jz = m[3];
    const R irho = R(1) / (par<R>(p.rho0, p.pf.rho0) + drho);
    ux = jx * irho + R(0.5) * par<R>(p.F[0], p.pf.F[0]) * irho;
    uy = jy * irho + R(0.5) * par<R>(p.F[1], p.pf.F[1]) * irho;
    uz = jz * irho + R(0.5) * par<R>(p.F[2], p.pf.F[2]) * irho;
}

// One level of the coupled sweep in two kernels, each about half the code
// (one kernel held both and was bound by instruction fetch): PART 1, the h
// adjoint (gather of mu_h, transposed h collision, the velocity derivative w
// written to wbuf[3][N], dJ/dQ, the wall-temperature terms); PART 2, the f
// adjoint (gather of mu_f, the reversed f collision with w, dJ/dF).  PART 1
// runs first.
template <typename R, int QH, bool CUM, int PART>
__global__ void __launch_bounds__(kBlock) k_adjoint_flow(
    const R* __restrict__ muf_next, const R* __restrict__ muh_next, R* __restrict__ muf_out, R* __restrict__ muh_out,
    const R* __restrict__ gf, const R* __restrict__ gh, const float* __restrict__ theta,
    double* __restrict__ dtheta, double* __restrict__ acc6, const R* __restrict__ din, R* __restrict__ wbuf,
    const uint8_t* __restrict__ flags, const int32_t* __restrict__ seg_base, const uint32_t* __restrict__ wmask,
    const int32_t* __restrict__ woff, const float* __restrict__ lq, const int32_t* __restrict__ lwall,
    const int32_t* __restrict__ rseg_base, const uint32_t* __restrict__ rmask, const int32_t* __restrict__ roff,
    const int32_t* __restrict__ rlink, double* __restrict__ dlink, const AdjObjective obj, const DevParams p) {
    using D = Dual<R>;
    constexpr bool HP = PART == 1, FP = PART == 2;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in_range = n < p.N;
    const uint8_t fl = in_range ? flags[n] : (uint8_t)T_SOLID;
    const bool is_wall = (fl & F_WALL) != 0, is_rw = (fl & F_RWALL) != 0;
    const uint32_t bal_w = __ballot_sync(0xffffffffu, is_wall);
    const uint32_t bal_r = __ballot_sync(0xffffffffu, is_rw);
    if (!in_range) return;
    const int N = p.N;
    const int type = fl & 3;
    if (type == T_SOLID) {
        if constexpr (FP) {
#pragma unroll
            for (int a = 0; a < 27; ++a) muf_out[a * N + n] = R(0);
        } else {
#pragma unroll
            for (int i = 0; i < QH; ++i) muh_out[i * N + n] = R(0);
        }
        return;
    }
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    int x, y, z;
    node_xyz(n, p, x, y, z);
    int xt[3] = {x - 1, x, x + 1};
    if (p.periodic_x) {
        if (xt[0] < 0) xt[0] += p.nx;
        if (xt[2] >= p.nx) xt[2] -= p.nx;
    } else {
        if (xt[0] < 0) xt[0] = -1;
        if (xt[2] >= p.nx) xt[2] = -1;
    }
    const int yt[3] = {((y == 0) ? p.ny - 1 : y - 1) * p.nx, y * p.nx, ((y == p.ny - 1) ? 0 : y + 1) * p.nx};
    const int pl = p.nx * p.ny;
    const int zt[3] = {((z == 0) ? p.nz - 1 : z - 1) * pl, z * pl, ((z == p.nz - 1) ? 0 : z + 1) * pl};
    const R wsurf = (obj.kind == 0) ? (R)obj.weight : R(0);
    // force objective: d/ds_f of weight * e_a,comp (f*_a(x_b) + f_abar(x_b)) per link of obj.wall
    const R wforce = (obj.kind == 2) ? (R)obj.weight : R(0);
    // symmetry rows: a push into a symmetry row lands on this row, e_y
    // reversed (the row's copies, k_mirror; as in k_adjoint)
    const bool rlo = p.mirror_lo && y == 1, rhi = p.mirror_hi && y == p.ny - 2;
    // lambda = P^T mu^{k+1} (+ the objective's terms)
    R lf[FP ? 27 : 1], lh[HP ? QH : 1];
    if constexpr (FP) {
#pragma unroll
        for (int a = 0; a < 27; ++a) {
            const int xx = xt[EX(a) + 1];
            const bool refl = (EY(a) == -1 && rlo) || (EY(a) == 1 && rhi);
            const int row = refl ? y * p.nx : yt[EY(a) + 1];
            lf[a] = (xx < 0) ? R(0) : muf_next[(refl ? FLIPY(a) : a) * N + xx + row + zt[EZ(a) + 1]];
        }
        if (!p.periodic_x && x == p.nx - 1) {
#pragma unroll
            for (int a = 0; a < 27; ++a) {
                if (EX(a) != -1) continue;
                const bool refl = (EY(a) == -1 && rlo) || (EY(a) == 1 && rhi);
                lf[a] += muf_next[(refl ? FLIPY(a) : a) * N + x + (refl ? y * p.nx : yt[EY(a) + 1]) + zt[EZ(a) + 1]];
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < QH; ++i) {
            const int a = HDIR<QH>(i);
            const int xx = xt[EX(a) + 1];
            const bool refl = (EY(a) == -1 && rlo) || (EY(a) == 1 && rhi);
            const int row = refl ? y * p.nx : yt[EY(a) + 1];
            lh[i] = (xx < 0) ? R(0) : muh_next[(refl ? HFLIPY<QH>(i) : i) * N + xx + row + zt[EZ(a) + 1]];
        }
        if (!p.periodic_x && x == p.nx - 1) {
#pragma unroll
            for (int i = 0; i < QH; ++i) {
                const int a = HDIR<QH>(i);
                if (EX(a) != -1) continue;
                const bool refl = (EY(a) == -1 && rlo) || (EY(a) == 1 && rhi);
                lh[i] += muh_next[(refl ? HFLIPY<QH>(i) : i) * N + x + (refl ? y * p.nx : yt[EY(a) + 1]) +
                                  zt[EZ(a) + 1]];
            }
        }
    }
    if (is_rw) {
        // this node is x_f of links (t = y + e_a, a) with q <= 1/2
        const int idx = __ldg(rseg_base + (n >> 5)) + __popc(bal_r & lt);
        const uint32_t rm = __ldg(rmask + idx);
        const int ro = __ldg(roff + idx);
        if constexpr (FP) {
#pragma unroll
            for (int a = 0; a < 27; ++a) {
                if (!(rm & (1u << a))) continue;
                const int l = __ldg(rlink + ro + __popc(rm & ((1u << a) - 1u)));
                const float q = __ldg(lq + l);
                const int t = xt[EX(a) + 1] + yt[EY(a) + 1] + zt[EZ(a) + 1];
                const R cf = (__ldg(lwall + l) == obj.wall) ? wforce * (R)ecomp(a, obj.comp) : R(0);
                lf[a] += (R(1) - R(2) * (R)q) * (muf_next[OPP(a) * N + t] + cf);
            }
        } else {
#pragma unroll
            for (int i = 0; i < QH; ++i) {
                const int a = HDIR<QH>(i);
                if (!(rm & (1u << a))) continue;
                const int l = __ldg(rlink + ro + __popc(rm & ((1u << a) - 1u)));
                const float q = __ldg(lq + l);
                const R cw = (__ldg(lwall + l) == obj.wall) ? wsurf : R(0);
                const int t = xt[EX(a) + 1] + yt[EY(a) + 1] + zt[EZ(a) + 1];
                lh[i] -= (R(1) - R(2) * (R)q) * (muh_next[HOPP<QH>(i) * N + t] + cw);
            }
        }
    }
    if (is_wall) {
        const int idx = __ldg(seg_base + (n >> 5)) + __popc(bal_w & lt);
        const uint32_t mask = __ldg(wmask + idx);
        const int off = __ldg(woff + idx);
        if constexpr (FP) {
#pragma unroll
            for (int b = 0; b < 27; ++b) {
                if (!(mask & (1u << b))) continue;
                const int ib = OPP(b);
                const int l = off + __popc(mask & ((1u << b) - 1u));
                const float q = __ldg(lq + l);
                const bool thin = (mask >> ib) & 1u;
                R d_ab, d_abb;
                ibb_partials<R>(q, thin, d_ab, d_abb);
                const R cf = (__ldg(lwall + l) == obj.wall) ? wforce * (R)ecomp(b, obj.comp) : R(0);
                const R m = muf_next[ib * N + n] + cf;
                lf[b] += d_ab * m + cf;
                lf[ib] += d_abb * m;
            }
        } else {
#pragma unroll
            for (int i = 0; i < QH; ++i) {
                const int b = HDIR<QH>(i);
                if (!(mask & (1u << b))) continue;
                const int ib = HOPP<QH>(i);
                const int l = off + __popc(mask & ((1u << b) - 1u));
                const float q = __ldg(lq + l);
                const R cw = (__ldg(lwall + l) == obj.wall) ? wsurf : R(0);
                const bool thin = (mask >> HDIR<QH>(ib)) & 1u;
                R d_ab, d_abb, d_T;
                iabb_partials<R>(q, thin, p.wall_bc, d_ab, d_abb, d_T);
                const R m = muh_next[ib * N + n] + cw;
                lh[i] += d_ab * m - cw;
                lh[ib] += d_abb * m;
                dlink[l] += (double)d_T * HW<QH>(i) * (double)m;
            }
        }
    }
    if constexpr (HP) {
        if (obj.kind == 1 && x == obj.plane) {
#pragma unroll
            for (int i = 0; i < QH; ++i) lh[i] += (R)obj.weight * (R)EX(HDIR<QH>(i));
        }
    }
    if (!gf) {  // the initial level: its state is given; write lambda
        if constexpr (FP) {
#pragma unroll
            for (int a = 0; a < 27; ++a) muf_out[a * N + n] = lf[a];
        } else {
#pragma unroll
            for (int i = 0; i < QH; ++i) muh_out[i * N + n] = lh[i];
        }
        return;
    }
    if (type == T_INLET && !p.zou_he) {
        // the inlet holds the equilibria at u_in: din[d * (27 + QH) + .] = d s_in / d u_in,d
#pragma unroll 1
        for (int d = 0; d < 3; ++d) {
            double acc = 0.0;
            if constexpr (FP) {
#pragma unroll
                for (int a = 0; a < 27; ++a) acc += (double)(din[d * (27 + QH) + a] * lf[a]);
            } else {
#pragma unroll
                for (int i = 0; i < QH; ++i) acc += (double)(din[d * (27 + QH) + 27 + i] * lh[i]);
            }
            acc6[(size_t)n * 6 + 3 + d] += acc;
        }
        if constexpr (FP) {
#pragma unroll
            for (int a = 0; a < 27; ++a) muf_out[a * N + n] = R(0);
        } else {
#pragma unroll
            for (int i = 0; i < QH; ++i) muh_out[i * N + n] = R(0);
        }
        return;
    }
    // the level's f moments (raw_moments_f order): the h part needs only
    // the density and momentum, the f part all ten
    R g[10];
#pragma unroll
    for (int k = 0; k < (HP ? 4 : 10); ++k) g[k] = gf[k * N + n];
    if constexpr (HP) {
        R hpre[QH];
#pragma unroll
        for (int i = 0; i < QH; ++i) hpre[i] = gh[i * N + n];
        const R Q = theta ? (R)__ldg(theta + n) : R(0);
        R ux, uy, uz;
        flow_velocity<R>(g, p, ux, uy, uz);
        // w = (dC_h/du)^T lambda_h: reverse mode for the central-moment kinds,
        // three forward-mode passes in u for the nonlinear Cumulants-1st
        R w[3];
        if constexpr (CUM) {
#pragma unroll 1
            for (int k = 0; k < 3; ++k) {
                D hd[QH];
#pragma unroll
                for (int i = 0; i < QH; ++i) hd[i] = D(hpre[i]);
                const D vx(ux, k == 0 ? R(1) : R(0), 0), vy(uy, k == 1 ? R(1) : R(0), 0),
                    vz(uz, k == 2 ? R(1) : R(0), 0);
                collide_h<D, QH, CUM>(hd, vx, vy, vz, D(Q), p);
                R acc = R(0);
#pragma unroll
                for (int i = 0; i < QH; ++i) acc += lh[i] * hd[i].d;
                w[k] = acc;
            }
        }
        // mu_h = (dC_h/dg_h)^T lambda_h and dJ/dQ, transposed exactly (the
        // h-only adjoint's code; Cumulants-1st needs the post-collision
        // state); the central-moment kinds get w from the same z
        double dth = 0.0;
        R muh[QH];
        if constexpr (CUM) {
            R hp[QH];
#pragma unroll
            for (int i = 0; i < QH; ++i) hp[i] = hpre[i];
            collide_h<R, QH, true>(hp, ux, uy, uz, Q, p);
            h_collision_transpose<R, QH, CUM>(lh, hp, ux, uy, uz, Q, p, muh, dth);
        } else {
            h_transpose_and_velocity<R, QH>(lh, hpre, ux, uy, uz, Q, p, muh, dth, w);
        }
        wbuf[n] = w[0];
        wbuf[N + n] = w[1];
        wbuf[2 * N + n] = w[2];
        // (a Zou-He inlet node writes the adjoint of its full arrival vector
        // here; k_zou_he_adjoint then transposes the rule that built it)
#pragma unroll
        for (int i = 0; i < QH; ++i) muh_out[i * N + n] = muh[i];
        if (dtheta) dtheta[n] += dth;
    } else {
        const R w[3] = {wbuf[n], wbuf[N + n], wbuf[2 * N + n]};
        // G_k for the ten unit-moment perturbations (k < 10) and the force (10..12)
        R G[13];
        collide_f_adjoint<R>(g, p, lf, w, G);
#pragma unroll
        for (int d = 0; d < 3; ++d) acc6[(size_t)n * 6 + d] += (double)G[10 + d];
        R mf[27];
        moments_transpose_f<R>(G, mf);
#pragma unroll
        for (int b = 0; b < 27; ++b) muf_out[b * N + n] = mf[b];
    }
}

// The Zou-He transpose of every inlet node of a level of the coupled sweep,
// after k_adjoint_flow (one thread per inlet node, in place; it would raise
// the register count of the whole sweep kernel if done there)
template <typename R, int QH>
__global__ void __launch_bounds__(kBlock) k_zou_he_adjoint(R* __restrict__ muf, R* __restrict__ muh,
                                                            const R* __restrict__ gf, const R* __restrict__ gh,
                                                            const uint8_t* __restrict__ flags,
                                                            double* __restrict__ acc6, const DevParams p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.ny * p.nz) return;
    const int n = p.nx * i;  // x = 0, row i = y + ny z
    if ((flags[n] & 3) != T_INLET) return;
    const int N = p.N;
    R g[27], h[QH], mf[27], mh[QH];
    const R* inl = gf + (size_t)10 * N;  // the inlet nodes' arrivals [27][ny nz]
#pragma unroll
    for (int a = 0; a < 27; ++a) {
        g[a] = inl[(size_t)a * p.ny * p.nz + i];
        mf[a] = muf[a * N + n];
    }
#pragma unroll
    for (int k = 0; k < QH; ++k) {
        h[k] = gh[k * N + n];
        mh[k] = muh[k * N + n];
    }
    zou_he_transpose_coupled<R, QH>(g, h, mf, mh, p, acc6 + (size_t)n * 6 + 3);
#pragma unroll
    for (int a = 0; a < 27; ++a) muf[a * N + n] = mf[a];
#pragma unroll
    for (int k = 0; k < QH; ++k) muh[k * N + n] = mh[k];
}

template <typename R, int QH>
cudaError_t launch_adjoint_flow(const Buffers& b, const DevParams& p, const R* f_level, const R* h_level,
                                const R* muf_next, const R* muh_next, R* muf_out, R* muh_out, AdjObjective obj,
                                double* dtheta, double* acc6, const R* din, R* wbuf, cudaStream_t s) {
    const int grid = (p.N + kBlock - 1) / kBlock;
#define LBM_ADJF_ARGS                                                                                            \
    muf_next, muh_next, muf_out, muh_out, f_level, h_level, b.theta, dtheta, acc6, din, wbuf, b.flags,          \
        b.seg_base, b.wmask, b.woff, b.lq, b.lwall, b.rseg_base, b.rmask, b.roff, b.rlink, b.dlink, obj, p
    if (p.hkind == 3) {
        k_adjoint_flow<R, QH, true, 1><<<grid, kBlock, 0, s>>>(LBM_ADJF_ARGS);
        k_adjoint_flow<R, QH, true, 2><<<grid, kBlock, 0, s>>>(LBM_ADJF_ARGS);
    } else {
        k_adjoint_flow<R, QH, false, 1><<<grid, kBlock, 0, s>>>(LBM_ADJF_ARGS);
        k_adjoint_flow<R, QH, false, 2><<<grid, kBlock, 0, s>>>(LBM_ADJF_ARGS);
    }
#undef LBM_ADJF_ARGS
    if (p.zou_he && f_level) {
        const int rows = p.ny * p.nz;
        k_zou_he_adjoint<R, QH><<<(rows + kBlock - 1) / kBlock, kBlock, 0, s>>>(muf_out, muh_out, f_level, h_level,
                                                                              b.flags, acc6, p);
    }
    return cudaGetLastError();
}

// copy of the post-collision h deviations (storage S) into an adjoint record
template <typename S, int QH>
__global__ void k_record_h(const S* __restrict__ hA, typename Acc<S>::R* __restrict__ rec, const DevParams p) {
    using R = typename Acc<S>::R;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)QH * p.N) return;
    rec[i] = ld<R>(hA + i);
}

template <typename S, int QH>
cudaError_t launch_record_h(const Buffers& b, const DevParams& p, void* rec, cudaStream_t s) {
    const size_t total = (size_t)QH * p.N;
    const unsigned grid = (unsigned)((total + kBlock - 1) / kBlock);
    k_record_h<S, QH><<<grid, kBlock, 0, s>>>((const S*)b.hA, (typename Acc<S>::R*)rec, p);
    return cudaGetLastError();
}

template <int NV>
__global__ void k_reduce_accumulate(const double* __restrict__ part, int nparts, int pick, double weight,
                                    double* __restrict__ acc) {
    __shared__ double sh[32 * NV];
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += part[i * NV + k];
    block_sum<NV>(v, sh);
    if (threadIdx.x == 0) acc[0] += weight * v[pick];
}

// x-flux sum e_x h through the plane x = plane (Sec. 4.4 section flux; the
// shift w T_ref carries no x-flux)
template <typename S, int QH>
__global__ void __launch_bounds__(kRedThreads) k_section_flux(const S* __restrict__ hA,
                                                              const uint8_t* __restrict__ flags, int plane,
                                                              double* __restrict__ part, const DevParams p) {
    using R = typename Acc<S>::R;
    __shared__ double sh[32];
    double v[1] = {0.0};
    const size_t N = (size_t)p.N;
    const int nrow = p.ny * p.nz;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrow; r += gridDim.x * blockDim.x) {
        const int n = plane + p.nx * r;
        if ((flags[n] & 3) == T_SOLID) continue;
#pragma unroll
        for (int i = 0; i < QH; ++i) {
            const int ex = EX(HDIR<QH>(i));
            if (ex != 0) v[0] += (double)ex * (double)ld<R>(hA + i * N + n);
        }
    }
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

template <typename S, int QH>
cudaError_t launch_objective(const Buffers& b, const DevParams& p, AdjObjective obj, double* scratch, double* acc,
                             cudaStream_t s) {
    if (obj.kind == 2) {
        k_wall_force<S><<<kRedBlocks, kRedThreads, 0, s>>>((const S*)b.fA, b.wnode, b.wmask, b.woff, b.lq, b.lwall,
                                                          b.nw, obj.wall, scratch, p);
        k_reduce_accumulate<3><<<1, 1024, 0, s>>>(scratch, kRedBlocks, obj.comp, obj.weight, acc);
        return cudaGetLastError();
    }
    if (obj.kind == 0)
        k_surface_flux<S, QH><<<kRedBlocks, kRedThreads, 0, s>>>((const S*)b.hA, b.wnode, b.wmask, b.woff, b.lq,
                                                                b.lwall, b.Twall, b.nw, obj.wall, scratch, p);
    else
        k_section_flux<S, QH><<<kRedBlocks, kRedThreads, 0, s>>>((const S*)b.hA, b.flags, obj.plane, scratch, p);
    k_reduce_accumulate<1><<<1, 1024, 0, s>>>(scratch, kRedBlocks, 0, obj.weight, acc);
    return cudaGetLastError();
}

#endif  // LBM_KERNEL_TU

}  // namespace lbmd
