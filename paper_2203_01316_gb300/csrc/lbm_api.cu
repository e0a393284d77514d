// Host implementation of the C ABI declared in include/lbm.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"

using lbmd::Acc;
using lbmd::Buffers;
using lbmd::DevParams;

struct lbm_ctx {
    lbm_params p{};
    int N = 0, qh = 27;
    size_t ssize = 4;  // bytes per stored value
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    void* f[2] = {nullptr, nullptr};  // population arrays (inside guarded allocations)
    void* h[2] = {nullptr, nullptr};
    void* f_alloc[2] = {nullptr, nullptr};
    void* h_alloc[2] = {nullptr, nullptr};
    int cur_f = 0, cur_h = 0;  // f[cur_f], h[cur_h]: post-collision state of the current level
    uint8_t* d_flags = nullptr;
    int nw = 0;
    int32_t* d_wnode = nullptr;
    int32_t* d_segbase = nullptr;
    uint32_t* d_wmask = nullptr;
    int32_t* d_woff = nullptr;
    int64_t nl = 0;
    float* d_lq = nullptr;
    int32_t* d_lwall = nullptr;
    int32_t* d_rsegbase = nullptr;  // adjoint: reverse (x_f) link table
    uint32_t* d_rmask = nullptr;
    int32_t* d_roff = nullptr;
    int32_t* d_rlink = nullptr;
    double* d_dlink = nullptr;      // adjoint: per link dJ/dT_w accumulators
    double* d_flowacc = nullptr;    // coupled adjoint: per node (dJ/dF, dJ/du_in) accumulators, [N][6]
    void* d_din = nullptr;          // coupled adjoint: d(inlet state)/du_in, R[3][27 + qh]
    void* d_wflow = nullptr;        // coupled adjoint: velocity derivative of the h step, R[3][N]
    uint32_t* d_stepctr = nullptr;  // 16-bit storage: the time level replayed step graphs read
    std::vector<double> h_din;      // the uploaded copy of d_din
    int n_walls = 1;
    float* d_Twall = nullptr;
    std::vector<float> Twall{0.0f};
    float* d_theta = nullptr;
    void* d_inlet = nullptr;  // R[27 + qh]
    double* d_scratch = nullptr;  // 3 * kRedBlocks partials + 4 results
    double* d_stage = nullptr;    // 5 * N doubles for host-side outputs
    int64_t n_fluid_like = 0;     // non-solid node count
    bool geometry = false, initialised = false;
    std::vector<int32_t> h_lnode, h_ldir, h_lwall;
    std::vector<float> h_lq;
    DevParams dp{};
    std::string err;
    // allocation fault injection (tests): LBM_FAULT_ALLOC=k in the environment
    // at lbm_create makes the context's k-th device allocation report out of
    // memory without allocating
    long fault_alloc = 0;
    long n_alloc = 0;
    // CUDA graphs of two plain steps (lbm_step, LBM_STEP_AUTO): replayed
    // while the launches they captured stay the same, i.e. while buffers()
    // and dp (but for its step counter) match what was captured
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        lbmd::Buffers b{};
        lbmd::DevParams p{};
    } graphs[2];
    int graph_next = 0;
    bool graph_broken = false;  // capture failed once: plain launches from then on
};

static std::string g_create_err;

// user flag of a symmetry-row node (stored as solid on the device)
static constexpr uint8_t kMirror = 4;

// message slot of calls made without a context (read with lbm_last_error(NULL))
void lbm_internal_set_global_error(const std::string& msg) { g_create_err = msg; }

namespace {

// every device allocation of a context goes through here (fault injection)
template <typename T> cudaError_t dev_alloc(lbm_ctx* c, T** p, size_t bytes) {
    if (c->fault_alloc > 0 && ++c->n_alloc == c->fault_alloc) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc((void**)p, bytes);
}

// multiplier and shift of node_xyz's division by d (see DevParams::mx)
static void fast_divisor(int d, uint32_t& m, int& s) {
    if (d <= 1) {
        m = 0;
        s = 0;
        return;
    }
    int l = 1;
    while ((int64_t(1) << l) < d) ++l;
    const uint64_t num = uint64_t(1) << (31 + l);
    m = (uint32_t)((num + (uint64_t)d - 1) / (uint64_t)d);
    s = l - 1;
}

template <typename S_, int Q_> struct Tag {
    using S = S_;
    static constexpr int Q = Q_;
};

template <typename Fn> cudaError_t dispatch(const lbm_ctx* c, Fn&& fn) {
    const bool q27 = c->qh == 27;
    switch (c->p.storage) {
        case LBM_F32: return q27 ? fn(Tag<float, 27>{}) : fn(Tag<float, 7>{});
        case LBM_F64: return q27 ? fn(Tag<double, 27>{}) : fn(Tag<double, 7>{});
        case LBM_F16_SHIFTED: return q27 ? fn(Tag<__half, 27>{}) : fn(Tag<__half, 7>{});
        default: return q27 ? fn(Tag<__nv_bfloat16, 27>{}) : fn(Tag<__nv_bfloat16, 7>{});
    }
}

lbm_status fail(lbm_ctx* c, lbm_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_err = msg;
    return s;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* where) {
    return fail(c, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                      \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

Buffers buffers(const lbm_ctx* c) {
    Buffers b{};
    b.fA = c->f[c->cur_f];
    b.fB = c->f[1 - c->cur_f];
    b.hA = c->h[c->cur_h];
    b.hB = c->h[1 - c->cur_h];
    b.flags = c->d_flags;
    b.theta = c->d_theta;
    b.inlet_post = c->d_inlet;
    b.wnode = c->d_wnode;
    b.seg_base = c->d_segbase;
    b.wmask = c->d_wmask;
    b.woff = c->d_woff;
    b.lq = c->d_lq;
    b.lwall = c->d_lwall;
    b.Twall = c->d_Twall;
    b.nw = c->nw;
    b.rseg_base = c->d_rsegbase;
    b.rmask = c->d_rmask;
    b.roff = c->d_roff;
    b.rlink = c->d_rlink;
    b.dlink = c->d_dlink;
    b.urec = nullptr;
    return b;
}

// 1-D equilibrium weight of velocity e at velocity u (product form of the
// discrete Maxwellian of Appendix A)
double w1eq(int e, double u) {
    const double cs2 = 1.0 / 3.0;
    return e == 0 ? 1.0 - u * u - cs2 : 0.5 * (u * u + e * u + cs2);
}

// derivative of w1eq with respect to u
double dw1eq(int e, double u) { return e == 0 ? -2.0 * u : u + 0.5 * e; }

// d(inlet post-collision state)/du_in,d for d = 0, 1, 2: [3][27 + qh]
std::vector<double> inlet_derivative(const lbm_ctx* c) {
    const int qh = c->qh;
    std::vector<double> v((size_t)3 * (27 + qh), 0.0);
    const double* u = c->dp.uin;
    const double T = c->dp.Tin;
    for (int d = 0; d < 3; ++d) {
        double* row = v.data() + (size_t)d * (27 + qh);
        for (int a = 0; a < 27; ++a) {
            const int e[3] = {lbmd::EX(a), lbmd::EY(a), lbmd::EZ(a)};
            double prod = 1.0;
            for (int k = 0; k < 3; ++k) prod *= (k == d) ? dw1eq(e[k], u[k]) : w1eq(e[k], u[k]);
            row[a] = prod;
            if (qh == 27) row[27 + a] = T * prod;
        }
        if (qh == 7) {
            row[27] = -2.0 * T * u[d];
            row[28 + d] = 0.5 * T * (2.0 * u[d] + 1.0);
            row[31 + d] = 0.5 * T * (2.0 * u[d] - 1.0);
        }
    }
    return v;
}

// inlet post-collision deviations (f^eq(1, u_in) - w rho0, h^eq(T_in, u_in) - w Tref)
lbm_status upload_inlet(lbm_ctx* c) {
    std::vector<double> v(27 + c->qh);
    const double* u = c->dp.uin;
    for (int a = 0; a < 27; ++a) {
        const int ex = lbmd::EX(a), ey = lbmd::EY(a), ez = lbmd::EZ(a);
        v[a] = w1eq(ex, u[0]) * w1eq(ey, u[1]) * w1eq(ez, u[2]) - lbmd::W27(a) * c->dp.rho0;
    }
    const double T = c->dp.Tin, cs2 = 1.0 / 3.0;
    if (c->qh == 27) {
        for (int a = 0; a < 27; ++a)
            v[27 + a] = T * w1eq(lbmd::EX(a), u[0]) * w1eq(lbmd::EY(a), u[1]) * w1eq(lbmd::EZ(a), u[2]) -
                        lbmd::W27(a) * c->dp.Tref;
    } else {
        double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        v[27] = T * (1.0 - 3.0 * cs2 - u2);
        for (int d = 0; d < 3; ++d) {
            v[28 + d] = 0.5 * T * (cs2 + u[d] * u[d] + u[d]) - c->dp.Tref / 6.0;
            v[31 + d] = 0.5 * T * (cs2 + u[d] * u[d] - u[d]) - c->dp.Tref / 6.0;
        }
    }
    if (c->p.storage == LBM_F64) {
        CK(cudaMemcpyAsync(c->d_inlet, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream),
           "inlet upload");
    } else {
        std::vector<float> vf(v.begin(), v.end());
        CK(cudaMemcpyAsync(c->d_inlet, vf.data(), vf.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream),
           "inlet upload");
    }
    CK(cudaStreamSynchronize(c->stream), "inlet upload");
    return LBM_OK;
}

void free_geometry(lbm_ctx* c) {
    cudaFree(c->d_wnode);
    cudaFree(c->d_segbase);
    cudaFree(c->d_wmask);
    cudaFree(c->d_woff);
    cudaFree(c->d_lq);
    cudaFree(c->d_lwall);
    cudaFree(c->d_rsegbase);
    cudaFree(c->d_rmask);
    cudaFree(c->d_roff);
    cudaFree(c->d_rlink);
    cudaFree(c->d_dlink);
    c->d_rsegbase = nullptr;
    c->d_rmask = nullptr;
    c->d_roff = nullptr;
    c->d_rlink = nullptr;
    c->d_dlink = nullptr;
    c->d_wnode = nullptr;
    c->d_segbase = nullptr;
    c->d_wmask = nullptr;
    c->d_woff = nullptr;
    c->d_lq = nullptr;
    c->d_lwall = nullptr;
    c->nw = 0;
    c->dp.nwall = 0;
    c->nl = 0;
}

template <typename T> lbm_status to_host(lbm_ctx* c, const T* src, size_t count, int is_device, std::vector<T>& out) {
    out.resize(count);
    if (count == 0) return LBM_OK;
    if (!src) return fail(c, LBM_ERR_INVALID, "null array");
    if (is_device) {
        CK(cudaMemcpy(out.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost), "device->host copy");
    } else {
        std::memcpy(out.data(), src, count * sizeof(T));
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_create(const lbm_params* params, lbm_ctx** out) {
    g_create_err.clear();
    if (!params || !out) return fail(nullptr, LBM_ERR_INVALID, "null argument");
    *out = nullptr;
    lbm_params p = *params;
    if (p.nx < 1 || p.ny < 1 || p.nz < 1) return fail(nullptr, LBM_ERR_INVALID, "grid dimensions must be >= 1");
    const int64_t N = (int64_t)p.nx * p.ny * p.nz;
    if (N * 27 >= (int64_t(1) << 31)) return fail(nullptr, LBM_ERR_INVALID, "nx*ny*nz*27 must stay below 2^31");
    if (!p.periodic_x && p.nx < 4) return fail(nullptr, LBM_ERR_INVALID, "an inlet/outlet channel needs nx >= 4");
    if (p.lat_h != 27 && p.lat_h != 7) return fail(nullptr, LBM_ERR_INVALID, "lat_h must be 27 or 7");
    if (p.hkind < 0 || p.hkind > 3) return fail(nullptr, LBM_ERR_INVALID, "unknown hkind");
    if (p.storage < 0 || p.storage > 3) return fail(nullptr, LBM_ERR_INVALID, "unknown storage");
    if (p.step_kernel < 0 || p.step_kernel > 1) return fail(nullptr, LBM_ERR_INVALID, "unknown step_kernel");
    if (p.wall_bc < 0 || p.wall_bc > 2) return fail(nullptr, LBM_ERR_INVALID, "unknown wall_bc");
    if (p.inlet_bc < 0 || p.inlet_bc > 1) return fail(nullptr, LBM_ERR_INVALID, "unknown inlet_bc");
    if (!(p.nu > 0.0) || !std::isfinite(p.nu)) return fail(nullptr, LBM_ERR_INVALID, "nu must be > 0");
    double k = p.k, Pr = p.Pr;
    if (k > 0.0 && Pr > 0.0) {
        if (std::fabs(p.nu / k - Pr) > 1e-12 * Pr) return fail(nullptr, LBM_ERR_INVALID, "nu/k disagrees with Pr");
    } else if (k > 0.0) {
        Pr = p.nu / k;
    } else if (Pr > 0.0) {
        k = p.nu / Pr;
    } else {
        return fail(nullptr, LBM_ERR_INVALID, "one of k, Pr must be > 0");
    }
    if (!(k > 0.0) || !std::isfinite(k)) return fail(nullptr, LBM_ERR_INVALID, "k must be > 0");
    if (!(p.omega_bulk > 0.0 && p.omega_bulk < 2.0))
        return fail(nullptr, LBM_ERR_INVALID, "omega_bulk must lie in (0, 2)");
    p.k = k;
    p.Pr = Pr;

    lbm_ctx* ctx = new lbm_ctx();
    lbm_ctx* c = ctx;
    c->p = p;
    c->N = (int)N;
    c->qh = p.lat_h;
    c->ssize = p.storage == LBM_F64 ? 8 : (p.storage == LBM_F32 ? 4 : 2);
    if (const char* fa = std::getenv("LBM_FAULT_ALLOC")) c->fault_alloc = std::strtol(fa, nullptr, 10);
    cudaGetDevice(&c->device);
    auto bail = [&](lbm_status s) {
        g_create_err = c->err;
        lbm_destroy(ctx);
        return s;
    };
    if (p.cuda_stream) {
        c->stream = (cudaStream_t)p.cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "stream create"));
        c->own_stream = true;
    }
    const size_t fb = (size_t)27 * N * c->ssize, hb = (size_t)c->qh * N * c->ssize;
    for (int i = 0; i < 2; ++i) {
        if (dev_alloc(c, &c->f_alloc[i], fb) != cudaSuccess || dev_alloc(c, &c->h_alloc[i], hb) != cudaSuccess)
            return bail(fail(c, LBM_ERR_NOMEM, "population arrays: out of device memory"));
        cudaMemsetAsync(c->f_alloc[i], 0, fb, c->stream);
        cudaMemsetAsync(c->h_alloc[i], 0, hb, c->stream);
        c->f[i] = c->f_alloc[i];
        c->h[i] = c->h_alloc[i];
    }
    if (dev_alloc(c, &c->d_flags, N) != cudaSuccess ||
        dev_alloc(c, &c->d_inlet, (27 + 27) * sizeof(double)) != cudaSuccess ||
        dev_alloc(c, &c->d_scratch, (3 * lbmd::kRedBlocks + 4) * sizeof(double)) != cudaSuccess ||
        dev_alloc(c, &c->d_Twall, sizeof(float)) != cudaSuccess)
        return bail(fail(c, LBM_ERR_NOMEM, "context buffers: out of device memory"));
    if (c->ssize == 2 && dev_alloc(c, &c->d_stepctr, sizeof(uint32_t)) != cudaSuccess)
        return bail(fail(c, LBM_ERR_NOMEM, "step counter: out of device memory"));

    cudaMemsetAsync(c->d_flags, 0, N, c->stream);
    cudaMemsetAsync(c->d_Twall, 0, sizeof(float), c->stream);

    DevParams& d = c->dp;
    d.nx = p.nx;
    d.ny = p.ny;
    d.nz = p.nz;
    d.N = (int)N;
    d.periodic_x = p.periodic_x ? 1 : 0;
    d.omega1 = 1.0 / (3.0 * p.nu + 0.5);
    d.omega_bulk = p.omega_bulk;
    const double sH = 1.0 / (3.0 * k + 0.5);  // Sec. 2.1.1: s^H = 1/(k/cs^2 + 1/2)
    for (int o = 0; o <= 6; ++o) {
        double s = 1.0;
        if (p.hkind == LBM_H_CM_SRT) s = sH;
        else if (p.hkind == LBM_H_CM_1ST || p.hkind == LBM_H_CUM_1ST) s = (o == 1) ? sH : 1.0;
        else s = (o % 2 == 1) ? sH : 1.0;
        d.sh[o] = s;
    }
    d.rho0 = p.rho0;
    d.Tref = p.T_ref;
    d.stochastic = p.round_nearest ? 0 : 1;
    d.hkind = p.hkind;
    d.wall_bc = p.wall_bc;
    d.zou_he = (p.inlet_bc == LBM_INLET_ZOU_HE && !p.periodic_x) ? 1 : 0;
    d.nwall = 0;
    d.step_ctr = nullptr;
    fast_divisor(p.nx, d.mx, d.sx);
    fast_divisor(p.ny, d.my, d.sy);
    d.step = 0;
    for (int i = 0; i < 3; ++i) d.F[i] = d.uin[i] = 0.0;
    d.Tin = 0.0;
    lbmd::sync_float_params(d);
    lbm_status s = upload_inlet(c);
    if (s != LBM_OK) return bail(s);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "create"));
    *out = ctx;
    return LBM_OK;
}

lbm_status lbm_destroy(lbm_ctx* c) {
    if (!c) return LBM_OK;
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int i = 0; i < 2; ++i) {
        cudaFree(c->f_alloc[i]);
        cudaFree(c->h_alloc[i]);
    }
    free_geometry(c);
    cudaFree(c->d_flags);
    cudaFree(c->d_inlet);
    cudaFree(c->d_scratch);
    cudaFree(c->d_stage);
    cudaFree(c->d_Twall);
    cudaFree(c->d_theta);
    cudaFree(c->d_flowacc);
    cudaFree(c->d_din);
    cudaFree(c->d_wflow);
    cudaFree(c->d_stepctr);
    for (auto& gr : c->graphs)
        if (gr.exec) cudaGraphExecDestroy(gr.exec);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_ctx* c, const uint8_t* flags, int64_t n_links, const int32_t* link_node,
                            const int32_t* link_dir, const float* link_q, const int32_t* link_wall, int n_walls,
                            int is_device) {
    if (!c) return LBM_ERR_INVALID;
    DeviceGuard g(c->device);
    if (n_links < 0 || n_walls < 1 || n_walls > (1 << 20)) return fail(c, LBM_ERR_INVALID, "bad n_links or n_walls");
    const int N = c->N, nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    std::vector<uint8_t> fl;
    std::vector<int32_t> ln, ld, lw;
    std::vector<float> lq;
    lbm_status s;
    if ((s = to_host(c, flags, (size_t)N, is_device, fl)) != LBM_OK) return s;
    if ((s = to_host(c, link_node, (size_t)n_links, is_device, ln)) != LBM_OK) return s;
    if ((s = to_host(c, link_dir, (size_t)n_links, is_device, ld)) != LBM_OK) return s;
    if ((s = to_host(c, link_q, (size_t)n_links, is_device, lq)) != LBM_OK) return s;
    if ((s = to_host(c, link_wall, (size_t)n_links, is_device, lw)) != LBM_OK) return s;

    auto nbr = [&](int n, int ex, int ey, int ez) -> int {
        int x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
        x += ex;
        y = (y + ey + ny) % ny;
        z = (z + ez + nz) % nz;
        if (c->p.periodic_x) x = (x + nx) % nx;
        else if (x < 0 || x >= nx) return -1;
        return x + nx * (y + ny * z);
    };
    int64_t nonsolid = 0;
    bool mirror_row[2] = {false, false};  // symmetry rows y = 0, y = ny - 1
    for (int n = 0; n < N; ++n) {
        const uint8_t t = fl[n];
        if (t > 4) return fail(c, LBM_ERR_INVALID, "flag value above 4 at node " + std::to_string(n));
        const int x = n % nx, y = (n / nx) % ny;
        if (t == kMirror) {
            if (ny < 3 || (y != 0 && y != ny - 1))
                return fail(c, LBM_ERR_INVALID, "symmetry node outside the rows y = 0 and y = ny-1");
            const int src = n + (y == 0 ? nx : -nx);
            if (fl[src] == lbmd::T_SOLID || fl[src] == kMirror)
                return fail(c, LBM_ERR_INVALID, "the node beside symmetry node " + std::to_string(n) + " is solid");
            mirror_row[y == 0 ? 0 : 1] = true;
            continue;
        }
        if (c->p.periodic_x) {
            if (t == lbmd::T_INLET || t == lbmd::T_OUTLET)
                return fail(c, LBM_ERR_INVALID, "inlet/outlet flag in a periodic-x grid");
        } else {
            if ((x == 0) != (t == lbmd::T_INLET)) return fail(c, LBM_ERR_INVALID, "the x=0 plane must be all inlet");
            if ((x == nx - 1) != (t == lbmd::T_OUTLET))
                return fail(c, LBM_ERR_INVALID, "the x=nx-1 plane must be all outlet");
            if (x == nx - 2 && t == lbmd::T_SOLID) return fail(c, LBM_ERR_INVALID, "solid node next to the outlet");
            if (c->dp.zou_he && x == 1 && t == lbmd::T_SOLID)
                return fail(c, LBM_ERR_INVALID, "solid node next to a Zou-He inlet");
        }
        if (t != lbmd::T_SOLID) ++nonsolid;
    }
    for (int side = 0; side < 2; ++side) {  // a symmetry row is whole
        if (!mirror_row[side]) continue;
        const int y = side == 0 ? 0 : ny - 1;
        for (int z = 0; z < nz; ++z)
            for (int x = 0; x < nx; ++x)
                if (fl[x + (size_t)nx * (y + (size_t)ny * z)] != kMirror)
                    return fail(c, LBM_ERR_INVALID, "a symmetry row must cover the whole x-z row");
    }
    // links: validate, sort by (node, dir)
    std::vector<int64_t> order(n_links);
    for (int64_t l = 0; l < n_links; ++l) {
        const int n = ln[l], a = ld[l];
        if (n < 0 || n >= N || a < 1 || a >= 27) return fail(c, LBM_ERR_INVALID, "link node/dir out of range");
        if (fl[n] != lbmd::T_FLUID) return fail(c, LBM_ERR_INVALID, "link from a non-fluid node " + std::to_string(n));
        {
            const int y = (n / nx) % ny;
            if ((mirror_row[0] && y == 1) || (mirror_row[1] && y == ny - 2))
                return fail(c, LBM_ERR_INVALID, "wall link from a node next to a symmetry row");
        }
        const int t = nbr(n, lbmd::EX(a), lbmd::EY(a), lbmd::EZ(a));
        if (t < 0 || fl[t] != lbmd::T_SOLID)
            return fail(c, LBM_ERR_INVALID, "link target is not solid (node " + std::to_string(n) + ")");
        if (!(lq[l] > 0.0f && lq[l] <= 1.0f)) return fail(c, LBM_ERR_INVALID, "link q outside (0,1]");
        if (lw[l] < 0 || lw[l] >= n_walls) return fail(c, LBM_ERR_INVALID, "link wall id out of range");
        order[l] = l;
    }
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        return ln[a] != ln[b] ? ln[a] < ln[b] : ld[a] < ld[b];
    });
    std::vector<int32_t> wnode, woff;
    std::vector<uint32_t> wmask;
    std::vector<int32_t> sn(n_links), sd(n_links), sw(n_links);
    std::vector<float> sq(n_links);
    for (int64_t i = 0; i < n_links; ++i) {
        const int64_t l = order[i];
        sn[i] = ln[l];
        sd[i] = ld[l];
        sq[i] = lq[l];
        sw[i] = lw[l];
        if (i > 0 && sn[i] == sn[i - 1] && sd[i] == sd[i - 1]) return fail(c, LBM_ERR_INVALID, "duplicate link");
        if (i == 0 || sn[i] != sn[i - 1]) {
            wnode.push_back(sn[i]);
            woff.push_back((int32_t)i);
            wmask.push_back(0u);
        }
        wmask.back() |= 1u << sd[i];
    }
    // completeness: every fluid->solid link listed; outlet nodes see no solid.
    // Nested loops with per-row neighbour offsets (y, z periodic).
    std::vector<uint8_t> iflags(fl);
    for (auto& v : iflags)
        if (v == kMirror) v = lbmd::T_SOLID;  // the step never writes a symmetry node
    size_t wi = 0;
    const int64_t plane = (int64_t)nx * ny;
    for (int z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y) {
            int64_t rowoff[27];  // index offset of the neighbour row of direction a
            for (int a = 0; a < 27; ++a) {
                const int yy = (y + lbmd::EY(a) + ny) % ny, zz = (z + lbmd::EZ(a) + nz) % nz;
                rowoff[a] = (int64_t)zz * plane + (int64_t)yy * nx;
            }
            const int64_t row = (int64_t)z * plane + (int64_t)y * nx;
            for (int x = 0; x < nx; ++x) {
                const int n = (int)(row + x);
                if (fl[n] == lbmd::T_SOLID || fl[n] == lbmd::T_INLET || fl[n] == kMirror) continue;
                uint32_t m = 0;
                for (int a = 1; a < 27; ++a) {
                    int xx = x + lbmd::EX(a);
                    if (xx < 0 || xx >= nx) {
                        if (!c->p.periodic_x) continue;
                        xx = (xx + nx) % nx;
                    }
                    if (fl[rowoff[a] + xx] == lbmd::T_SOLID) m |= 1u << a;
                }
                if (!m) continue;
                if (fl[n] == lbmd::T_OUTLET) return fail(c, LBM_ERR_INVALID, "outlet node next to a solid");
                while (wi < wnode.size() && wnode[wi] < n) ++wi;
                if (wi >= wnode.size() || wnode[wi] != n || wmask[wi] != m)
                    return fail(c, LBM_ERR_INVALID,
                                "fluid->solid links of node " + std::to_string(n) + " are not all listed");
                iflags[n] |= lbmd::F_WALL;
            }
        }
    }
    // adjoint reverse table: node y = x - e_a of each link (x, a) with
    // q <= 1/2 whose y is fluid or outlet (Eq. IABB reads h*_a(y) there)
    // the first-order variants bounce back half-way: q = 1/2 on the device
    std::vector<float> qdev(sq);
    if (c->p.wall_bc != 0) std::fill(qdev.begin(), qdev.end(), 0.5f);
    std::vector<std::pair<int64_t, int32_t>> rev;  // (y*32 + a, link index)
    for (int64_t i = 0; i < n_links; ++i) {
        if (!(qdev[i] < 0.5f)) continue;  // coefficient 1 - 2q vanishes at q = 1/2
        const int a = sd[i];
        const int yv = nbr(sn[i], -lbmd::EX(a), -lbmd::EY(a), -lbmd::EZ(a));
        if (yv < 0 || fl[yv] == lbmd::T_SOLID || fl[yv] == lbmd::T_INLET) continue;
        rev.push_back({(int64_t)yv * 32 + a, (int32_t)i});
    }
    std::sort(rev.begin(), rev.end());
    std::vector<int32_t> rnode, roff, rlink;
    std::vector<uint32_t> rmask;
    for (size_t i = 0; i < rev.size(); ++i) {
        const int yv = (int)(rev[i].first / 32), a = (int)(rev[i].first % 32);
        if (i == 0 || rnode.back() != yv) {
            rnode.push_back(yv);
            roff.push_back((int32_t)i);
            rmask.push_back(0u);
        }
        rmask.back() |= 1u << a;
        rlink.push_back(rev[i].second);
        iflags[yv] |= lbmd::F_RWALL;
    }
    // wall nodes before each 32-node segment (warp) of the step kernel
    const int nseg = (N + 31) / 32;
    std::vector<int32_t> segbase(nseg);
    {
        size_t k = 0;
        for (int sgm = 0; sgm < nseg; ++sgm) {
            while (k < wnode.size() && wnode[k] < sgm * 32) ++k;
            segbase[sgm] = (int32_t)k;
        }
    }
    std::vector<int32_t> rsegbase(nseg);
    {
        size_t k = 0;
        for (int sgm = 0; sgm < nseg; ++sgm) {
            while (k < rnode.size() && rnode[k] < sgm * 32) ++k;
            rsegbase[sgm] = (int32_t)k;
        }
    }
    // upload; until it completes the context has no geometry (a failure part
    // way through must not leave tables that later kernels would read)
    c->geometry = false;
    c->initialised = false;
    // from here on the old geometry is gone: a failure below leaves the
    // context without one (steps refused until a geometry is set)
    free_geometry(c);
    c->geometry = false;
    c->initialised = false;
    c->nw = (int)wnode.size();
    c->dp.nwall = c->nw;
    c->nl = n_links;
    CK(cudaMemcpyAsync(c->d_flags, iflags.data(), N, cudaMemcpyHostToDevice, c->stream), "flags upload");
    if (c->nw > 0) {
        if (dev_alloc(c, &c->d_wnode, c->nw * sizeof(int32_t)) != cudaSuccess ||
            dev_alloc(c, &c->d_wmask, c->nw * sizeof(uint32_t)) != cudaSuccess ||
            dev_alloc(c, &c->d_segbase, nseg * sizeof(int32_t)) != cudaSuccess ||
            dev_alloc(c, &c->d_woff, c->nw * sizeof(int32_t)) != cudaSuccess ||
            dev_alloc(c, &c->d_lq, n_links * sizeof(float)) != cudaSuccess ||
            dev_alloc(c, &c->d_lwall, n_links * sizeof(int32_t)) != cudaSuccess) {
            free_geometry(c);
            return fail(c, LBM_ERR_NOMEM, "wall tables: out of device memory");
        }
        CK(cudaMemcpyAsync(c->d_wnode, wnode.data(), c->nw * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream), "wall upload");
        CK(cudaMemcpyAsync(c->d_segbase, segbase.data(), nseg * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream), "wall upload");
        CK(cudaMemcpyAsync(c->d_wmask, wmask.data(), c->nw * sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream), "wall upload");
        CK(cudaMemcpyAsync(c->d_woff, woff.data(), c->nw * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream), "wall upload");
        CK(cudaMemcpyAsync(c->d_lq, qdev.data(), n_links * sizeof(float), cudaMemcpyHostToDevice, c->stream), "link upload");
        CK(cudaMemcpyAsync(c->d_lwall, sw.data(), n_links * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream), "link upload");
        if (dev_alloc(c, &c->d_dlink, n_links * sizeof(double)) != cudaSuccess ||
            dev_alloc(c, &c->d_rsegbase, nseg * sizeof(int32_t)) != cudaSuccess) {
            free_geometry(c);
            return fail(c, LBM_ERR_NOMEM, "adjoint tables: out of device memory");
        }
        CK(cudaMemsetAsync(c->d_dlink, 0, n_links * sizeof(double), c->stream), "link accumulators");
        CK(cudaMemcpyAsync(c->d_rsegbase, rsegbase.data(), nseg * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream),
           "reverse table upload");
        if (!rnode.empty()) {
            const size_t nr = rnode.size();
            if (dev_alloc(c, &c->d_rmask, nr * sizeof(uint32_t)) != cudaSuccess ||
                dev_alloc(c, &c->d_roff, nr * sizeof(int32_t)) != cudaSuccess ||
                dev_alloc(c, &c->d_rlink, rlink.size() * sizeof(int32_t)) != cudaSuccess) {
                free_geometry(c);
                return fail(c, LBM_ERR_NOMEM, "adjoint tables: out of device memory");
            }
            CK(cudaMemcpyAsync(c->d_rmask, rmask.data(), nr * sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream),
               "reverse table upload");
            CK(cudaMemcpyAsync(c->d_roff, roff.data(), nr * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream),
               "reverse table upload");
            CK(cudaMemcpyAsync(c->d_rlink, rlink.data(), rlink.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                               c->stream),
               "reverse table upload");
        }
    }
    if ((int)c->Twall.size() != n_walls) {
        cudaFree(c->d_Twall);
        c->d_Twall = nullptr;
        c->Twall.clear();
        if (dev_alloc(c, &c->d_Twall, n_walls * sizeof(float)) != cudaSuccess)
            return fail(c, LBM_ERR_NOMEM, "wall temperatures: out of device memory");
        c->Twall.assign(n_walls, 0.0f);
    }
    c->n_walls = n_walls;
    CK(cudaMemcpyAsync(c->d_Twall, c->Twall.data(), n_walls * sizeof(float), cudaMemcpyHostToDevice, c->stream), "wall T upload");
    CK(cudaStreamSynchronize(c->stream), "geometry upload");
    c->h_lnode = std::move(sn);
    c->h_ldir = std::move(sd);
    c->h_lq = std::move(sq);
    c->h_lwall = std::move(sw);
    c->n_fluid_like = nonsolid;
    c->dp.mirror_lo = mirror_row[0] ? 1 : 0;
    c->dp.mirror_hi = mirror_row[1] ? 1 : 0;
    c->geometry = true;
    c->initialised = false;
    return LBM_OK;
}

lbm_status lbm_build_spheres(lbm_ctx* c, int n_spheres, const double* centres, const double* radii,
                             const int32_t* wall_ids, int n_walls, uint8_t* flags_out) {
    if (!c) return LBM_ERR_INVALID;
    if (n_spheres < 0 || (n_spheres > 0 && (!centres || !radii)))
        return fail(c, LBM_ERR_INVALID, "bad sphere list");
    if (n_walls < 1) return fail(c, LBM_ERR_INVALID, "n_walls must be >= 1");
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    std::vector<lbmd::GeoSphere> sp(n_spheres);
    for (int i = 0; i < n_spheres; ++i) {
        const double R = radii[i];
        if (!(R > 0.0) || !(2.0 * R < ny) || !(2.0 * R < nz))
            return fail(c, LBM_ERR_INVALID, "sphere radius must be positive and below ny/2 and nz/2");
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(centres[3 * i + d])) return fail(c, LBM_ERR_INVALID, "sphere centre not finite");
        const int w = wall_ids ? wall_ids[i] : 0;
        if (w < 0 || w >= n_walls) return fail(c, LBM_ERR_INVALID, "sphere wall id out of range");
        sp[i] = {centres[3 * i], centres[3 * i + 1], centres[3 * i + 2], R, w};
    }
    DeviceGuard g(c->device);
    const int64_t N = c->N;
    const int nb = (int)((N + lbmd::kGeoBlock - 1) / lbmd::kGeoBlock);
    lbmd::GeoSphere* d_sp = nullptr;
    uint8_t* d_fl = nullptr;
    uint32_t* d_mask = nullptr;
    int* d_bsum = nullptr;
    int64_t* d_boff = nullptr;
    int32_t *d_node = nullptr, *d_dir = nullptr, *d_wall = nullptr;
    float* d_q = nullptr;
    auto release = [&]() {
        cudaFree(d_sp); cudaFree(d_fl); cudaFree(d_mask); cudaFree(d_bsum); cudaFree(d_boff);
        cudaFree(d_node); cudaFree(d_dir); cudaFree(d_q); cudaFree(d_wall);
    };
    lbm_status st = LBM_OK;
    int64_t total = 0;
    if (dev_alloc(c, &d_sp, std::max<size_t>(1, sp.size()) * sizeof(lbmd::GeoSphere)) != cudaSuccess ||
        dev_alloc(c, &d_fl, (size_t)N) != cudaSuccess || dev_alloc(c, &d_mask, (size_t)N * 4) != cudaSuccess ||
        dev_alloc(c, &d_bsum, (size_t)nb * 4) != cudaSuccess ||
        dev_alloc(c, &d_boff, (size_t)(nb + 1) * 8) != cudaSuccess) {
        release();
        return fail(c, LBM_ERR_NOMEM, "sphere geometry: out of device memory");
    }
    cudaError_t e = cudaSuccess;
    if (!sp.empty())
        e = cudaMemcpyAsync(d_sp, sp.data(), sp.size() * sizeof(lbmd::GeoSphere), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = lbmd::launch_sphere_flags(d_fl, d_mask, nx, ny, nz, c->p.periodic_x, d_sp, n_spheres, d_bsum, d_boff,
                                      c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, d_boff + nb, 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(c, e, "sphere geometry");
    }
    const size_t nl = (size_t)std::max<int64_t>(total, 1);
    if (dev_alloc(c, &d_node, nl * 4) != cudaSuccess || dev_alloc(c, &d_dir, nl * 4) != cudaSuccess ||
        dev_alloc(c, &d_q, nl * 4) != cudaSuccess || dev_alloc(c, &d_wall, nl * 4) != cudaSuccess) {
        release();
        return fail(c, LBM_ERR_NOMEM, "sphere geometry links: out of device memory");
    }
    e = lbmd::launch_sphere_links(d_mask, nx, ny, nz, d_sp, n_spheres, d_boff, d_node, d_dir, d_q, d_wall,
                                  c->stream);
    if (e == cudaSuccess && flags_out)
        e = cudaMemcpyAsync(flags_out, d_fl, (size_t)N, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(c, e, "sphere geometry links");
    }
    st = lbm_set_geometry(c, d_fl, total, d_node, d_dir, d_q, d_wall, n_walls, 1);
    release();
    return st;
}

lbm_status lbm_set_bc(lbm_ctx* c, int wall_id, double T_wall) {
    if (!c) return LBM_ERR_INVALID;
    DeviceGuard g(c->device);
    if (wall_id < 0 || wall_id >= (int)c->Twall.size()) return fail(c, LBM_ERR_INVALID, "wall id out of range");
    if (!std::isfinite(T_wall)) return fail(c, LBM_ERR_INVALID, "wall temperature not finite");
    c->Twall[wall_id] = (float)T_wall;
    CK(cudaMemcpyAsync(c->d_Twall + wall_id, &c->Twall[wall_id], sizeof(float), cudaMemcpyHostToDevice, c->stream),
       "wall T upload");
    CK(cudaStreamSynchronize(c->stream), "wall T upload");
    return LBM_OK;
}

lbm_status lbm_set_inlet(lbm_ctx* c, double ux, double uy, double uz, double T_in) {
    if (!c) return LBM_ERR_INVALID;
    DeviceGuard g(c->device);
    if (!std::isfinite(ux) || !std::isfinite(uy) || !std::isfinite(uz) || !std::isfinite(T_in))
        return fail(c, LBM_ERR_INVALID, "inlet state not finite");
    c->dp.uin[0] = ux;
    c->dp.uin[1] = uy;
    c->dp.uin[2] = uz;
    c->dp.Tin = T_in;
    lbmd::sync_float_params(c->dp);
    return upload_inlet(c);
}

lbm_status lbm_set_force(lbm_ctx* c, double Fx, double Fy, double Fz) {
    if (!c) return LBM_ERR_INVALID;
    if (!std::isfinite(Fx) || !std::isfinite(Fy) || !std::isfinite(Fz)) return fail(c, LBM_ERR_INVALID, "force not finite");
    c->dp.F[0] = Fx;
    c->dp.F[1] = Fy;
    c->dp.F[2] = Fz;
    lbmd::sync_float_params(c->dp);
    return LBM_OK;
}

lbm_status lbm_set_source(lbm_ctx* c, const float* theta, int is_device) {
    if (!c) return LBM_ERR_INVALID;
    DeviceGuard g(c->device);
    if (!theta) {
        CK(cudaStreamSynchronize(c->stream), "source clear");
        cudaFree(c->d_theta);
        c->d_theta = nullptr;
        return LBM_OK;
    }
    if (!c->d_theta && dev_alloc(c, &c->d_theta, (size_t)c->N * sizeof(float)) != cudaSuccess)
        return fail(c, LBM_ERR_NOMEM, "source: out of device memory");
    CK(cudaMemcpyAsync(c->d_theta, theta, (size_t)c->N * sizeof(float),
                       is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream),
       "source upload");
    CK(cudaStreamSynchronize(c->stream), "source upload");
    return LBM_OK;
}

static lbm_status ensure_stage(lbm_ctx* c) {
    if (!c->d_stage && dev_alloc(c, &c->d_stage, (size_t)5 * c->N * sizeof(double)) != cudaSuccess)
        return fail(c, LBM_ERR_NOMEM, "staging buffer: out of device memory");
    return LBM_OK;
}

lbm_status lbm_init_fields(lbm_ctx* c, const double* rho, const double* u, const double* T, int is_device) {
    if (!c) return LBM_ERR_INVALID;
    DeviceGuard g(c->device);
    if (!c->geometry) return fail(c, LBM_ERR_STATE, "set the geometry first");
    if (!rho || !u || !T) return fail(c, LBM_ERR_INVALID, "null field");
    const size_t N = (size_t)c->N;
    const double *dr = rho, *du = u, *dT = T;
    if (!is_device) {
        lbm_status s = ensure_stage(c);
        if (s != LBM_OK) return s;
        CK(cudaMemcpyAsync(c->d_stage, rho, N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "fields upload");
        CK(cudaMemcpyAsync(c->d_stage + N, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "fields upload");
        CK(cudaMemcpyAsync(c->d_stage + 4 * N, T, N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "fields upload");
        dr = c->d_stage;
        du = c->d_stage + N;
        dT = c->d_stage + 4 * N;
    }
    Buffers b = buffers(c);
    b.fB = c->f[c->cur_f];  // write the current level in place
    b.hB = c->h[c->cur_h];
    c->dp.step = 0;
    const DevParams p = c->dp;
    cudaStream_t s = c->stream;
    CK(dispatch(c, [&](auto tag) {
           using Tg = decltype(tag);
           return lbmd::launch_init<typename Tg::S, Tg::Q>(b, p, dr, du, dT, s);
       }),
       "init launch");
    if (!is_device) CK(cudaStreamSynchronize(c->stream), "init");
    c->initialised = true;
    return LBM_OK;
}

// the Zou-He inlet plane, after each step
static cudaError_t zou_he_inlet(lbm_ctx* c, const Buffers& b, const DevParams& p, bool advance_h) {
    if (!p.zou_he) return cudaSuccess;
    return dispatch(c, [&](auto tag) {
        using Tg = decltype(tag);
        return lbmd::launch_inlet<typename Tg::S, Tg::Q>(b, p, c->stream, advance_h);
    });
}

// symmetry rows take their mirrored populations before each step
static cudaError_t fill_mirror(lbm_ctx* c, const Buffers& b, const DevParams& p) {
    if (!p.mirror_lo && !p.mirror_hi) return cudaSuccess;
    return dispatch(c, [&](auto tag) {
        using Tg = decltype(tag);
        return lbmd::launch_mirror<typename Tg::S, Tg::Q>(b, p, c->stream);
    });
}

// the launches of one plain step (symmetry rows, the step, the Zou-He inlet)
// the time-level counter of replayed 16-bit step graphs: set before a run
// of replays, advanced inside each captured step
__global__ void k_step_counter(uint32_t* ctr, uint32_t value, int advance) {
    if (advance) *ctr += 1u;
    else *ctr = value;
}

// one plain step; in_graph: the step is being captured for replay, so with
// stochastically rounded 16-bit storage its kernels read the time level from
// the device counter, which the step advances first
static lbm_status step_once(lbm_ctx* c, bool in_graph = false) {
    const Buffers b = buffers(c);
    c->dp.step += 1;
    DevParams p = c->dp;
    cudaError_t e;
    if (in_graph && c->d_stepctr) {
        k_step_counter<<<1, 1, 0, c->stream>>>(c->d_stepctr, 0u, 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "step counter launch");
        p.step_ctr = c->d_stepctr;
    }
    if ((e = fill_mirror(c, b, p)) != cudaSuccess) return cuda_fail(c, e, "symmetry rows launch");
    e = dispatch(c, [&](auto tag) {
        using Tg = decltype(tag);
        return lbmd::launch_step<typename Tg::S, Tg::Q>(b, p, c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
    if ((e = zou_he_inlet(c, b, p, true)) != cudaSuccess) return cuda_fail(c, e, "inlet launch");
    c->cur_f = 1 - c->cur_f;
    c->cur_h = 1 - c->cur_h;
    return LBM_OK;
}

// A graph of two plain steps for the current buffers and parameters
// (captured on first use, cached in two slots), or nullptr when none can be
// had (the stream is being captured by the caller, or capture failed).  Two
// steps bring the A/B buffers back to the same roles, so the graph replays
// as long as the signature matches; the step counter is not part of it (the
// stochastic rounding of 16-bit storage reads the time level from a device
// counter that the graph advances).
static lbm_ctx::StepGraph* step_graph(lbm_ctx* c) {
    lbm_ctx::StepGraph key;
    key.b = buffers(c);
    key.p = c->dp;
    key.p.step = 0;
    for (auto& gr : c->graphs)
        if (gr.exec && std::memcmp(&gr.b, &key.b, sizeof key.b) == 0 && std::memcmp(&gr.p, &key.p, sizeof key.p) == 0)
            return &gr;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return nullptr;
    }
    const int cf = c->cur_f, ch = c->cur_h;
    const uint32_t step = c->dp.step;
    const std::string err = c->err;
    cudaGraph_t graph = nullptr;
    lbm_status st = LBM_OK;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = step_once(c, true);
        if (st == LBM_OK) st = step_once(c, true);
        e = cudaStreamEndCapture(c->stream, &graph);
    }
    // the captured launches did not run: undo their bookkeeping
    c->cur_f = cf;
    c->cur_h = ch;
    c->dp.step = step;
    c->err = err;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && st == LBM_OK && graph) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || st != LBM_OK || !exec) {
        cudaGetLastError();
        c->graph_broken = true;
        return nullptr;
    }
    lbm_ctx::StepGraph& slot = c->graphs[c->graph_next];
    c->graph_next ^= 1;
    if (slot.exec) cudaGraphExecDestroy(slot.exec);
    slot = key;
    slot.exec = exec;
    return &slot;
}

lbm_status lbm_step(lbm_ctx* c, int n) {
    if (!c) return LBM_ERR_INVALID;
    if (n < 0) return fail(c, LBM_ERR_INVALID, "n must be >= 0");
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "initialise the fields first");
    DeviceGuard g(c->device);
    // launch-bound stretches replay graphs of two steps (LBM_STEP_AUTO)
    const bool graphs = c->p.step_kernel == LBM_STEP_AUTO && !c->graph_broken && n >= 4;
    if (graphs) {
        bool counter_set = false;
        while (n >= 2) {
            lbm_ctx::StepGraph* gr = step_graph(c);
            if (!gr) break;
            if (c->d_stepctr && !counter_set) {  // the graph's steps continue from dp.step
                k_step_counter<<<1, 1, 0, c->stream>>>(c->d_stepctr, c->dp.step, 0);
                CK(cudaGetLastError(), "step counter launch");
                counter_set = true;
            }
            CK(cudaGraphLaunch(gr->exec, c->stream), "step graph launch");
            c->dp.step += 2;
            n -= 2;
        }
    }
    for (int i = 0; i < n; ++i) {
        const lbm_status st = step_once(c);
        if (st != LBM_OK) return st;
    }
    return LBM_OK;
}

lbm_status lbm_macros(lbm_ctx* c, double* rho, double* u, double* T, int is_device) {
    if (!c) return LBM_ERR_INVALID;
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "initialise the fields first");
    if (!rho || !u || !T) return fail(c, LBM_ERR_INVALID, "null output");
    DeviceGuard g(c->device);
    const size_t N = (size_t)c->N;
    double *dr = rho, *du = u, *dT = T;
    if (!is_device) {
        lbm_status s = ensure_stage(c);
        if (s != LBM_OK) return s;
        dr = c->d_stage;
        du = c->d_stage + N;
        dT = c->d_stage + 4 * N;
    }
    const Buffers b = buffers(c);
    const DevParams p = c->dp;
    CK(dispatch(c, [&](auto tag) {
           using Tg = decltype(tag);
           return lbmd::launch_macros<typename Tg::S, Tg::Q>(b, p, dr, du, dT, c->stream);
       }),
       "macros launch");
    if (!is_device) {
        CK(cudaMemcpyAsync(rho, dr, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "macros copy");
        CK(cudaMemcpyAsync(u, du, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "macros copy");
        CK(cudaMemcpyAsync(T, dT, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "macros copy");
    }
    CK(cudaStreamSynchronize(c->stream), "macros");
    if (!is_device) {
        for (size_t i = 0; i < N; ++i)
            if (!std::isfinite(rho[i]) || !std::isfinite(T[i]) || !std::isfinite(u[i]) ||
                !std::isfinite(u[N + i]) || !std::isfinite(u[2 * N + i]))
                return fail(c, LBM_ERR_DIVERGED, "non-finite macroscopic value at node " + std::to_string(i));
    }
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx* c, double* f, double* h, int is_device) {
    if (!c) return LBM_ERR_INVALID;
    DeviceGuard g(c->device);
    const size_t N = (size_t)c->N;
    double *df = f, *dh = h;
    double* tmp = nullptr;
    if (!is_device) {
        if (dev_alloc(c, &tmp, (27 + c->qh) * N * sizeof(double)) != cudaSuccess)
            return fail(c, LBM_ERR_NOMEM, "population staging: out of device memory");
        df = f ? tmp : nullptr;
        dh = h ? tmp + 27 * N : nullptr;
    }
    const Buffers b = buffers(c);
    const DevParams p = c->dp;
    cudaError_t e = dispatch(c, [&](auto tag) {
        using Tg = decltype(tag);
        return lbmd::launch_populations<typename Tg::S, Tg::Q>(b, p, df, dh, c->stream);
    });
    if (e == cudaSuccess && !is_device) {
        if (f) e = cudaMemcpyAsync(f, df, 27 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && h) e = cudaMemcpyAsync(h, dh, c->qh * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "populations");
    return LBM_OK;
}

lbm_status lbm_balances(lbm_ctx* c, double* mass, double* energy) {
    if (!c) return LBM_ERR_INVALID;
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "initialise the fields first");
    DeviceGuard g(c->device);
    const Buffers b = buffers(c);
    const DevParams p = c->dp;
    double* out = c->d_scratch + 3 * lbmd::kRedBlocks;
    CK(dispatch(c, [&](auto tag) {
           using Tg = decltype(tag);
           return lbmd::launch_balances<typename Tg::S, Tg::Q>(b, p, c->d_scratch, out, c->stream);
       }),
       "balances launch");
    double r[3];
    CK(cudaMemcpyAsync(r, out, sizeof(r), cudaMemcpyDeviceToHost, c->stream), "balances copy");
    CK(cudaStreamSynchronize(c->stream), "balances");
    if (mass) *mass = r[0] + c->dp.rho0 * (double)c->n_fluid_like;
    if (energy) *energy = r[1] + c->dp.Tref * (double)c->n_fluid_like;
    if (r[2] != 0.0) return fail(c, LBM_ERR_DIVERGED, std::to_string((long long)r[2]) + " nodes hold non-finite populations");
    return LBM_OK;
}

lbm_status lbm_surface_flux(lbm_ctx* c, int wall_id, double* flux) {
    if (!c || !flux) return LBM_ERR_INVALID;
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "initialise the fields first");
    if (wall_id < 0 || wall_id >= c->n_walls) return fail(c, LBM_ERR_INVALID, "wall id out of range");
    DeviceGuard g(c->device);
    const Buffers b = buffers(c);
    const DevParams p = c->dp;
    double* out = c->d_scratch + 3 * lbmd::kRedBlocks;
    CK(dispatch(c, [&](auto tag) {
           using Tg = decltype(tag);
           return lbmd::launch_surface_flux<typename Tg::S, Tg::Q>(b, p, wall_id, c->d_scratch, out, c->stream);
       }),
       "flux launch");
    CK(cudaMemcpyAsync(flux, out, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "flux copy");
    CK(cudaStreamSynchronize(c->stream), "flux");
    return LBM_OK;
}

lbm_status lbm_wall_force(lbm_ctx* c, int wall_id, double* force) {
    if (!c || !force) return LBM_ERR_INVALID;
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "initialise the fields first");
    if (wall_id < 0 || wall_id >= c->n_walls) return fail(c, LBM_ERR_INVALID, "wall id out of range");
    DeviceGuard g(c->device);
    const Buffers b = buffers(c);
    const DevParams p = c->dp;
    double* out = c->d_scratch + 3 * lbmd::kRedBlocks;
    CK(dispatch(c, [&](auto tag) {
           using Tg = decltype(tag);
           return lbmd::launch_wall_force<typename Tg::S, Tg::Q>(b, p, wall_id, c->d_scratch, out, c->stream);
       }),
       "wall force launch");
    CK(cudaMemcpyAsync(force, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "wall force copy");
    CK(cudaStreamSynchronize(c->stream), "wall force");
    return LBM_OK;
}

lbm_status lbm_nusselt(lbm_ctx* c, int wall_id, double length, double area, double dT, double* nu_out) {
    if (!c || !nu_out) return LBM_ERR_INVALID;
    if (!(area > 0.0) || dT == 0.0 || !(length > 0.0)) return fail(c, LBM_ERR_INVALID, "length, area must be > 0, dT != 0");
    double q = 0.0;
    lbm_status s = lbm_surface_flux(c, wall_id, &q);
    if (s != LBM_OK) return s;
    *nu_out = q * length / (c->p.k * area * dT);
    return LBM_OK;
}

struct StateHeader {
    char magic[8];
    uint32_t version;
    int32_t nx, ny, nz, qh, storage;
    uint64_t fbytes, hbytes;
    uint64_t step;  // time level (random stream of the 16-bit stochastic rounding)
};

lbm_status lbm_state_size(lbm_ctx* c, size_t* bytes) {
    if (!c || !bytes) return LBM_ERR_INVALID;
    *bytes = sizeof(StateHeader) + (size_t)(27 + c->qh) * c->N * c->ssize;
    return LBM_OK;
}

lbm_status lbm_save_state(lbm_ctx* c, void* host_buf, size_t* bytes, int is_device) {
    if (!c || !bytes || !host_buf) return LBM_ERR_INVALID;
    DeviceGuard g(c->device);
    size_t need = 0;
    lbm_state_size(c, &need);
    if (*bytes < need) {
        *bytes = need;
        return fail(c, LBM_ERR_INVALID, "state buffer too small");
    }
    StateHeader hd{};
    std::memcpy(hd.magic, "LBMSTATE", 8);
    hd.version = 2;
    hd.step = c->dp.step;
    hd.nx = c->p.nx;
    hd.ny = c->p.ny;
    hd.nz = c->p.nz;
    hd.qh = c->qh;
    hd.storage = c->p.storage;
    hd.fbytes = (uint64_t)27 * c->N * c->ssize;
    hd.hbytes = (uint64_t)c->qh * c->N * c->ssize;
    char* out = (char*)host_buf;
    const cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (is_device) {
        CK(cudaMemcpyAsync(out, &hd, sizeof(hd), cudaMemcpyHostToDevice, c->stream), "state copy");
    } else {
        std::memcpy(out, &hd, sizeof(hd));
    }
    CK(cudaMemcpyAsync(out + sizeof(hd), c->f[c->cur_f], hd.fbytes, kind, c->stream), "state copy");
    CK(cudaMemcpyAsync(out + sizeof(hd) + hd.fbytes, c->h[c->cur_h], hd.hbytes, kind, c->stream), "state copy");
    CK(cudaStreamSynchronize(c->stream), "state copy");
    *bytes = need;
    return LBM_OK;
}

lbm_status lbm_load_state(lbm_ctx* c, const void* host_buf, size_t bytes, int is_device) {
    if (!c || !host_buf) return LBM_ERR_INVALID;
    DeviceGuard g(c->device);
    if (!c->geometry) return fail(c, LBM_ERR_STATE, "set the geometry first");
    StateHeader hd{};
    if (bytes < sizeof(hd)) return fail(c, LBM_ERR_INVALID, "state buffer too small");
    if (is_device) {
        CK(cudaMemcpy(&hd, host_buf, sizeof(hd), cudaMemcpyDeviceToHost), "state header");
    } else {
        std::memcpy(&hd, host_buf, sizeof(hd));
    }
    if (std::memcmp(hd.magic, "LBMSTATE", 8) != 0 || hd.version != 2 || hd.nx != c->p.nx || hd.ny != c->p.ny ||
        hd.nz != c->p.nz || hd.qh != c->qh || hd.storage != c->p.storage ||
        hd.fbytes != (uint64_t)27 * c->N * c->ssize || hd.hbytes != (uint64_t)c->qh * c->N * c->ssize ||
        bytes < sizeof(hd) + hd.fbytes + hd.hbytes)
        return fail(c, LBM_ERR_INVALID, "state does not match this context");
    const char* in = (const char*)host_buf;
    const cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(c->f[c->cur_f], in + sizeof(hd), hd.fbytes, kind, c->stream), "state load");
    CK(cudaMemcpyAsync(c->h[c->cur_h], in + sizeof(hd) + hd.fbytes, hd.hbytes, kind, c->stream), "state load");
    CK(cudaStreamSynchronize(c->stream), "state load");
    c->dp.step = (uint32_t)hd.step;
    c->initialised = true;
    return LBM_OK;
}

lbm_status lbm_stream_map(lbm_ctx* c, int32_t* src, int is_device) {
    if (!c || !src) return LBM_ERR_INVALID;
    if (!c->geometry) return fail(c, LBM_ERR_STATE, "set the geometry first");
    DeviceGuard g(c->device);
    const size_t count = (size_t)27 * c->N;
    int32_t* d = src;
    if (!is_device && dev_alloc(c, &d, count * sizeof(int32_t)) != cudaSuccess)
        return fail(c, LBM_ERR_NOMEM, "stream map staging: out of device memory");
    const Buffers b = buffers(c);
    cudaError_t e = lbmd::launch_stream_map(b, c->dp, c->qh, d, c->stream);
    if (e == cudaSuccess && !is_device) e = cudaMemcpyAsync(src, d, count * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (!is_device) cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream map");
    return LBM_OK;
}

lbm_status lbm_get_links(lbm_ctx* c, int64_t* n_links, int32_t* node, int32_t* dir, float* q, int32_t* wall) {
    if (!c || !n_links) return LBM_ERR_INVALID;
    const int64_t cap = *n_links;
    const int64_t total = (int64_t)c->h_lnode.size();
    const int64_t m = std::min(cap, total);
    for (int64_t i = 0; i < m; ++i) {
        if (node) node[i] = c->h_lnode[i];
        if (dir) dir[i] = c->h_ldir[i];
        if (q) q[i] = c->h_lq[i];
        if (wall) wall[i] = c->h_lwall[i];
    }
    *n_links = total;
    return LBM_OK;
}

static lbmd::AdjObjective to_adj(const lbm_objective* o) {
    lbmd::AdjObjective a{};
    a.kind = o ? o->kind : 0;
    a.wall = o ? o->wall_id : -1;
    a.plane = o ? o->plane_x : -1;
    a.comp = o ? o->component : 0;
    a.weight = o ? o->weight : 0.0;
    if (!o) a.kind = 0, a.wall = -1;
    return a;
}

static lbm_status check_objective(lbm_ctx* c, const lbm_objective* o) {
    if (!o) return LBM_OK;
    if (o->kind == LBM_OBJ_SURFACE_FLUX) {
        if (o->wall_id < 0 || o->wall_id >= c->n_walls) return fail(c, LBM_ERR_INVALID, "objective wall id out of range");
    } else if (o->kind == LBM_OBJ_SECTION_FLUX) {
        if (o->plane_x < 0 || o->plane_x >= c->p.nx) return fail(c, LBM_ERR_INVALID, "objective plane out of range");
    } else if (o->kind == LBM_OBJ_WALL_FORCE) {
        if (o->wall_id < 0 || o->wall_id >= c->n_walls) return fail(c, LBM_ERR_INVALID, "objective wall id out of range");
        if (o->component < 0 || o->component > 2) return fail(c, LBM_ERR_INVALID, "force component must be 0, 1 or 2");
    } else {
        return fail(c, LBM_ERR_INVALID, "unknown objective kind");
    }
    if (!std::isfinite(o->weight)) return fail(c, LBM_ERR_INVALID, "objective weight not finite");
    return LBM_OK;
}

lbm_status lbm_step_record(lbm_ctx* c, int n, void* u_rec, int advance_h) {
    if (!c) return LBM_ERR_INVALID;
    if (n < 0) return fail(c, LBM_ERR_INVALID, "n must be >= 0");
    if (n > 0 && !u_rec) return fail(c, LBM_ERR_INVALID, "null velocity record");
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "initialise the fields first");
    DeviceGuard g(c->device);
    const size_t rsize = c->p.storage == LBM_F64 ? sizeof(double) : sizeof(float);
    for (int i = 0; i < n; ++i) {
        Buffers b = buffers(c);
        c->dp.step += 1;
        const DevParams p = c->dp;
        b.urec = (char*)u_rec + (size_t)i * 3 * c->N * rsize;
        cudaError_t e = fill_mirror(c, b, p);
        if (e != cudaSuccess) return cuda_fail(c, e, "symmetry rows launch");
        e = dispatch(c, [&](auto tag) {
            using Tg = decltype(tag);
            return lbmd::launch_step<typename Tg::S, Tg::Q>(b, p, c->stream, advance_h != 0);
        });
        if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
        if ((e = zou_he_inlet(c, b, p, advance_h != 0)) != cudaSuccess) return cuda_fail(c, e, "inlet launch");
        c->cur_f = 1 - c->cur_f;
        if (advance_h) c->cur_h = 1 - c->cur_h;
    }
    return LBM_OK;
}

lbm_status lbm_step_record_h(lbm_ctx* c, int n, void* u_rec, void* h_rec) {
    if (!c) return LBM_ERR_INVALID;
    if (n < 0) return fail(c, LBM_ERR_INVALID, "n must be >= 0");
    if (n > 0 && (!u_rec || !h_rec)) return fail(c, LBM_ERR_INVALID, "null velocity or h record");
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "initialise the fields first");
    DeviceGuard g(c->device);
    const size_t rsize = c->p.storage == LBM_F64 ? sizeof(double) : sizeof(float);
    for (int i = 0; i < n; ++i) {
        lbm_status st = lbm_step_record(c, 1, (char*)u_rec + (size_t)i * 3 * c->N * rsize, 1);
        if (st != LBM_OK) return st;
        const Buffers b = buffers(c);
        const DevParams p = c->dp;
        void* rec = (char*)h_rec + (size_t)i * c->qh * c->N * rsize;
        cudaError_t e = dispatch(c, [&](auto tag) {
            using Tg = decltype(tag);
            return lbmd::launch_record_h<typename Tg::S, Tg::Q>(b, p, rec, c->stream);
        });
        if (e != cudaSuccess) return cuda_fail(c, e, "h record launch");
    }
    return LBM_OK;
}

static lbm_status adjoint_step_impl(lbm_ctx* c, const void* u_level, const void* h_level, const void* mu_next,
                                    void* out, const lbm_objective* obj, double* dJ_dtheta) {
    if (!c || !mu_next || !out) return LBM_ERR_INVALID;
    if (!c->geometry) return fail(c, LBM_ERR_STATE, "set the geometry first");
    if (c->p.hkind == LBM_H_CUM_1ST && u_level && !h_level)
        return fail(c, LBM_ERR_INVALID,
                    "the Cumulants-1st adjoint needs the level's h record (lbm_step_record_h, lbm_adjoint_step_h)");
    lbm_status st = check_objective(c, obj);
    if (st != LBM_OK) return st;
    if (obj && obj->kind == LBM_OBJ_WALL_FORCE)
        return fail(c, LBM_ERR_INVALID, "a wall-force objective needs the coupled adjoint (lbm_adjoint_flow_step)");
    DeviceGuard g(c->device);
    const Buffers b = buffers(c);
    const DevParams p = c->dp;
    const lbmd::AdjObjective a = to_adj(obj);
    cudaError_t e;
    if (c->p.storage == LBM_F64) {
        using R = double;
        e = c->qh == 27 ? lbmd::launch_adjoint<R, 27>(b, p, (const R*)u_level, (const R*)h_level, (const R*)mu_next,
                                                     (R*)out, a, dJ_dtheta, c->stream)
                        : lbmd::launch_adjoint<R, 7>(b, p, (const R*)u_level, (const R*)h_level, (const R*)mu_next,
                                                    (R*)out, a, dJ_dtheta, c->stream);
    } else {
        using R = float;
        e = c->qh == 27 ? lbmd::launch_adjoint<R, 27>(b, p, (const R*)u_level, (const R*)h_level, (const R*)mu_next,
                                                     (R*)out, a, dJ_dtheta, c->stream)
                        : lbmd::launch_adjoint<R, 7>(b, p, (const R*)u_level, (const R*)h_level, (const R*)mu_next,
                                                    (R*)out, a, dJ_dtheta, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint launch");
    return LBM_OK;
}

lbm_status lbm_adjoint_step(lbm_ctx* c, const void* u_level, const void* mu_next, void* out,
                            const lbm_objective* obj, double* dJ_dtheta) {
    return adjoint_step_impl(c, u_level, nullptr, mu_next, out, obj, dJ_dtheta);
}

// elements of one level's f record of the coupled adjoint: ten moments per
// node, then the Zou-He inlet nodes' full arrivals
static int64_t flow_frec_elems(const lbm_ctx* c) {
    return (int64_t)10 * c->N + (c->dp.zou_he ? (int64_t)27 * c->p.ny * c->p.nz : 0);
}

lbm_status lbm_flow_record_size(lbm_ctx* c, int64_t* f_elems, int64_t* h_elems) {
    if (!c || !f_elems || !h_elems) return LBM_ERR_INVALID;
    *f_elems = flow_frec_elems(c);
    *h_elems = (int64_t)c->qh * c->N;
    return LBM_OK;
}

lbm_status lbm_step_record_pre(lbm_ctx* c, int n, void* f_rec, void* h_rec) {
    if (!c) return LBM_ERR_INVALID;
    if (n < 0) return fail(c, LBM_ERR_INVALID, "n must be >= 0");
    if (n > 0 && (!f_rec || !h_rec)) return fail(c, LBM_ERR_INVALID, "null f or h record");
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "initialise the fields first");
    if (c->p.storage != LBM_F32 && c->p.storage != LBM_F64)
        return fail(c, LBM_ERR_INVALID, "pre-collision records need FP32 or FP64 storage");
    DeviceGuard g(c->device);
    const size_t rsize = c->ssize;
    for (int i = 0; i < n; ++i) {
        Buffers b = buffers(c);
        c->dp.step += 1;
        const DevParams p = c->dp;
        b.frec = (char*)f_rec + (size_t)i * flow_frec_elems(c) * rsize;
        b.hrec = (char*)h_rec + (size_t)i * c->qh * c->N * rsize;
        cudaError_t e = fill_mirror(c, b, p);
        if (e != cudaSuccess) return cuda_fail(c, e, "symmetry rows launch");
        e = dispatch(c, [&](auto tag) {
            using Tg = decltype(tag);
            return lbmd::launch_step<typename Tg::S, Tg::Q>(b, p, c->stream, true);
        });
        if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
        if ((e = zou_he_inlet(c, b, p, true)) != cudaSuccess) return cuda_fail(c, e, "inlet launch");
        c->cur_f = 1 - c->cur_f;
        c->cur_h = 1 - c->cur_h;
    }
    return LBM_OK;
}

lbm_status lbm_adjoint_flow_step(lbm_ctx* c, const void* f_level, const void* h_level, const void* muf_next,
                                 const void* muh_next, void* muf_out, void* muh_out, const lbm_objective* obj,
                                 double* dJ_dtheta) {
    if (!c || !muf_next || !muh_next || !muf_out || !muh_out) return LBM_ERR_INVALID;
    if (!c->geometry) return fail(c, LBM_ERR_STATE, "set the geometry first");
    if (c->p.storage != LBM_F32 && c->p.storage != LBM_F64)
        return fail(c, LBM_ERR_INVALID, "the coupled adjoint needs FP32 or FP64 storage");
    if ((f_level == nullptr) != (h_level == nullptr))
        return fail(c, LBM_ERR_INVALID, "give both level records or neither (initial level)");
    lbm_status st = check_objective(c, obj);
    if (st != LBM_OK) return st;
    DeviceGuard g(c->device);
    const size_t rsize = c->ssize;
    if (!c->d_flowacc) {
        if (dev_alloc(c, &c->d_flowacc, (size_t)c->N * 6 * sizeof(double)) != cudaSuccess)
            return fail(c, LBM_ERR_NOMEM, "coupled adjoint accumulators: out of device memory");
        CK(cudaMemsetAsync(c->d_flowacc, 0, (size_t)c->N * 6 * sizeof(double), c->stream), "accumulators");
    }
    if (!c->d_din && dev_alloc(c, &c->d_din, (size_t)3 * (27 + c->qh) * rsize) != cudaSuccess)
        return fail(c, LBM_ERR_NOMEM, "inlet derivative table: out of device memory");
    if (!c->d_wflow && dev_alloc(c, &c->d_wflow, (size_t)3 * c->N * rsize) != cudaSuccess)
        return fail(c, LBM_ERR_NOMEM, "coupled adjoint velocity derivative: out of device memory");
    std::vector<double> din = inlet_derivative(c);
    if (din != c->h_din) {
        CK(cudaStreamSynchronize(c->stream), "inlet derivative table");
        if (c->p.storage == LBM_F64) {
            CK(cudaMemcpy(c->d_din, din.data(), din.size() * sizeof(double), cudaMemcpyHostToDevice),
               "inlet derivative table");
        } else {
            std::vector<float> df(din.begin(), din.end());
            CK(cudaMemcpy(c->d_din, df.data(), df.size() * sizeof(float), cudaMemcpyHostToDevice),
               "inlet derivative table");
        }
        c->h_din = din;
    }
    const Buffers b = buffers(c);
    const DevParams p = c->dp;
    const lbmd::AdjObjective a = to_adj(obj);
    cudaError_t e;
    if (c->p.storage == LBM_F64) {
        using R = double;
        e = c->qh == 27 ? lbmd::launch_adjoint_flow<R, 27>(b, p, (const R*)f_level, (const R*)h_level,
                                                          (const R*)muf_next, (const R*)muh_next, (R*)muf_out,
                                                          (R*)muh_out, a, dJ_dtheta, c->d_flowacc,
                                                          (const R*)c->d_din, (R*)c->d_wflow, c->stream)
                        : lbmd::launch_adjoint_flow<R, 7>(b, p, (const R*)f_level, (const R*)h_level,
                                                         (const R*)muf_next, (const R*)muh_next, (R*)muf_out,
                                                         (R*)muh_out, a, dJ_dtheta, c->d_flowacc,
                                                         (const R*)c->d_din, (R*)c->d_wflow, c->stream);
    } else {
        using R = float;
        e = c->qh == 27 ? lbmd::launch_adjoint_flow<R, 27>(b, p, (const R*)f_level, (const R*)h_level,
                                                          (const R*)muf_next, (const R*)muh_next, (R*)muf_out,
                                                          (R*)muh_out, a, dJ_dtheta, c->d_flowacc,
                                                          (const R*)c->d_din, (R*)c->d_wflow, c->stream)
                        : lbmd::launch_adjoint_flow<R, 7>(b, p, (const R*)f_level, (const R*)h_level,
                                                         (const R*)muf_next, (const R*)muh_next, (R*)muf_out,
                                                         (R*)muh_out, a, dJ_dtheta, c->d_flowacc,
                                                         (const R*)c->d_din, (R*)c->d_wflow, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "coupled adjoint launch");
    return LBM_OK;
}

lbm_status lbm_adjoint_flow_gradient(lbm_ctx* c, double* dJ_dF, double* dJ_duin, int reset) {
    if (!c || !dJ_dF || !dJ_duin) return LBM_ERR_INVALID;
    DeviceGuard g(c->device);
    for (int d = 0; d < 3; ++d) dJ_dF[d] = dJ_duin[d] = 0.0;
    if (!c->d_flowacc) return LBM_OK;
    CK(lbmd::launch_reduce6(c->d_flowacc, c->N, c->d_scratch, c->stream), "flow gradient reduction");
    double out[6];
    CK(cudaMemcpyAsync(out, c->d_scratch, sizeof(out), cudaMemcpyDeviceToHost, c->stream), "flow gradient copy");
    if (reset)
        CK(cudaMemsetAsync(c->d_flowacc, 0, (size_t)c->N * 6 * sizeof(double), c->stream), "flow gradient reset");
    CK(cudaStreamSynchronize(c->stream), "flow gradient");
    for (int d = 0; d < 3; ++d) {
        dJ_dF[d] = out[d];
        dJ_duin[d] = out[3 + d];
    }
    return LBM_OK;
}

lbm_status lbm_adjoint_step_h(lbm_ctx* c, const void* u_level, const void* h_level, const void* mu_next, void* out,
                              const lbm_objective* obj, double* dJ_dtheta) {
    return adjoint_step_impl(c, u_level, h_level, mu_next, out, obj, dJ_dtheta);
}

lbm_status lbm_adjoint_wall_gradient(lbm_ctx* c, double* dJ_dTwall, int reset) {
    if (!c || !dJ_dTwall) return LBM_ERR_INVALID;
    DeviceGuard g(c->device);
    for (int w = 0; w < c->n_walls; ++w) dJ_dTwall[w] = 0.0;
    if (c->nl == 0) return LBM_OK;
    std::vector<double> acc((size_t)c->nl);
    CK(cudaMemcpyAsync(acc.data(), c->d_dlink, c->nl * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
       "link gradient copy");
    if (reset) CK(cudaMemsetAsync(c->d_dlink, 0, c->nl * sizeof(double), c->stream), "link gradient reset");
    CK(cudaStreamSynchronize(c->stream), "link gradient");
    for (int64_t l = 0; l < c->nl; ++l) dJ_dTwall[c->h_lwall[l]] += acc[l];
    return LBM_OK;
}

lbm_status lbm_objective_accumulate(lbm_ctx* c, const lbm_objective* obj, double* J_device) {
    if (!c || !obj || !J_device) return LBM_ERR_INVALID;
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "initialise the fields first");
    lbm_status st = check_objective(c, obj);
    if (st != LBM_OK) return st;
    DeviceGuard g(c->device);
    const Buffers b = buffers(c);
    const DevParams p = c->dp;
    const lbmd::AdjObjective a = to_adj(obj);
    CK(dispatch(c, [&](auto tag) {
           using Tg = decltype(tag);
           return lbmd::launch_objective<typename Tg::S, Tg::Q>(b, p, a, c->d_scratch, J_device, c->stream);
       }),
       "objective launch");
    return LBM_OK;
}

lbm_status lbm_section_flux(lbm_ctx* c, int plane_x, double* flux) {
    if (!c || !flux) return LBM_ERR_INVALID;
    lbm_objective o{LBM_OBJ_SECTION_FLUX, 0, plane_x, 0, 1.0};
    double* acc = c->d_scratch + 3 * lbmd::kRedBlocks + 3;
    DeviceGuard g(c->device);
    CK(cudaMemsetAsync(acc, 0, sizeof(double), c->stream), "section flux");
    lbm_status st = lbm_objective_accumulate(c, &o, acc);
    if (st != LBM_OK) return st;
    CK(cudaMemcpyAsync(flux, acc, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "section flux copy");
    CK(cudaStreamSynchronize(c->stream), "section flux");
    return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* c) {
    if (!c) return LBM_ERR_INVALID;
    DeviceGuard g(c->device);
    CK(cudaStreamSynchronize(c->stream), "sync");
    CK(cudaGetLastError(), "sync");
    return LBM_OK;
}

const char* lbm_last_error(lbm_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

}  // extern "C"
