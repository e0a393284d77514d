// Device-side lattice tables and collision operators of the thermal LBM
// (arXiv 2203.01316).  Everything here runs in registers of one thread per
// node.
//
// Storage is "deviation" form: a stored f value is f - w*rho0 and a stored h
// value is h - w*T_ref (h being the App. D shifted variable).  The collision
// works on the central moments of these deviations,
//     dk_mno = kappa_mno(f) - rho0 * K_mno(v),
// where K_mno(v) = K_m(v_x) K_n(v_y) K_o(v_z) are the central moments of the
// weights about the shift v: K_0 = 1, K_1(v) = -v, K_2(v) = cs^2 + v^2.
// All quantities handled are then small, so FP32 (and FP16/BF16 storage)
// keep their relative precision.
//
// The central-moment transform T(v) of Appendix C factorises over the three
// axes (T = T1(v_x) x T1(v_y) x T1(v_z) on the 27-moment set of Sec. 2.1), so
// it is applied as 3 passes of nine 3-point transforms; the inverse likewise.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

namespace lbmd {

// ---- D3Q27 velocity list of Sec. 2.1 ------------------------------------
__host__ __device__ __forceinline__ constexpr int EX(int a) {
    constexpr int t[27] = {0, 1, 0, 0, 1, 1, 0, -1, 0, 0, 1, 1, -1, -1, 0, 0, 1, -1, -1, 0, -1, 1, 1, 1, -1, -1, -1};
    return t[a];
}
__host__ __device__ __forceinline__ constexpr int EY(int a) {
    constexpr int t[27] = {0, 0, 1, 0, 1, 0, 1, 0, -1, 0, -1, 0, 1, 0, 1, -1, 1, -1, 0, -1, 1, -1, 1, -1, 1, -1, -1};
    return t[a];
}
__host__ __device__ __forceinline__ constexpr int EZ(int a) {
    constexpr int t[27] = {0, 0, 0, 1, 0, 1, 1, 0, 0, -1, 0, -1, 0, 1, -1, 1, 1, 0, -1, -1, 1, 1, -1, -1, -1, 1, -1};
    return t[a];
}
// direction with velocity (x, y, z)
__host__ __device__ __forceinline__ constexpr int DIR(int x, int y, int z) {
    int r = -1;
    for (int a = 0; a < 27; ++a)
        if (EX(a) == x && EY(a) == y && EZ(a) == z) r = a;
    return r;
}
__host__ __device__ __forceinline__ constexpr int OPP(int a) { return DIR(-EX(a), -EY(a), -EZ(a)); }
// slot of direction a in the 3x3x3 cube used by the transforms: (ez+1)*9 + (ey+1)*3 + (ex+1)
__host__ __device__ __forceinline__ constexpr int CUBE(int a) { return (EZ(a) + 1) * 9 + (EY(a) + 1) * 3 + (EX(a) + 1); }
// D3Q27 weights: product of the 1-D weights (2/3 at rest, 1/6 moving)
__host__ __device__ __forceinline__ constexpr double W1(int e) { return e == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ __forceinline__ constexpr double W27(int a) { return W1(EX(a)) * W1(EY(a)) * W1(EZ(a)); }

// ---- D3Q7 (velocities {0,+x,+y,+z,-x,-y,-z} = D3Q27 indices 0,1,2,3,7,8,9)
__host__ __device__ __forceinline__ constexpr int D7(int i) {
    constexpr int t[7] = {0, 1, 2, 3, 7, 8, 9};
    return t[i];
}
__host__ __device__ __forceinline__ constexpr int OPP7(int i) { return i == 0 ? 0 : (i <= 3 ? i + 3 : i - 3); }
__host__ __device__ __forceinline__ constexpr double W7(int i) { return i == 0 ? 0.0 : 1.0 / 6.0; }

// h lattice helpers: velocity index in the D3Q27 list, opposite, weight
template <int QH> __host__ __device__ __forceinline__ constexpr int HDIR(int i) { return QH == 27 ? i : D7(i); }
template <int QH> __host__ __device__ __forceinline__ constexpr int HOPP(int i) { return QH == 27 ? OPP(i) : OPP7(i); }
// velocity with the y component reversed (D3Q27 index; D3Q7: +y <-> -y)
__host__ __device__ __forceinline__ constexpr int FLIPY(int a) { return DIR(EX(a), -EY(a), EZ(a)); }
template <int QH> __host__ __device__ __forceinline__ constexpr int HFLIPY(int i) {
    return QH == 27 ? FLIPY(i) : (i == 2 ? 5 : (i == 5 ? 2 : i));
}
template <int QH> __host__ __device__ __forceinline__ constexpr double HW(int i) { return QH == 27 ? W27(i) : W7(i); }

// ---- storage types -------------------------------------------------------
template <typename S> struct Acc { using R = float; };
template <> struct Acc<double> { using R = double; };

template <typename R> __device__ __forceinline__ R ld(const float* p) { return (R)__ldg(p); }
template <typename R> __device__ __forceinline__ R ld(const double* p) { return (R)__ldg(p); }
template <typename R> __device__ __forceinline__ R ld(const __half* p) { return (R)__half2float(__ldg(p)); }
template <typename R> __device__ __forceinline__ R ld(const __nv_bfloat16* p) { return (R)__bfloat162float(__ldg(p)); }

__device__ __forceinline__ void st(float* p, float v) { *p = v; }
__device__ __forceinline__ void st(double* p, double v) { *p = v; }
__device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// Random bits of the stochastic rounding of one node's 16-bit stores: a
// strong hash of (node, array, time level) starts a Weyl sequence (the
// golden-ratio increment 0x9E3779B9) that advances once per pair of stores.
// Each draw is uniform because its start is; reproducible, one add per draw.
struct SrStream {
    uint32_t s;
    __device__ __forceinline__ uint32_t next() {
        const uint32_t r = s;
        s += 0x9E3779B9u;
        return r;
    }
};

// counter-based 32-bit hash (the "lowbias32" integer mixer of C. Wellons) of
// (node and array, time level): the start of a node's SrStream
__device__ __forceinline__ uint32_t sr_bits(uint32_t key, uint32_t step) {
    uint32_t x = key ^ (step * 0x9E3779B9u);
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// ---- moment algebra --------------------------------------------------------
// lattice constants are formed in double and converted once, so that they
// stay compile-time constants for every arithmetic type (1/3 rounds to the
// same float either way)
template <typename R> __device__ __forceinline__ constexpr R cs2() { return R(1.0 / 3.0); }

// forward-mode dual number v + d eps: runs the collision functions (templated
// on the arithmetic type) to give directional derivatives for the coupled
// adjoint
template <typename T> struct Dual {
    T v, d;
    __host__ __device__ constexpr Dual() : v(0), d(0) {}
    __host__ __device__ constexpr Dual(double x) : v((T)x), d(0) {}
    __host__ __device__ constexpr Dual(T x, T dx, int) : v(x), d(dx) {}
    friend __host__ __device__ constexpr Dual operator+(const Dual& a, const Dual& b) {
        return Dual(a.v + b.v, a.d + b.d, 0);
    }
    friend __host__ __device__ constexpr Dual operator-(const Dual& a, const Dual& b) {
        return Dual(a.v - b.v, a.d - b.d, 0);
    }
    friend __host__ __device__ constexpr Dual operator*(const Dual& a, const Dual& b) {
        return Dual(a.v * b.v, a.d * b.v + a.v * b.d, 0);
    }
    friend __host__ __device__ constexpr Dual operator/(const Dual& a, const Dual& b) {
        return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v), 0);
    }
    friend __host__ __device__ constexpr Dual operator-(const Dual& a) { return Dual(-a.v, -a.d, 0); }
    __host__ __device__ constexpr Dual& operator+=(const Dual& b) { return *this = *this + b; }
    __host__ __device__ constexpr Dual& operator-=(const Dual& b) { return *this = *this - b; }
    __host__ __device__ constexpr Dual& operator*=(const Dual& b) { return *this = *this * b; }
    __host__ __device__ constexpr Dual& operator/=(const Dual& b) { return *this = *this / b; }
};

// scalar type underlying an arithmetic type (constants are formed in it)
template <typename T> struct ScalarOf { using type = T; };
template <typename T> struct ScalarOf<Dual<T>> { using type = T; };

// a parameter in arithmetic type R: the float copy for FP32-based types
template <typename R> __device__ __forceinline__ R par(double d, float f) {
    if constexpr (sizeof(typename ScalarOf<R>::type) == 4) return R(f);
    else return R(d);
}

// slot of moment mno in the cube after the forward passes
__host__ __device__ __forceinline__ constexpr int MIDX(int m, int n, int o) { return o * 9 + n * 3 + m; }

// equilibrium central moments for psi = 1 (Sec. 2.1.1): 1 at 000, cs^2 per
// index 2, zero when any index is 1; formed in the scalar type underlying R
// (float or double) so that it stays a constant for every arithmetic type
template <typename R> __device__ __forceinline__ R Eq(int m, int n, int o) {
    using T = typename ScalarOf<R>::type;
    if (m == 1 || n == 1 || o == 1) return R(0);
    T v = T(1);
    if (m == 2) v *= cs2<T>();
    if (n == 2) v *= cs2<T>();
    if (o == 2) v *= cs2<T>();
    return R(v);
}

template <typename R> __device__ __forceinline__ R Kd(int m, R v) {
    return m == 0 ? R(1) : (m == 1 ? -v : cs2<R>() + v * v);
}

// D_mno(v) = E_mno - K_mno(v), expanded so the result keeps its relative
// precision (it is O(v)).
template <typename R>
__device__ __forceinline__ R Dm(int m, int n, int o, R vx, R vy, R vz, R tx, R ty, R tz) {
    if (m == 1 || n == 1 || o == 1) return -(Kd<R>(m, vx) * Kd<R>(n, vy) * Kd<R>(o, vz));
    const R c = cs2<R>();
    const R a = (m == 2) ? tx : R(0);
    const R b = (n == 2) ? ty : R(0);
    const R d = (o == 2) ? tz : R(0);
    const int cnt = (m == 2) + (n == 2) + (o == 2);
    if (cnt == 0) return R(0);
    if (cnt == 1) return -(a + b + d);
    if (cnt == 2) {
        // two of a, b, d are non-zero: cs^2 (p + q) + p q
        const R p = (m == 2) ? a : b;
        const R q = (o == 2) ? d : b;
        return -(c * (p + q) + p * q);
    }
    return -(c * c * (a + b + d) + c * (a * b + a * d + b * d) + a * b * d);
}

// forward 3-point central transform with shift v: (g-, g0, g+) -> (k0, k1, k2)
template <typename R> __device__ __forceinline__ void fwd3(R& a, R& b, R& c, R v) {
    const R m0 = a + b + c;
    const R m1 = c - a;
    const R m2 = c + a;
    const R k1 = m1 - v * m0;
    const R k2 = m2 - v * (m1 + k1);
    a = m0;
    b = k1;
    c = k2;
}
// inverse: (k0, k1, k2) -> (g-, g0, g+)
template <typename R> __device__ __forceinline__ void inv3(R& a, R& b, R& c, R v) {
    const R m0 = a;
    const R m1 = b + v * m0;
    const R m2 = c + v * (b + m1);
    a = R(0.5) * (m2 - m1);
    b = m0 - m2;
    c = R(0.5) * (m2 + m1);
}

template <typename R> __device__ __forceinline__ void forward_cube(R* c, R vx, R vy, R vz) {
#pragma unroll
    for (int j = 0; j < 9; ++j) fwd3<R>(c[3 * j], c[3 * j + 1], c[3 * j + 2], vx);
#pragma unroll
    for (int z = 0; z < 3; ++z)
#pragma unroll
        for (int x = 0; x < 3; ++x) fwd3<R>(c[9 * z + x], c[9 * z + 3 + x], c[9 * z + 6 + x], vy);
#pragma unroll
    for (int j = 0; j < 9; ++j) fwd3<R>(c[j], c[9 + j], c[18 + j], vz);
}

template <typename R> __device__ __forceinline__ void inverse_cube(R* c, R vx, R vy, R vz) {
#pragma unroll
    for (int j = 0; j < 9; ++j) inv3<R>(c[j], c[9 + j], c[18 + j], vz);
#pragma unroll
    for (int z = 0; z < 3; ++z)
#pragma unroll
        for (int x = 0; x < 3; ++x) inv3<R>(c[9 * z + x], c[9 * z + 3 + x], c[9 * z + 6 + x], vy);
#pragma unroll
    for (int j = 0; j < 9; ++j) inv3<R>(c[3 * j], c[3 * j + 1], c[3 * j + 2], vx);
}

// The same inverse in six operations per three-point group instead of
// eight.  With k2 entering halved, g+ = k2/2 + (v + 1/2) k1 + v(v + 1)/2 k0,
// g- = k2/2 + (v - 1/2) k1 + v(v - 1)/2 k0 and g0 = k0 - g+ - g- (the raw
// moments g+ + g- = k2 + 2 v k1 + v^2 k0 and g+ - g- = k1 + v k0 of the
// shifted transform).  The caller fills the cube with every moment scaled by
// 2^-(number of its indices equal to 2): each pass is linear and leaves the
// other indices alone, so every later pass also receives its index-2 slots
// halved.
template <typename R> struct InvAxis {
    R p1, p0, m1, m0;
};
template <typename R> __device__ __forceinline__ InvAxis<R> inv_axis(R v) {
    const R hv = R(0.5) * v;
    return {v + R(0.5), hv * v + hv, v - R(0.5), hv * v - hv};
}
template <typename R> __device__ __forceinline__ void inv3h(R& a, R& b, R& c, const InvAxis<R>& k) {
    const R gp = c + k.p1 * b + k.p0 * a;
    const R gm = c + k.m1 * b + k.m0 * a;
    b = a - gp - gm;
    a = gm;
    c = gp;
}
template <typename R> __device__ __forceinline__ void inverse_cube_h(R* c, R vx, R vy, R vz) {
    const InvAxis<R> kx = inv_axis(vx), ky = inv_axis(vy), kz = inv_axis(vz);
#pragma unroll
    for (int j = 0; j < 9; ++j) inv3h<R>(c[j], c[9 + j], c[18 + j], kz);
#pragma unroll
    for (int z = 0; z < 3; ++z)
#pragma unroll
        for (int x = 0; x < 3; ++x) inv3h<R>(c[9 * z + x], c[9 * z + 3 + x], c[9 * z + 6 + x], ky);
#pragma unroll
    for (int j = 0; j < 9; ++j) inv3h<R>(c[3 * j], c[3 * j + 1], c[3 * j + 2], kx);
}

// E and D scaled by 2^-(indices equal to 2), for inverse_cube_h.  Every
// index-2 factor of E and of K is c_s^2 + v^2 (E: v = 0), so the scaled forms
// are E and D with c_s^2 and v^2 both halved: hx = vx^2 / 2 etc.
template <typename R> __device__ __forceinline__ constexpr R cs2h() { return R(1.0 / 6.0); }
template <typename R> __device__ __forceinline__ R Eqh(int m, int n, int o) {
    using T = typename ScalarOf<R>::type;
    if (m == 1 || n == 1 || o == 1) return R(0);
    T v = T(1);
    if (m == 2) v *= cs2h<T>();
    if (n == 2) v *= cs2h<T>();
    if (o == 2) v *= cs2h<T>();
    return R(v);
}
template <typename R> __device__ __forceinline__ R Kdh(int m, R v, R h) {
    return m == 0 ? R(1) : (m == 1 ? -v : cs2h<R>() + h);
}
template <typename R>
__device__ __forceinline__ R Dmh(int m, int n, int o, R vx, R vy, R vz, R hx, R hy, R hz) {
    if (m == 1 || n == 1 || o == 1) return -(Kdh<R>(m, vx, hx) * Kdh<R>(n, vy, hy) * Kdh<R>(o, vz, hz));
    const R c = cs2h<R>();
    const R a = (m == 2) ? hx : R(0);
    const R b = (n == 2) ? hy : R(0);
    const R d = (o == 2) ? hz : R(0);
    const int cnt = (m == 2) + (n == 2) + (o == 2);
    if (cnt == 0) return R(0);
    if (cnt == 1) return -(a + b + d);
    if (cnt == 2) {
        const R p = (m == 2) ? a : b;
        const R q = (o == 2) ? d : b;
        return -(c * (p + q) + p * q);
    }
    return -(c * c * (a + b + d) + c * (a * b + a * d + b * d) + a * b * d);
}
// 2^-(indices equal to 2) for slot mno
__host__ __device__ __forceinline__ constexpr double HALVES(int m, int n, int o) {
    return (m == 2 ? 0.5 : 1.0) * (n == 2 ? 0.5 : 1.0) * (o == 2 ? 0.5 : 1.0);
}

// ---- parameters -------------------------------------------------------------
struct DevParams {
    int nx, ny, nz, N, periodic_x;
    int stochastic;      // 16-bit storage: 1 stochastic rounding, 0 round to nearest
    int hkind;           // 0..2 central-moment kinds, 3 Cumulants-1st
    int wall_bc;         // 0 Eq. IBB + Eq. IABB, 1 BB + EQ, 2 BB + ABB (BB/ABB: q = 1/2 on the device)
    int mirror_lo, mirror_hi;  // rows y = 0 / y = ny-1 are symmetry rows
    int zou_he;                // inlet plane: 0 fixed equilibria, 1 Zou-He (k_inlet after the step)
    int nwall;                 // wall nodes (entries of the wall table)
    // n / nx and r / ny for 0 <= n, r < 2^31 as umulhi(n, m) >> s (the
    // round-up method for 31-bit dividends: m = ceil(2^(31+l) / d),
    // l = ceil(log2 d) >= 1, s = l - 1); m = 0 for a divisor of 1
    uint32_t mx, my;
    int sx, sy;
    uint32_t step;       // time level being written (seeds the stochastic rounding)
    // in replayed CUDA graphs the time level is read from this device counter,
    // which the graph advances before each step (nullptr: use step)
    const uint32_t* step_ctr;
    double omega1, omega_bulk;  // f: shear and bulk rates
    double sh[7];               // h: rate of central moments of each order 0..6
    double rho0, Tref;
    double F[3];
    double uin[3], Tin;
    // the same parameters rounded to float once on the host (sync_float_params):
    // FP32 arithmetic reads these, so no kernel converts a double per use
    struct {
        float omega1, omega_bulk, sh[7], rho0, Tref, F[3], uin[3], Tin;
    } pf;
};

// refresh DevParams::pf after changing a double parameter (host)
inline void sync_float_params(DevParams& d) {
    d.pf.omega1 = (float)d.omega1;
    d.pf.omega_bulk = (float)d.omega_bulk;
    for (int i = 0; i < 7; ++i) d.pf.sh[i] = (float)d.sh[i];
    d.pf.rho0 = (float)d.rho0;
    d.pf.Tref = (float)d.Tref;
    for (int i = 0; i < 3; ++i) {
        d.pf.F[i] = (float)d.F[i];
        d.pf.uin[i] = (float)d.uin[i];
    }
    d.pf.Tin = (float)d.Tin;
}

// ---- raw moments of order <= 2 of 27 populations -------------------------
// Sums along x, then y, then z over the 3x3x3 cube, keeping only what the
// ten moments need (66 additions instead of the 171 of summing each
// population into each moment)
template <typename R>
__device__ __forceinline__ void raw_moments_f(const R* fd, R& m000, R& m100, R& m010, R& m001, R& m200, R& m020,
                                              R& m002, R& m110, R& m101, R& m011) {
    R X0[9], X1[9], X2[9];  // x moments 0, 1, 2 of the line (y, z) = (j % 3 - 1, j / 3 - 1)
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const int ey = j % 3 - 1, ez = j / 3 - 1;
        const R a = fd[DIR(-1, ey, ez)], b = fd[DIR(0, ey, ez)], c = fd[DIR(1, ey, ez)];
        X2[j] = a + c;
        X1[j] = c - a;
        X0[j] = X2[j] + b;
    }
    R Y00[3], Y01[3], Y02[3], Y10[3], Y11[3], Y20[3];  // [z]: x moment, y moment
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int j = 3 * k;
        Y02[k] = X0[j] + X0[j + 2];
        Y01[k] = X0[j + 2] - X0[j];
        Y00[k] = Y02[k] + X0[j + 1];
        Y11[k] = X1[j + 2] - X1[j];
        Y10[k] = X1[j] + X1[j + 1] + X1[j + 2];
        Y20[k] = X2[j] + X2[j + 1] + X2[j + 2];
    }
    m002 = Y00[0] + Y00[2];
    m001 = Y00[2] - Y00[0];
    m000 = m002 + Y00[1];
    m010 = Y01[0] + Y01[1] + Y01[2];
    m011 = Y01[2] - Y01[0];
    m020 = Y02[0] + Y02[1] + Y02[2];
    m100 = Y10[0] + Y10[1] + Y10[2];
    m101 = Y10[2] - Y10[0];
    m110 = Y11[0] + Y11[1] + Y11[2];
    m200 = Y20[0] + Y20[1] + Y20[2];
}

// ---- f: cumulant collision (Eq. hydro_cu_collision) ----------------------
// fd: pulled deviations in, post-collision deviations out.  Second-order
// cumulants relax with omega1 (off-diagonal, deviators) and omega_bulk
// (trace); cumulants of order >= 3 go to zero (rate 1), so the post-collision
// central moments about the new mean mu* = mu + F/rho are those of a
// distribution whose cumulants stop at order two (Isserlis' products).
// Returns u = mu + F/(2 rho) (velocity that shifts h) and rho.
// collide_f with the body force as an argument (the coupled adjoint passes a
// dual-number F to differentiate with respect to it)
template <typename R>
__device__ __forceinline__ void collide_f_force(R* fd, const DevParams& p, const R Fx, const R Fy, const R Fz, R& ux,
                                                R& uy, R& uz, R& rho_out) {
    R drho, jx, jy, jz, mxx, myy, mzz, mxy, mxz, myz;
    raw_moments_f<R>(fd, drho, jx, jy, jz, mxx, myy, mzz, mxy, mxz, myz);
    const R c = cs2<R>();
    const R rho0 = par<R>(p.rho0, p.pf.rho0);
    const R rho = rho0 + drho;
    const R irho = R(1) / rho;
    const R mux = jx * irho, muy = jy * irho, muz = jz * irho;
    // second central moments about mu, minus rho cs^2 on the diagonal
    R axx = mxx - drho * c - jx * mux;
    R ayy = myy - drho * c - jy * muy;
    R azz = mzz - drho * c - jz * muz;
    R kxy = mxy - jx * muy;
    R kxz = mxz - jx * muz;
    R kyz = myz - jy * muz;
    const R om1 = R(1) - par<R>(p.omega1, p.pf.omega1);
    const R omb = R(1) - par<R>(p.omega_bulk, p.pf.omega_bulk);
    R dxy = (axx - ayy) * om1;
    R dxz = (axx - azz) * om1;
    R tr = (axx + ayy + azz) * omb;
    kxy *= om1;
    kxz *= om1;
    kyz *= om1;
    const R sxx = (tr + dxy + dxz) * (R(1) / R(3));
    const R syy = sxx - dxy;
    const R szz = sxx - dxz;
    // shifts: mean after collision, velocity for h
    const R vx = mux + Fx * irho, vy = muy + Fy * irho, vz = muz + Fz * irho;
    ux = mux + R(0.5) * Fx * irho;
    uy = muy + R(0.5) * Fy * irho;
    uz = muz + R(0.5) * Fz * irho;
    rho_out = rho;
    // halved squares and halved second-order moments: the cube is filled
    // scaled by 2^-(indices equal to 2) for inverse_cube_h
    const R hx = R(0.5) * vx * vx, hy = R(0.5) * vy * vy, hz = R(0.5) * vz * vz;
    const R ch = cs2h<R>();
    const R sxh = R(0.5) * sxx, syh = R(0.5) * syy, szh = R(0.5) * szz;

    // non-equilibrium part of the post-collision central moments
    // (kappa* - rho E), zero for odd orders, each scaled like its slot:
    // kappa_220 = c(sxx + syy) + (sxx syy + 2 kxy^2)/rho etc., the Isserlis
    // products of the relaxed second-order cumulants
    const R n220 = ch * (sxh + syh) + (sxh * syh + R(0.5) * kxy * kxy) * irho;
    const R n202 = ch * (sxh + szh) + (sxh * szh + R(0.5) * kxz * kxz) * irho;
    const R n022 = ch * (syh + szh) + (syh * szh + R(0.5) * kyz * kyz) * irho;
    const R n211 = ch * kyz + (sxh * kyz + kxy * kxz) * irho;
    const R n121 = ch * kxz + (syh * kxz + kxy * kyz) * irho;
    const R n112 = ch * kxy + (szh * kxy + kxz * kyz) * irho;
    const R n222 = ch * ch * (sxh + syh + szh) +
                   (ch * (sxh * syh + sxh * szh + syh * szh) + R(0.5) * ch * (kxy * kxy + kxz * kxz + kyz * kyz)) * irho +
                   (sxh * syh * szh + R(0.5) * (sxh * kyz * kyz + syh * kxz * kxz + szh * kxy * kxy) +
                    kxy * kxz * kyz) * irho * irho;

    R cb[27];
#pragma unroll
    for (int o = 0; o < 3; ++o)
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                R neq = R(0);
                if (m == 1 && n == 1 && o == 0) neq = kxy;
                if (m == 1 && n == 0 && o == 1) neq = kxz;
                if (m == 0 && n == 1 && o == 1) neq = kyz;
                if (m == 2 && n == 0 && o == 0) neq = sxh;
                if (m == 0 && n == 2 && o == 0) neq = syh;
                if (m == 0 && n == 0 && o == 2) neq = szh;
                if (m == 2 && n == 2 && o == 0) neq = n220;
                if (m == 2 && n == 0 && o == 2) neq = n202;
                if (m == 0 && n == 2 && o == 2) neq = n022;
                if (m == 2 && n == 1 && o == 1) neq = n211;
                if (m == 1 && n == 2 && o == 1) neq = n121;
                if (m == 1 && n == 1 && o == 2) neq = n112;
                if (m == 2 && n == 2 && o == 2) neq = n222;
                cb[MIDX(m, n, o)] = neq + drho * Eqh<R>(m, n, o) + rho0 * Dmh<R>(m, n, o, vx, vy, vz, hx, hy, hz);
            }
    inverse_cube_h<R>(cb, vx, vy, vz);
#pragma unroll
    for (int a = 0; a < 27; ++a) fd[a] = cb[CUBE(a)];
}

template <typename R>
__device__ __forceinline__ void collide_f(R* fd, const DevParams& p, R& ux, R& uy, R& uz, R& rho_out) {
    collide_f_force<R>(fd, p, par<R>(p.F[0], p.pf.F[0]), par<R>(p.F[1], p.pf.F[1]), par<R>(p.F[2], p.pf.F[2]), ux, uy, uz, rho_out);
}

// ---- h: central-moment collision (Eq. H_cm_collision + App. D source) ----
// Y* = Y + s (H E - Y) + (1 - s/2) Q E per moment, s = p.sh[order]; with
// Y = dY + Tref K:  dY* = (1-s) dY + s (dH E + Tref D) + (1 - s/2) Q E,
// dH = H - Tref, H = sum(h) + Q/2.
// TRT (compile time): the CM-TRT kind, whose even orders relax with rate 1,
// so they go straight to equilibrium plus half the source and their
// pre-collision values are never needed (the odd orders, whose equilibrium
// part E vanishes, keep s^H)
// m0 (if given) receives the pre-collision zeroth moment sum(h)
template <typename R, bool TRT = false>
__device__ __forceinline__ void collide_h27(R* hd, R ux, R uy, R uz, R Q, const DevParams& p, R* m0 = nullptr) {
    R cb[27];
#pragma unroll
    for (int a = 0; a < 27; ++a) cb[CUBE(a)] = hd[a];
    forward_cube<R>(cb, ux, uy, uz);
    if (m0) *m0 = cb[0];
    const R Tref = par<R>(p.Tref, p.pf.Tref);
    const R dH = cb[0] + R(0.5) * Q;
    // relaxed moments scaled by 2^-(indices equal to 2) for inverse_cube_h:
    // E and D come scaled (Eqh, Dmh), the pre-collision moment y is scaled
    // through its coefficient
    const R hx = R(0.5) * ux * ux, hy = R(0.5) * uy * uy, hz = R(0.5) * uz * uz;
#pragma unroll
    for (int o = 0; o < 3; ++o)
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const R E = Eqh<R>(m, n, o);
                const R D = Dmh<R>(m, n, o, ux, uy, uz, hx, hy, hz);
                const R sc = R(HALVES(m, n, o));
                R& y = cb[MIDX(m, n, o)];
                if constexpr (TRT) {
                    if ((m + n + o) % 2 == 0) {
                        y = dH * E + Tref * D + R(0.5) * Q * E;
                    } else {
                        const R s = par<R>(p.sh[1], p.pf.sh[1]);
                        y = ((R(1) - s) * sc) * y + s * (Tref * D);
                    }
                } else {
                    const R s = par<R>(p.sh[m + n + o], p.pf.sh[m + n + o]);
                    y = ((R(1) - s) * sc) * y + s * (dH * E + Tref * D) + (R(1) - R(0.5) * s) * Q * E;
                }
            }
    inverse_cube_h<R>(cb, ux, uy, uz);
#pragma unroll
    for (int a = 0; a < 27; ++a) hd[a] = cb[CUBE(a)];
}

// D3Q7 (pops 0, +x, +y, +z, -x, -y, -z; moments 000, 100, 010, 001, 200, 020, 002)
template <typename R, bool TRT = false>
__device__ __forceinline__ void collide_h7(R* hd, R ux, R uy, R uz, R Q, const DevParams& p, R* m0_out = nullptr) {
    const R u[3] = {ux, uy, uz};
    const R m0 = hd[0] + hd[1] + hd[2] + hd[3] + hd[4] + hd[5] + hd[6];
    if (m0_out) *m0_out = m0;
    const R Tref = par<R>(p.Tref, p.pf.Tref);
    const R dH = m0 + R(0.5) * Q;
    const R c = cs2<R>();
    const R s1 = par<R>(p.sh[1], p.pf.sh[1]);
    R y0, y1[3], y2[3];
    if constexpr (TRT) {  // orders 0 and 2 relax with rate 1
        y0 = dH + R(0.5) * Q;
    } else {
        const R s0 = par<R>(p.sh[0], p.pf.sh[0]);
        y0 = (R(1) - s0) * m0 + s0 * dH + (R(1) - R(0.5) * s0) * Q;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const R m1 = hd[1 + d] - hd[4 + d];
        const R k1 = m1 - u[d] * m0;
        // D_1 = u, D_2 = -u^2; E_1 = 0, E_2 = cs^2
        y1[d] = (R(1) - s1) * k1 + s1 * (Tref * u[d]);
        if constexpr (TRT) {
            y2[d] = dH * c - Tref * u[d] * u[d] + R(0.5) * Q * c;
        } else {
            const R s2 = par<R>(p.sh[2], p.pf.sh[2]);
            const R m2 = hd[1 + d] + hd[4 + d];
            const R k2 = m2 - u[d] * (m1 + k1);
            y2[d] = (R(1) - s2) * k2 + s2 * (dH * c - Tref * u[d] * u[d]) + (R(1) - R(0.5) * s2) * Q * c;
        }
    }
    R rest = y0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const R M1 = y1[d] + u[d] * y0;
        const R M2 = y2[d] + u[d] * (y1[d] + M1);
        hd[1 + d] = R(0.5) * (M2 + M1);
        hd[4 + d] = R(0.5) * (M2 - M1);
        rest -= M2;
    }
    hd[0] = rest;
}

template <typename R, int QH>
__device__ __forceinline__ void heq_dev(R* hd, R dpsi, R ux, R uy, R uz, const DevParams& p);

// ---- h: Cumulants-1st (Eq. H_cu_collision + App. D source) -----------------
// With every cumulant of order >= 2 set to its equilibrium (c_s^2 on the
// diagonal of the second order, zero elsewhere), the post-collision cumulants
// (H + Q/2, v, c_s^2 I, 0, ...) are those of the discrete Maxwellian at the
// relaxed mean velocity v = (1 - s) m + s u, m = sum(e h)/sum(h): the result
// is that equilibrium.  The zeroth moment sum(h) must be positive.
template <typename R, int QH>
__device__ __forceinline__ void collide_h_cum(R* hd, R ux, R uy, R uz, R Q, const DevParams& p, R* m0 = nullptr) {
    R dH = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < QH; ++i) {
        const int a = HDIR<QH>(i);
        const R v = hd[i];
        dH += v;
        if (EX(a) != 0) jx += EX(a) * v;
        if (EY(a) != 0) jy += EY(a) * v;
        if (EZ(a) != 0) jz += EZ(a) * v;
    }
    if (m0) *m0 = dH;
    const R Ht = par<R>(p.Tref, p.pf.Tref) + dH;  // zeroth moment of the stored (App. D shifted) h
    const R iH = R(1) / Ht;
    const R s = par<R>(p.sh[1], p.pf.sh[1]);
    // v = u + (1 - s)(m - u): exactly u at s = 1
    const R vx = ux + (R(1) - s) * (jx * iH - ux);
    const R vy = uy + (R(1) - s) * (jy * iH - uy);
    const R vz = uz + (R(1) - s) * (jz * iH - uz);
    heq_dev<R, QH>(hd, dH + Q, vx, vy, vz, p);
}

// CUM: the Cumulants-1st kind (compile time, so the central-moment kinds
// keep their register allocation)
template <typename R, int QH, bool CUM = false, bool TRT = false>
__device__ __forceinline__ void collide_h(R* hd, R ux, R uy, R uz, R Q, const DevParams& p, R* m0 = nullptr) {
    if constexpr (CUM) {
        collide_h_cum<R, QH>(hd, ux, uy, uz, Q, p, m0);
    } else if constexpr (QH == 27) {
        collide_h27<R, TRT>(hd, ux, uy, uz, Q, p, m0);
    } else {
        collide_h7<R, TRT>(hd, ux, uy, uz, Q, p, m0);
    }
}

// ---- equilibria in deviation form ------------------------------------------
// f^eq(rho0 + drho, u) - w rho0: central moments about u are drho E + rho0 D(u)
// (the density enters as its deviation, like heq_dev's zeroth moment)
template <typename R>
__device__ __forceinline__ void feq_dev(R* fd, R drho, R ux, R uy, R uz, const DevParams& p) {
    const R rho0 = par<R>(p.rho0, p.pf.rho0);
    const R tx = ux * ux, ty = uy * uy, tz = uz * uz;
    R cb[27];
#pragma unroll
    for (int o = 0; o < 3; ++o)
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
            for (int m = 0; m < 3; ++m)
                cb[MIDX(m, n, o)] = drho * Eq<R>(m, n, o) + rho0 * Dm<R>(m, n, o, ux, uy, uz, tx, ty, tz);
    inverse_cube<R>(cb, ux, uy, uz);
#pragma unroll
    for (int a = 0; a < 27; ++a) fd[a] = cb[CUBE(a)];
}

// h^eq(Tref + dpsi, u) - w Tref on the h lattice; the zeroth moment enters as
// its deviation dpsi, so no Tref is added and subtracted again in FP32
template <typename R, int QH>
__device__ __forceinline__ void heq_dev(R* hd, R dpsi, R ux, R uy, R uz, const DevParams& p) {
    const R Tref = par<R>(p.Tref, p.pf.Tref);
    if constexpr (QH == 27) {
        const R tx = ux * ux, ty = uy * uy, tz = uz * uz;
        R cb[27];
#pragma unroll
        for (int o = 0; o < 3; ++o)
#pragma unroll
            for (int n = 0; n < 3; ++n)
#pragma unroll
                for (int m = 0; m < 3; ++m)
                    cb[MIDX(m, n, o)] = dpsi * Eq<R>(m, n, o) + Tref * Dm<R>(m, n, o, ux, uy, uz, tx, ty, tz);
        inverse_cube<R>(cb, ux, uy, uz);
#pragma unroll
        for (int a = 0; a < 27; ++a) hd[a] = cb[CUBE(a)];
    } else {
        const R u[3] = {ux, uy, uz};
        R rest = dpsi;
        const R c = cs2<R>();
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const R y1 = Tref * u[d];
            const R y2 = dpsi * c - Tref * u[d] * u[d];
            const R M1 = y1 + u[d] * dpsi;
            const R M2 = y2 + u[d] * (y1 + M1);
            hd[1 + d] = R(0.5) * (M2 + M1);
            hd[4 + d] = R(0.5) * (M2 - M1);
            rest -= M2;
        }
        hd[0] = rest;
    }
}

}  // namespace lbmd
