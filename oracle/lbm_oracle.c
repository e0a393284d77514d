/*
 * FP64 CPU oracle of the coupled f+h thermal lattice Boltzmann step of
 * Gruszczynski & Laniewski-Wollk, "A comparative study of 3D Cumulant and
 * Central Moments lattice Boltzmann schemes with interpolated boundary
 * conditions ..." (arXiv 2203.01316).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test suite, the
 * package smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, table or header with the CUDA library.
 *
 * Everything is done the literal way:
 *   - the D3Q27 velocity list is typed from Sec. 2.1 (Lattice Boltzmann
 *     Method), the 27 moment indices in the order given there;
 *   - the raw-moment matrix M and the central-moment matrix T(u) are built
 *     row by row from Eqs. (M) and (T) of Appendix C, and T(u) is applied by
 *     an explicit 27x27 product; its inverse is applied by solving T x = y
 *     with Gaussian elimination (T = N M, so T^-1 = M^-1 N^-1);
 *   - equilibria are T(u)^-1 applied to the central-moment equilibrium
 *     vector of Sec. 2.1.1 (Appendix A route);
 *   - cumulants are the coefficients of the logarithm of the normalised
 *     central-moment generating function, evaluated in the polynomial ring
 *     truncated to degree <= 2 per axis (closed on the 27 indices, so exact);
 *   - the f collision is Eq. (hydro_cu_collision), the h collision
 *     Eq. (H_cm_collision) with the CM-SRT / CM-1st / CM-TRT rate sets of
 *     Sec. 2.1.1, or Eq. (H_cu_collision) with the Cumulants-1st rates, the
 *     source term per Appendix D;
 *   - streaming is the push form of the evolution equation of Sec. 2.1,
 *     followed by Eq. (IBB) and Eq. (IABB) on every wall link.
 *
 * Readings of points the paper leaves open (each is listed in the design
 * notes of the repository):
 *   R1 f relaxation (the paper defers to Geier 2015): off-diagonal second
 *      cumulants and the deviators c200-c020, c200-c002 relax with
 *      omega1 = 1/(3 nu + 1/2); the trace with omega_bulk (default 1) toward
 *      3 cs^2; cumulants of order 3, 4, 5, 6 relax with omega3..omega6
 *      (default 1) toward 0.
 *   R2 body force: the first-order cumulant (the mean velocity) gains F/rho
 *      in collision; u = (sum e f + F/2)/rho is the velocity that shifts h.
 *   R3 source for the CM kinds: source moments Q*E (equilibrium-shaped),
 *      added as (1 - S/2) Q E; h stores the App. D shifted variable, so
 *      H = sum h + Q/2.
 *   R4 IABB wall equilibrium: u_w = 0, so h^eq_i(x_w) = w_i T_w.
 *   R5 thin gap (x_f = x_b - e_a is solid or outside the domain): the q > 1/2
 *      branch evaluated at q = 1/2 (plain BB / ABB).
 *   R6 inlet plane x = 0: post-collision populations are the equilibria at
 *      (rho = 1, u_in) and (T_in, u_in); outlet plane x = nx-1: an incoming
 *      population with e_x < 0 is the post-collision value at
 *      (nx-1, y-e_y, z-e_z) (zero normal gradient of the post-collision
 *      field).  y and z are always periodic.
 *   R7 D3Q7 = velocities {0,+x,+y,+z,-x,-y,-z} (indices 0,1,2,3,7,8,9 of the
 *      D3Q27 list), moments {000,100,010,001,200,020,002}, cs^2 = 1/3.
 *   R8 surface heat flux of one wall: sum over its IABB links of
 *      h_abar(x_b, t+1) - h*_a(x_b, t).
 *   R15 symmetry planes (Sec. 4.4): specular reflection (e_y reversed) at the
 *      plane halfway between a symmetry row and its neighbour row.
 *   R19 Cumulants-1st with the App. D source: order 0 -> H + Q, order 1
 *      relaxed to u with s^H, second-order diagonal cs^2, all else 0.
 *   R20 Zou-He inlet (Sec. 4.4): non-equilibrium bounce-back for f at u_in,
 *      the unknown h in the equilibrium shape with sum h = rho T_in.
 *   R21 force on a wall (not in the paper): momentum exchange over the links
 *      of Eq. IBB.
 *   R23 first-order walls (Sec. 3): BB = Eq. IBB at q = 1/2, ABB = Eq. IABB
 *      at q = 1/2, EQ: the population arriving from the wall is the wall
 *      equilibrium w_i T_w.
 *
 * Parity unpinned: none of the functions below lacks a pin; the cumulant
 * relaxation beyond second order is pinned only through R1's default rates.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CS2 (1.0 / 3.0)

/* ---- lattice: Sec. 2.1, velocity list e = [e_x, e_y, e_z] ---- */
static const int EX[27] = {0, 1, 0, 0, 1, 1, 0, -1, 0, 0, 1, 1, -1, -1, 0, 0, 1, -1, -1, 0, -1, 1, 1, 1, -1, -1, -1};
static const int EY[27] = {0, 0, 1, 0, 1, 0, 1, 0, -1, 0, -1, 0, 1, 0, 1, -1, 1, -1, 0, -1, 1, -1, 1, -1, 1, -1, -1};
static const int EZ[27] = {0, 0, 0, 1, 0, 1, 1, 0, 0, -1, 0, -1, 0, 1, -1, 1, 1, 0, -1, -1, 1, 1, -1, -1, -1, 1, -1};

/* moment indices mno in the order of Sec. 2.1 */
static const int MOM27[27][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1},
    {2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 2, 0}, {1, 0, 2}, {2, 1, 0}, {2, 0, 1},
    {0, 1, 2}, {0, 2, 1}, {1, 1, 1}, {2, 2, 0}, {2, 0, 2}, {0, 2, 2}, {2, 1, 1},
    {1, 2, 1}, {1, 1, 2}, {1, 2, 2}, {2, 1, 2}, {2, 2, 1}, {2, 2, 2}};

/* reading R7 */
static const int D3Q7_DIRS[7] = {0, 1, 2, 3, 7, 8, 9};
static const int MOM7[7][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2}};

typedef struct {
    int Q;
    int e[27][3];
    int mom[27][3];
    int dir27[27]; /* index of each velocity in the D3Q27 list */
    int opp[27];
    double w[27];  /* equilibrium at H = 1, u = 0 */
} lattice_t;

static double ipow(double b, int p) {
    double r = 1.0;
    for (int i = 0; i < p; ++i) r *= b;
    return r;
}

/* Eq. (M): M_mno|a = e_ax^m e_ay^n e_az^o */
static void build_M(const lattice_t* L, double* M) {
    for (int r = 0; r < L->Q; ++r)
        for (int a = 0; a < L->Q; ++a)
            M[r * L->Q + a] = ipow(L->e[a][0], L->mom[r][0]) * ipow(L->e[a][1], L->mom[r][1]) *
                              ipow(L->e[a][2], L->mom[r][2]);
}

/* Eq. (T): T_mno|a = (e_ax-ux)^m (e_ay-uy)^n (e_az-uz)^o */
static void build_T(const lattice_t* L, const double u[3], double* T) {
    for (int r = 0; r < L->Q; ++r)
        for (int a = 0; a < L->Q; ++a)
            T[r * L->Q + a] = ipow(L->e[a][0] - u[0], L->mom[r][0]) *
                              ipow(L->e[a][1] - u[1], L->mom[r][1]) *
                              ipow(L->e[a][2] - u[2], L->mom[r][2]);
}

static void matvec(int n, const double* A, const double* x, double* y) {
    for (int r = 0; r < n; ++r) {
        double s = 0.0;
        for (int c = 0; c < n; ++c) s += A[r * n + c] * x[c];
        y[r] = s;
    }
}

/* Solve A x = b by Gaussian elimination with partial pivoting.  Returns 0, or
 * -1 if A is singular. */
static int solve(int n, const double* A, const double* b, double* x) {
    double a[27 * 28];
    for (int r = 0; r < n; ++r) {
        for (int c = 0; c < n; ++c) a[r * (n + 1) + c] = A[r * n + c];
        a[r * (n + 1) + n] = b[r];
    }
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int r = k + 1; r < n; ++r)
            if (fabs(a[r * (n + 1) + k]) > fabs(a[piv * (n + 1) + k])) piv = r;
        if (a[piv * (n + 1) + k] == 0.0) return -1;
        if (piv != k)
            for (int c = 0; c <= n; ++c) {
                double t = a[k * (n + 1) + c];
                a[k * (n + 1) + c] = a[piv * (n + 1) + c];
                a[piv * (n + 1) + c] = t;
            }
        for (int r = k + 1; r < n; ++r) {
            double f = a[r * (n + 1) + k] / a[k * (n + 1) + k];
            for (int c = k; c <= n; ++c) a[r * (n + 1) + c] -= f * a[k * (n + 1) + c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = a[r * (n + 1) + n];
        for (int c = r + 1; c < n; ++c) s -= a[r * (n + 1) + c] * x[c];
        x[r] = s / a[r * (n + 1) + r];
    }
    return 0;
}

/* central-moment equilibrium vector of Sec. 2.1.1 for psi = 1: non-zero at
 * 000 (1), 200/020/002 (cs^2), 220/202/022 (cs^4), 222 (cs^6) */
static double eq_central(const int m[3]) {
    double v = 1.0;
    for (int d = 0; d < 3; ++d) {
        if (m[d] == 1) return 0.0;
        if (m[d] == 2) v *= CS2;
    }
    return v;
}

/* g^eq = M^-1 N^-1 Y^eq = T(u)^-1 Y^eq (Appendix A) */
static void equilibrium(const lattice_t* L, double psi, const double u[3], double* g) {
    double T[27 * 27], y[27];
    build_T(L, u, T);
    for (int r = 0; r < L->Q; ++r) y[r] = psi * eq_central(L->mom[r]);
    solve(L->Q, T, y, g);
}

static void lattice_init(lattice_t* L, int Q) {
    L->Q = Q;
    for (int a = 0; a < Q; ++a) {
        int d = (Q == 27) ? a : D3Q7_DIRS[a];
        L->dir27[a] = d;
        L->e[a][0] = EX[d];
        L->e[a][1] = EY[d];
        L->e[a][2] = EZ[d];
        for (int k = 0; k < 3; ++k) L->mom[a][k] = (Q == 27) ? MOM27[a][k] : MOM7[a][k];
    }
    for (int a = 0; a < Q; ++a) {
        L->opp[a] = -1;
        for (int b = 0; b < Q; ++b)
            if (L->e[b][0] == -L->e[a][0] && L->e[b][1] == -L->e[a][1] && L->e[b][2] == -L->e[a][2])
                L->opp[a] = b;
    }
    const double u0[3] = {0.0, 0.0, 0.0};
    equilibrium(L, 1.0, u0, L->w);
}

static lattice_t LAT27, LAT7;
static int lattices_ready = 0;
static void ensure_lattices(void) {
    if (!lattices_ready) {
        lattice_init(&LAT27, 27);
        lattice_init(&LAT7, 7);
        lattices_ready = 1;
    }
}
static const lattice_t* lattice(int Q) {
    ensure_lattices();
    return Q == 7 ? &LAT7 : &LAT27;
}

/* ---- cumulants: truncated polynomial ring, coefficient [i][j][k] at
 * index 9 i + 3 j + k, s_x^3 = s_y^3 = s_z^3 = 0 ---- */
static void poly_mul(const double* a, const double* b, double* r) {
    for (int n = 0; n < 27; ++n) r[n] = 0.0;
    for (int i1 = 0; i1 < 3; ++i1)
        for (int j1 = 0; j1 < 3; ++j1)
            for (int k1 = 0; k1 < 3; ++k1) {
                double av = a[9 * i1 + 3 * j1 + k1];
                if (av == 0.0) continue;
                for (int i2 = 0; i1 + i2 < 3; ++i2)
                    for (int j2 = 0; j1 + j2 < 3; ++j2)
                        for (int k2 = 0; k1 + k2 < 3; ++k2)
                            r[9 * (i1 + i2) + 3 * (j1 + j2) + (k1 + k2)] += av * b[9 * i2 + 3 * j2 + k2];
            }
}

static const double FACT[3] = {1.0, 1.0, 2.0};

/* ln(P) for P with P[0] = 1: ln(1+x) = sum_n (-1)^(n+1) x^n / n, x^7 = 0 */
static void poly_log(const double* P, double* Lg) {
    double x[27], xn[27], t[27];
    for (int n = 0; n < 27; ++n) x[n] = P[n];
    x[0] -= 1.0;
    for (int n = 0; n < 27; ++n) { xn[n] = x[n]; Lg[n] = 0.0; }
    for (int p = 1; p <= 6; ++p) {
        double c = ((p % 2) ? 1.0 : -1.0) / (double)p;
        for (int n = 0; n < 27; ++n) Lg[n] += c * xn[n];
        poly_mul(xn, x, t);
        for (int n = 0; n < 27; ++n) xn[n] = t[n];
    }
}

/* exp(Lg) for Lg[0] = 0: sum_n Lg^n / n!, Lg^7 = 0 */
static void poly_exp(const double* Lg, double* P) {
    double xn[27], t[27];
    double fact = 1.0;
    for (int n = 0; n < 27; ++n) { P[n] = 0.0; xn[n] = 0.0; }
    xn[0] = 1.0;
    for (int p = 0; p <= 6; ++p) {
        if (p > 0) fact *= (double)p;
        for (int n = 0; n < 27; ++n) P[n] += xn[n] / fact;
        poly_mul(xn, Lg, t);
        for (int n = 0; n < 27; ++n) xn[n] = t[n];
    }
}

/* Cumulant transform (Sec. 2.1, following Geier 2015): C[000] = rho,
 * C[100], C[010], C[001] = the mean velocity (first-order cumulants), and
 * for order >= 2 the cumulants of the normalised distribution, computed as
 * i! j! k! [s^ijk] ln( sum kappa_ijk / rho s^ijk / (i! j! k!) ) from the
 * central moments kappa about the mean. */
static void cumulants(const double* g, double* C) {
    const lattice_t* L = lattice(27);
    double rho = 0.0, mean[3] = {0, 0, 0};
    for (int a = 0; a < 27; ++a) {
        rho += g[a];
        for (int d = 0; d < 3; ++d) mean[d] += L->e[a][d] * g[a];
    }
    for (int d = 0; d < 3; ++d) mean[d] /= rho;
    double T[27 * 27], kap[27], P[27], Lg[27];
    build_T(L, mean, T);
    matvec(27, T, g, kap);
    for (int r = 0; r < 27; ++r) {
        const int* m = L->mom[r];
        P[9 * m[0] + 3 * m[1] + m[2]] = kap[r] / rho / (FACT[m[0]] * FACT[m[1]] * FACT[m[2]]);
    }
    poly_log(P, Lg);
    for (int r = 0; r < 27; ++r) {
        const int* m = L->mom[r];
        C[r] = FACT[m[0]] * FACT[m[1]] * FACT[m[2]] * Lg[9 * m[0] + 3 * m[1] + m[2]];
    }
    C[0] = rho;
    C[1] = mean[0];
    C[2] = mean[1];
    C[3] = mean[2];
}

/* inverse of cumulants(): exponentiate, scale by rho, and solve T(mean). */
static void cumulants_inverse(const double* C, double* g) {
    const lattice_t* L = lattice(27);
    double rho = C[0], mean[3] = {C[1], C[2], C[3]};
    double Lg[27], P[27], kap[27], T[27 * 27];
    for (int r = 0; r < 27; ++r) {
        const int* m = L->mom[r];
        int order = m[0] + m[1] + m[2];
        Lg[9 * m[0] + 3 * m[1] + m[2]] =
            (order >= 2) ? C[r] / (FACT[m[0]] * FACT[m[1]] * FACT[m[2]]) : 0.0;
    }
    poly_exp(Lg, P);
    for (int r = 0; r < 27; ++r) {
        const int* m = L->mom[r];
        kap[r] = rho * FACT[m[0]] * FACT[m[1]] * FACT[m[2]] * P[9 * m[0] + 3 * m[1] + m[2]];
    }
    build_T(L, mean, T);
    solve(27, T, kap, g);
}

/* ---- parameters ---- */
typedef struct {
    int nx, ny, nz;
    int qh;          /* 27 or 7 */
    int hkind;       /* 0 CM-TRT, 1 CM-SRT, 2 CM-1st */
    int periodic_x;  /* 1: periodic in x; 0: inlet plane x=0, outlet x=nx-1 */
    double nu, k;
    double omega_bulk, omega3, omega4, omega5, omega6;
    double F[3];
    double u_in[3], T_in;
    int wall_bc;     /* 0 Eq. IBB + Eq. IABB; 1 BB + EQ (first order); 2 BB + ABB */
    int inlet_bc;    /* 0 equilibrium inlet plane (reading R6); 1 Zou-He (reading R20) */
} orc_params;

enum { KIND_TRT = 0, KIND_SRT = 1, KIND_1ST = 2, KIND_CUM1 = 3 };

/* Eq. (hydro_cu_collision) with reading R1 (rates) and R2 (force).  Writes
 * the post-collision populations and the velocity u that shifts h. */
static void collide_f(const orc_params* p, const double* f, double* fs, double* u) {
    double C[27], Cs[27];
    cumulants(f, C);
    const double rho = C[0];
    const double w1 = 1.0 / (3.0 * p->nu + 0.5);
    const double wb = p->omega_bulk;
    for (int r = 0; r < 27; ++r) Cs[r] = C[r];
    for (int d = 0; d < 3; ++d) {
        Cs[1 + d] = C[1 + d] + p->F[d] / rho;
        u[d] = C[1 + d] + 0.5 * p->F[d] / rho;
    }
    /* second order: off-diagonal 110 (4), 101 (5), 011 (6) */
    for (int r = 4; r <= 6; ++r) Cs[r] = C[r] + w1 * (0.0 - C[r]);
    /* diagonal 200 (7), 020 (8), 002 (9): deviators with omega1, trace with
     * omega_bulk toward 3 cs^2 */
    double dxy = C[7] - C[8], dxz = C[7] - C[9], tr = C[7] + C[8] + C[9];
    dxy = dxy + w1 * (0.0 - dxy);
    dxz = dxz + w1 * (0.0 - dxz);
    tr = tr + wb * (3.0 * CS2 - tr);
    Cs[7] = (tr + dxy + dxz) / 3.0;
    Cs[8] = Cs[7] - dxy;
    Cs[9] = Cs[7] - dxz;
    const double wn[7] = {0, 0, 0, p->omega3, p->omega4, p->omega5, p->omega6};
    const lattice_t* L = lattice(27);
    for (int r = 10; r < 27; ++r) {
        int order = L->mom[r][0] + L->mom[r][1] + L->mom[r][2];
        Cs[r] = C[r] + wn[order] * (0.0 - C[r]);
    }
    cumulants_inverse(Cs, fs);
}

/* relaxation rate of moment r for the CM kinds of Sec. 2.1.1 */
static double rate_h(int kind, int order, double sH) {
    switch (kind) {
        case KIND_SRT: return sH;
        case KIND_1ST: return (order == 1) ? sH : 1.0;
        default: return (order % 2 == 1) ? sH : 1.0; /* CM-TRT */
    }
}

/* Eq. (H_cu_collision) with Appendix D's source, Cumulants-1st rates
 * (Sec. 2.1.1): first-order cumulants relax with s^H toward u, every higher
 * order is set to its equilibrium (c_s^2 on the diagonal of the second order,
 * zero otherwise), C^Q = [Q, 0, ...].  The cumulants are those of the stored
 * (shifted) h, normalised by its zeroth moment, which must be positive. */
static void collide_h_cumulant(const orc_params* p, const double* h, const double u[3], double Q, double* hs) {
    const double sH = 1.0 / (p->k / CS2 + 0.5);
    if (p->qh == 27) {
        const lattice_t* L = lattice(27);
        double C[27], Cs[27];
        cumulants(h, C);
        const double H = C[0] + 0.5 * Q;
        for (int r = 0; r < 27; ++r) {
            const int* m = L->mom[r];
            const int order = m[0] + m[1] + m[2];
            double eq, s;
            if (order == 0) { eq = H; s = 1.0; }
            else if (order == 1) { eq = u[m[1] ? 1 : (m[2] ? 2 : 0)]; s = sH; }
            else { eq = (order == 2 && (m[0] == 2 || m[1] == 2 || m[2] == 2)) ? CS2 : 0.0; s = 1.0; }
            Cs[r] = C[r] + s * (eq - C[r]) + ((r == 0) ? (1.0 - 0.5 * s) * Q : 0.0);
        }
        cumulants_inverse(Cs, hs);
        return;
    }
    /* D3Q7 (reading R7): the seven moments carry the mean and the per-axis
     * variance; the post-collision distribution has mean v and variance cs^2 */
    const lattice_t* L = lattice(7);
    double Ht = 0.0, mean[3] = {0, 0, 0};
    for (int a = 0; a < 7; ++a) {
        Ht += h[a];
        for (int d = 0; d < 3; ++d) mean[d] += L->e[a][d] * h[a];
    }
    double v[3];
    for (int d = 0; d < 3; ++d) {
        mean[d] /= Ht;
        v[d] = mean[d] + sH * (u[d] - mean[d]);
    }
    equilibrium(L, Ht + Q, v, hs);
}

/* Eq. (H_cm_collision) with the Appendix D source (reading R3).  h holds the
 * shifted variable h - q/2; Q is the source (zeroth moment) of this node. */
static void collide_h(const orc_params* p, const double* h, const double u[3], double Q, double* hs) {
    if (p->hkind == KIND_CUM1) {
        collide_h_cumulant(p, h, u, Q, hs);
        return;
    }
    const lattice_t* L = lattice(p->qh);
    const int n = L->Q;
    const double sH = 1.0 / (p->k / CS2 + 0.5);
    double T[27 * 27], Y[27], Ys[27];
    build_T(L, u, T);
    matvec(n, T, h, Y);
    double H = 0.0;
    for (int a = 0; a < n; ++a) H += h[a];
    H += 0.5 * Q;
    for (int r = 0; r < n; ++r) {
        const int* m = L->mom[r];
        double s = rate_h(p->hkind, m[0] + m[1] + m[2], sH);
        double E = eq_central(m);
        Ys[r] = Y[r] + s * (H * E - Y[r]) + (1.0 - 0.5 * s) * Q * E;
    }
    solve(n, T, Ys, hs);
}

/* index of the velocity of lattice L with the y component reversed */
static int flip_y(const lattice_t* L, int a) {
    for (int b = 0; b < L->Q; ++b)
        if (L->e[b][0] == L->e[a][0] && L->e[b][1] == -L->e[a][1] && L->e[b][2] == L->e[a][2]) return b;
    return a;
}

/* ---- simulation state ---- */
enum { FL_FLUID = 0, FL_SOLID = 1, FL_INLET = 2, FL_OUTLET = 3, FL_MIRROR = 4 };

typedef struct {
    orc_params p;
    int N;
    double* f;      /* pre-collision, [27][N] */
    double* h;      /* pre-collision, [qh][N] */
    double* fs;     /* post-collision scratch */
    double* hs;
    double* fn;     /* streaming target */
    double* hn;
    uint8_t* flags;   /* mirror nodes are kept as FL_SOLID here, see mirror */
    int* mirror;      /* per node: the node it mirrors (symmetry row), or -1 */
    int has_mirror;
    float* qtab;    /* [N*27], -1 where no wall link */
    int* wtab;      /* [N*27], wall id of the link */
    double* Twall;  /* per wall id */
    int nwalls;
    double* theta;  /* per node source Q, or NULL */
} orc_sim;

static int node_of(const orc_sim* s, int x, int y, int z) { return x + s->p.nx * (y + s->p.ny * z); }

/* neighbour x + e (y, z periodic; x periodic or bounded).  Returns -1 when it
 * leaves the domain through a non-periodic x face. */
static int neighbour(const orc_sim* s, int n, int ex, int ey, int ez) {
    int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    int x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    x += ex;
    y = ((y + ey) % ny + ny) % ny;
    z = ((z + ez) % nz + nz) % nz;
    if (s->p.periodic_x) x = ((x % nx) + nx) % nx;
    else if (x < 0 || x >= nx) return -1;
    return node_of(s, x, y, z);
}

orc_sim* orc_create(const orc_params* p) {
    ensure_lattices();
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->p = *p;
    s->N = p->nx * p->ny * p->nz;
    size_t N = (size_t)s->N;
    s->f = (double*)calloc(27 * N, sizeof(double));
    s->fs = (double*)calloc(27 * N, sizeof(double));
    s->fn = (double*)calloc(27 * N, sizeof(double));
    s->h = (double*)calloc((size_t)p->qh * N, sizeof(double));
    s->hs = (double*)calloc((size_t)p->qh * N, sizeof(double));
    s->hn = (double*)calloc((size_t)p->qh * N, sizeof(double));
    s->flags = (uint8_t*)calloc(N, 1);
    s->mirror = (int*)malloc(N * sizeof(int));
    for (size_t i = 0; i < N; ++i) s->mirror[i] = -1;
    s->qtab = (float*)malloc(27 * N * sizeof(float));
    s->wtab = (int*)calloc(27 * N, sizeof(int));
    for (size_t i = 0; i < 27 * N; ++i) s->qtab[i] = -1.0f;
    s->nwalls = 1;
    s->Twall = (double*)calloc(1, sizeof(double));
    return s;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    free(s->f); free(s->fs); free(s->fn); free(s->h); free(s->hs); free(s->hn);
    free(s->flags); free(s->mirror); free(s->qtab); free(s->wtab); free(s->Twall); free(s->theta);
    free(s);
}

/* Geometry: flags (0 fluid, 1 solid, 2 inlet, 3 outlet, 4 symmetry row) and
 * the wall links (node x_b, direction a with x_b + e_a solid, q in (0,1],
 * wall id).  Symmetry rows (the symmetry planes of Sec. 4.4, reading R15)
 * are the whole rows y = 0 and / or y = ny - 1; each of their nodes mirrors
 * the node next to it in y (y = 1 or y = ny - 2), which must not be solid.
 * Returns 0, or a negative code naming the first rule broken:
 *  -1 flag out of range, -2 inlet/outlet planes wrong, -3 link node not
 *  fluid, -4 link target not solid, -5 q outside (0,1], -6 duplicate link,
 *  -7 fluid->solid link missing, -8 solid adjacent to the outlet plane (or,
 *  with the Zou-He inlet, to the inlet plane),
 *  -9 wall id out of range, -10 symmetry rows wrong (or a wall link from a
 *  node next to one). */
int orc_set_geometry(orc_sim* s, const uint8_t* flags, int nlinks, const int* lnode,
                     const int* ldir, const float* lq, const int* lwall, int nwalls) {
    const int N = s->N, nx = s->p.nx, ny = s->p.ny;
    for (int n = 0; n < N; ++n) {
        if (flags[n] > 4) return -1;
        int x = n % nx, y = (n / nx) % ny;
        if (flags[n] == FL_MIRROR) {
            if (ny < 3 || (y != 0 && y != ny - 1)) return -10;
            int src = n + (y == 0 ? nx : -nx);
            if (flags[src] == FL_SOLID || flags[src] == FL_MIRROR) return -10;
            continue;
        }
        if ((y == 0 || y == ny - 1) && ny >= 3) {
            /* a symmetry row is whole */
            int other = n - x;
            for (int xx = 0; xx < nx; ++xx)
                if (flags[other + xx] == FL_MIRROR) return -10;
        }
        if (s->p.periodic_x) {
            if (flags[n] == FL_INLET || flags[n] == FL_OUTLET) return -2;
        } else {
            if ((x == 0) != (flags[n] == FL_INLET)) return -2;
            if ((x == nx - 1) != (flags[n] == FL_OUTLET)) return -2;
            if (x == nx - 2 && flags[n] == FL_SOLID) return -8;
            if (s->p.inlet_bc && x == 1 && flags[n] == FL_SOLID) return -8; /* Zou-He reads x = 1 */
        }
    }
    s->has_mirror = 0;
    for (int n = 0; n < N; ++n) {
        int y = (n / nx) % ny;
        s->mirror[n] = -1;
        if (flags[n] == FL_MIRROR) {
            s->mirror[n] = n + (y == 0 ? nx : -nx);
            s->has_mirror = 1;
        }
    }
    memcpy(s->flags, flags, (size_t)N);
    for (int n = 0; n < N; ++n)
        if (s->flags[n] == FL_MIRROR) s->flags[n] = FL_SOLID;
    for (size_t i = 0; i < 27 * (size_t)N; ++i) { s->qtab[i] = -1.0f; s->wtab[i] = 0; }
    const lattice_t* L = lattice(27);
    for (int l = 0; l < nlinks; ++l) {
        int n = lnode[l], a = ldir[l];
        if (n < 0 || n >= N || a < 0 || a >= 27) return -3;
        if (flags[n] != FL_FLUID) return -3;
        if (s->has_mirror) { /* solid bodies keep off the symmetry rows' neighbours */
            int y = (n / nx) % ny;
            if ((y == 1 && s->mirror[n - nx] >= 0) || (y == ny - 2 && s->mirror[n + nx] >= 0)) return -10;
        }
        int t = neighbour(s, n, L->e[a][0], L->e[a][1], L->e[a][2]);
        if (t < 0 || flags[t] != FL_SOLID) return -4;
        if (!(lq[l] > 0.0f && lq[l] <= 1.0f)) return -5;
        if (s->qtab[(size_t)n * 27 + a] >= 0.0f) return -6;
        if (lwall[l] < 0 || lwall[l] >= nwalls) return -9;
        s->qtab[(size_t)n * 27 + a] = lq[l];
        s->wtab[(size_t)n * 27 + a] = lwall[l];
    }
    for (int n = 0; n < N; ++n) {
        if (flags[n] == FL_SOLID || flags[n] == FL_MIRROR) continue;
        for (int a = 1; a < 27; ++a) {
            int t = neighbour(s, n, L->e[a][0], L->e[a][1], L->e[a][2]);
            if (t >= 0 && flags[t] == FL_SOLID) {
                if (flags[n] != FL_FLUID) {
                    if (flags[n] == FL_OUTLET) return -8;
                    continue; /* inlet populations into a solid are dropped */
                }
                if (s->qtab[(size_t)n * 27 + a] < 0.0f) return -7;
            }
        }
    }
    free(s->Twall);
    s->nwalls = nwalls;
    s->Twall = (double*)calloc((size_t)nwalls, sizeof(double));
    return 0;
}

void orc_set_wall_temperature(orc_sim* s, int wall, double T) {
    if (wall >= 0 && wall < s->nwalls) s->Twall[wall] = T;
}

void orc_set_theta(orc_sim* s, const double* theta) {
    if (!s->theta) s->theta = (double*)calloc((size_t)s->N, sizeof(double));
    memcpy(s->theta, theta, (size_t)s->N * sizeof(double));
}

static double theta_at(const orc_sim* s, int n) { return s->theta ? s->theta[n] : 0.0; }

/* Initial state: equilibria at (rho, u) for f and (H = rho T, u) for h, then
 * the App. D shift h - q/2 (q = Q h^eq(1, u)).  Inlet nodes take the inlet
 * state, solid nodes zero. */
void orc_init_fields(orc_sim* s, const double* rho, const double* u, const double* T) {
    const int N = s->N, qh = s->p.qh;
    const lattice_t* Lh = lattice(qh);
    for (int n = 0; n < N; ++n) {
        double fe[27], he[27], qe[27];
        if (s->flags[n] == FL_SOLID) {
            for (int a = 0; a < 27; ++a) s->f[(size_t)a * N + n] = 0.0;
            for (int a = 0; a < qh; ++a) s->h[(size_t)a * N + n] = 0.0;
            continue;
        }
        double r = rho[n], uu[3] = {u[n], u[N + n], u[2 * N + n]}, TT = T[n];
        if (s->flags[n] == FL_INLET) {
            r = 1.0;
            for (int d = 0; d < 3; ++d) uu[d] = s->p.u_in[d];
            TT = s->p.T_in;
        }
        equilibrium(lattice(27), r, uu, fe);
        equilibrium(Lh, r * TT, uu, he);
        double Q = theta_at(s, n);
        equilibrium(Lh, Q, uu, qe);
        for (int a = 0; a < 27; ++a) s->f[(size_t)a * N + n] = fe[a];
        for (int a = 0; a < qh; ++a) s->h[(size_t)a * N + n] = he[a] - 0.5 * qe[a];
    }
}

void orc_set_state(orc_sim* s, const double* f, const double* h) {
    memcpy(s->f, f, 27 * (size_t)s->N * sizeof(double));
    memcpy(s->h, h, (size_t)s->p.qh * s->N * sizeof(double));
}

void orc_get_state(const orc_sim* s, double* f, double* h) {
    memcpy(f, s->f, 27 * (size_t)s->N * sizeof(double));
    memcpy(h, s->h, (size_t)s->p.qh * s->N * sizeof(double));
}

static double* g_record_u = NULL; /* when set, orc_collide stores u [3][N] there */

/* Collision of every node: pre-collision state -> fs, hs. */
void orc_collide(orc_sim* s) {
    const int N = s->N, qh = s->p.qh;
    const lattice_t* Lh = lattice(qh);
    double feq_in[27], heq_in[27];
    equilibrium(lattice(27), 1.0, s->p.u_in, feq_in);
    equilibrium(Lh, s->p.T_in, s->p.u_in, heq_in);
#pragma omp parallel for schedule(dynamic, 64)
    for (int n = 0; n < N; ++n) {
        double f[27], h[27], fs[27], hs[27], u[3];
        uint8_t fl = s->flags[n];
        if (fl == FL_SOLID) {
            for (int a = 0; a < 27; ++a) s->fs[(size_t)a * N + n] = 0.0;
            for (int a = 0; a < qh; ++a) s->hs[(size_t)a * N + n] = 0.0;
            continue;
        }
        if (fl == FL_INLET && !s->p.inlet_bc) { /* reading R6 */
            for (int a = 0; a < 27; ++a) s->fs[(size_t)a * N + n] = feq_in[a];
            for (int a = 0; a < qh; ++a) s->hs[(size_t)a * N + n] = heq_in[a];
            continue;
        }
        for (int a = 0; a < 27; ++a) f[a] = s->f[(size_t)a * N + n];
        for (int a = 0; a < qh; ++a) h[a] = s->h[(size_t)a * N + n];
        collide_f(&s->p, f, fs, u);
        if (g_record_u)
            for (int d = 0; d < 3; ++d) g_record_u[(size_t)d * N + n] = u[d];
        collide_h(&s->p, h, u, theta_at(s, n), hs);
        for (int a = 0; a < 27; ++a) s->fs[(size_t)a * N + n] = fs[a];
        for (int a = 0; a < qh; ++a) s->hs[(size_t)a * N + n] = hs[a];
    }
}

void orc_set_post(orc_sim* s, const double* fs, const double* hs) {
    memcpy(s->fs, fs, 27 * (size_t)s->N * sizeof(double));
    memcpy(s->hs, hs, (size_t)s->p.qh * s->N * sizeof(double));
}

void orc_get_post(const orc_sim* s, double* fs, double* hs) {
    memcpy(fs, s->fs, 27 * (size_t)s->N * sizeof(double));
    memcpy(hs, s->hs, (size_t)s->p.qh * s->N * sizeof(double));
}

/* q used by the wall formulas: the first-order variants ignore the wall
 * position and bounce back half-way (BB = Eq. IBB at q = 1/2, ABB = Eq. IABB
 * at q = 1/2; Sec. 3) */
static double q_eff(const orc_sim* s, float q) { return s->p.wall_bc ? 0.5 : (double)q; }

/* Eq. (IBB) for one link: the population arriving at x_b in direction abar.
 * fa_b = f*_a(x_b), fab_b = f*_abar(x_b), fa_f = f*_a(x_f), thin = x_f not
 * usable (reading R5). */
static double ibb(double q, double fa_b, double fab_b, double fa_f, int thin) {
    if (q <= 0.5 && !thin) return 2.0 * q * fa_b + (1.0 - 2.0 * q) * fa_f;
    if (q <= 0.5) q = 0.5;
    return (fa_b + (2.0 * q - 1.0) * fab_b) / (2.0 * q);
}

/* Eq. (IABB) for one link; heq_w = h^eq_i(x_w) = w_i T_w (reading R4). */
static double iabb(double q, double ha_b, double hab_b, double ha_f, int thin, double heq_w) {
    if (q <= 0.5 && !thin) return -(2.0 * q * ha_b + (1.0 - 2.0 * q) * ha_f) + 2.0 * heq_w;
    if (q <= 0.5) q = 0.5;
    return (-ha_b + (2.0 * q - 1.0) * hab_b + 2.0 * heq_w) / (2.0 * q);
}

/* Zou-He inlet (Sec. 4.4; reading R20) at inlet node n after the pushes: the
 * populations with e_x = +1 (arriving from outside) are unknown.
 * f: non-equilibrium bounce-back at the prescribed velocity u_in,
 *     f_a = f_abar + f^eq_a(rho, u_in) - f^eq_abar(rho, u_in) - e_ya N_y - e_za N_z,
 * with rho from mass and x-momentum, rho (1 - u_x) = sum_{e_x=0} f + 2 sum_{e_x=-1} f,
 * and N_d = sum_{e_x=0} e_d (f - f^eq) / 6 so that the transverse momentum is
 * rho u_d exactly (the six unknowns with e_d != 0 share the correction).
 * h: the unknowns take the shape of the equilibrium at u_in with the amplitude
 * that makes the zeroth moment rho T_in.
 * zou_he_local applies the rule to one node's arrivals f[27], h[qh] (the
 * e_x = +1 entries are outputs only); for fixed u_in it is affine in (f, h). */
static void zou_he_local(const orc_params* p, const double* u, double* f, double* h) {
    const int qh = p->qh;
    const lattice_t* L = lattice(27);
    const lattice_t* Lh = lattice(qh);
    double known0 = 0.0, known_out = 0.0;
    for (int a = 0; a < 27; ++a) {
        if (L->e[a][0] == 0) known0 += f[a];
        else if (L->e[a][0] < 0) known_out += f[a];
    }
    const double rho = (known0 + 2.0 * known_out) / (1.0 - u[0]);
    double feq[27];
    equilibrium(L, rho, u, feq);
    double Nt[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 27; ++a) {
        if (L->e[a][0] != 0) continue;
        for (int d = 1; d < 3; ++d) Nt[d] += L->e[a][d] * (f[a] - feq[a]);
    }
    for (int d = 1; d < 3; ++d) Nt[d] /= 6.0;
    for (int a = 0; a < 27; ++a) {
        if (L->e[a][0] != 1) continue;
        int ab = L->opp[a];
        f[a] = f[ab] + feq[a] - feq[ab] - L->e[a][1] * Nt[1] - L->e[a][2] * Nt[2];
    }
    double M[27], known_h = 0.0, unknown_w = 0.0;
    equilibrium(Lh, 1.0, u, M);
    for (int a = 0; a < qh; ++a) {
        if (Lh->e[a][0] == 1) unknown_w += M[a];
        else known_h += h[a];
    }
    const double amp = (rho * p->T_in - known_h) / unknown_w;
    for (int a = 0; a < qh; ++a)
        if (Lh->e[a][0] == 1) h[a] = amp * M[a];
}

static void zou_he_inlet(orc_sim* s, int n) {
    const int N = s->N, qh = s->p.qh;
    double f[27], h[27];
    for (int a = 0; a < 27; ++a) f[a] = s->fn[(size_t)a * N + n];
    for (int a = 0; a < qh; ++a) h[a] = s->hn[(size_t)a * N + n];
    zou_he_local(&s->p, s->p.u_in, f, h);
    for (int a = 0; a < 27; ++a) s->fn[(size_t)a * N + n] = f[a];
    for (int a = 0; a < qh; ++a) s->hn[(size_t)a * N + n] = h[a];
}

/* Streaming of fs, hs (push, Sec. 2.1 evolution equation) with Eq. (IBB),
 * Eq. (IABB) and the planes of reading R6.  Result becomes the pre-collision
 * state.  Returns the number of non-solid populations left unset (0 when the
 * geometry is complete). */
int orc_stream(orc_sim* s) {
    const int N = s->N, qh = s->p.qh, nx = s->p.nx;
    const lattice_t* L = lattice(27);
    const lattice_t* Lh = lattice(qh);
    for (size_t i = 0; i < 27 * (size_t)N; ++i) s->fn[i] = NAN;
    for (size_t i = 0; i < (size_t)qh * N; ++i) s->hn[i] = NAN;
    /* symmetry rows (reading R15): specular reflection at the plane halfway
     * between a symmetry row and its neighbour row.  Each symmetry node takes
     * the post-collision populations of the node it mirrors with e_y
     * reversed and pushes them like any node; what arrives there is unused. */
    if (s->has_mirror) {
        for (int n = 0; n < N; ++n) {
            int m = s->mirror[n];
            if (m < 0) continue;
            for (int a = 0; a < 27; ++a)
                s->fs[(size_t)a * N + n] = s->fs[(size_t)flip_y(L, a) * N + m];
            for (int a = 0; a < qh; ++a)
                s->hs[(size_t)a * N + n] = s->hs[(size_t)flip_y(Lh, a) * N + m];
        }
    }
    for (int n = 0; n < N; ++n) {
        if (s->flags[n] == FL_SOLID && s->mirror[n] < 0) continue;
        for (int a = 0; a < 27; ++a) {
            int t = neighbour(s, n, L->e[a][0], L->e[a][1], L->e[a][2]);
            if (t < 0 || s->flags[t] == FL_SOLID) continue;
            s->fn[(size_t)a * N + t] = s->fs[(size_t)a * N + n];
        }
        for (int a = 0; a < qh; ++a) {
            int t = neighbour(s, n, Lh->e[a][0], Lh->e[a][1], Lh->e[a][2]);
            if (t < 0 || s->flags[t] == FL_SOLID) continue;
            s->hn[(size_t)a * N + t] = s->hs[(size_t)a * N + n];
        }
    }
    /* wall links */
    for (int n = 0; n < N; ++n) {
        if (s->flags[n] != FL_FLUID) continue;
        for (int a = 1; a < 27; ++a) {
            float q = s->qtab[(size_t)n * 27 + a];
            if (q < 0.0f) continue;
            int ab = L->opp[a];
            int xf = neighbour(s, n, -L->e[a][0], -L->e[a][1], -L->e[a][2]);
            int thin = (xf < 0 || s->flags[xf] == FL_SOLID);
            double fa_f = thin ? 0.0 : s->fs[(size_t)a * N + xf];
            s->fn[(size_t)ab * N + n] =
                ibb(q_eff(s, q), s->fs[(size_t)a * N + n], s->fs[(size_t)ab * N + n], fa_f, thin);
            /* the same link for h, when the direction belongs to h's lattice */
            for (int i = 0; i < qh; ++i) {
                if (Lh->dir27[i] != a) continue;
                int ib = Lh->opp[i];
                double ha_f = thin ? 0.0 : s->hs[(size_t)i * N + xf];
                double heq = Lh->w[i] * s->Twall[s->wtab[(size_t)n * 27 + a]];
                s->hn[(size_t)ib * N + n] =
                    (s->p.wall_bc == 1) ? heq /* EQ: the wall equilibrium itself */
                                        : iabb(q_eff(s, q), s->hs[(size_t)i * N + n], s->hs[(size_t)ib * N + n],
                                               ha_f, thin, heq);
            }
        }
    }
    /* planes (reading R6; Zou-He inlet, reading R20) */
    if (!s->p.periodic_x) {
        double feq_in[27], heq_in[27];
        equilibrium(L, 1.0, s->p.u_in, feq_in);
        equilibrium(Lh, s->p.T_in, s->p.u_in, heq_in);
        for (int n = 0; n < N; ++n) {
            int x = n % nx;
            if (s->flags[n] == FL_INLET && s->p.inlet_bc) {
                zou_he_inlet(s, n);
            } else if (s->flags[n] == FL_INLET) {
                for (int a = 0; a < 27; ++a) s->fn[(size_t)a * N + n] = feq_in[a];
                for (int a = 0; a < qh; ++a) s->hn[(size_t)a * N + n] = heq_in[a];
            } else if (s->flags[n] == FL_OUTLET && x == nx - 1) {
                for (int a = 0; a < 27; ++a) {
                    if (L->e[a][0] >= 0) continue;
                    int src = neighbour(s, n, 0, -L->e[a][1], -L->e[a][2]);
                    s->fn[(size_t)a * N + n] = s->fs[(size_t)a * N + src];
                }
                for (int a = 0; a < qh; ++a) {
                    if (Lh->e[a][0] >= 0) continue;
                    int src = neighbour(s, n, 0, -Lh->e[a][1], -Lh->e[a][2]);
                    s->hn[(size_t)a * N + n] = s->hs[(size_t)a * N + src];
                }
            }
        }
    }
    int missing = 0;
    for (int n = 0; n < N; ++n) {
        if (s->flags[n] == FL_SOLID) {
            for (int a = 0; a < 27; ++a) s->fn[(size_t)a * N + n] = 0.0;
            for (int a = 0; a < qh; ++a) s->hn[(size_t)a * N + n] = 0.0;
            if (s->mirror[n] >= 0) { /* a symmetry node holds no state of its own */
                for (int a = 0; a < 27; ++a) s->fs[(size_t)a * N + n] = 0.0;
                for (int a = 0; a < qh; ++a) s->hs[(size_t)a * N + n] = 0.0;
            }
            continue;
        }
        for (int a = 0; a < 27; ++a) missing += isnan(s->fn[(size_t)a * N + n]) ? 1 : 0;
        for (int a = 0; a < qh; ++a) missing += isnan(s->hn[(size_t)a * N + n]) ? 1 : 0;
    }
    double* t;
    t = s->f; s->f = s->fn; s->fn = t;
    t = s->h; s->h = s->hn; s->hn = t;
    return missing;
}

int orc_step(orc_sim* s, int nsteps) {
    for (int i = 0; i < nsteps; ++i) {
        orc_collide(s);
        int m = orc_stream(s);
        if (m) return m;
    }
    return 0;
}

/* Macroscopic fields of the pre-collision state (Sec. 2.1): rho = sum f,
 * u = (sum e f + F/2)/rho, H = sum h + Q/2, T = H/rho (c_v = 1).  Solid
 * nodes report 0; inlet nodes the inlet state. */
void orc_macros(const orc_sim* s, double* rho, double* u, double* T) {
    const int N = s->N, qh = s->p.qh;
    const lattice_t* L = lattice(27);
    for (int n = 0; n < N; ++n) {
        if (s->flags[n] == FL_SOLID) {
            rho[n] = 0.0; u[n] = u[N + n] = u[2 * N + n] = 0.0; T[n] = 0.0;
            continue;
        }
        if (s->flags[n] == FL_INLET) {
            rho[n] = 1.0;
            for (int d = 0; d < 3; ++d) u[d * N + n] = s->p.u_in[d];
            T[n] = s->p.T_in;
            continue;
        }
        double r = 0.0, j[3] = {0, 0, 0}, H = 0.0;
        for (int a = 0; a < 27; ++a) {
            double v = s->f[(size_t)a * N + n];
            r += v;
            for (int d = 0; d < 3; ++d) j[d] += L->e[a][d] * v;
        }
        for (int a = 0; a < qh; ++a) H += s->h[(size_t)a * N + n];
        H += 0.5 * theta_at(s, n);
        rho[n] = r;
        for (int d = 0; d < 3; ++d) u[d * N + n] = (j[d] + 0.5 * s->p.F[d]) / r;
        T[n] = H / r;
    }
}

/* Totals over non-solid nodes of rho and H (pre-collision definitions). */
void orc_balances(const orc_sim* s, double* mass, double* energy) {
    const int N = s->N, qh = s->p.qh;
    double m = 0.0, e = 0.0;
    for (int n = 0; n < N; ++n) {
        if (s->flags[n] == FL_SOLID) continue;
        for (int a = 0; a < 27; ++a) m += s->f[(size_t)a * N + n];
        for (int a = 0; a < qh; ++a) e += s->h[(size_t)a * N + n];
        e += 0.5 * theta_at(s, n);
    }
    *mass = m;
    *energy = e;
}

/* Surface heat flux of wall `wall` for the transition t -> t+1 from the
 * current state (reading R8; Sec. 4.4 surface-flux equation): collide, then
 * sum h_ibar(x_b,t+1) - h*_i(x_b,t) over the IABB links of that wall. */
double orc_surface_flux(orc_sim* s, int wall) {
    orc_collide(s);
    const int N = s->N, qh = s->p.qh;
    const lattice_t* L = lattice(27);
    const lattice_t* Lh = lattice(qh);
    double flux = 0.0;
    for (int n = 0; n < N; ++n) {
        if (s->flags[n] != FL_FLUID) continue;
        for (int i = 0; i < qh; ++i) {
            int a = Lh->dir27[i];
            if (a == 0) continue;
            float q = s->qtab[(size_t)n * 27 + a];
            if (q < 0.0f || s->wtab[(size_t)n * 27 + a] != wall) continue;
            int ib = Lh->opp[i];
            int xf = neighbour(s, n, -L->e[a][0], -L->e[a][1], -L->e[a][2]);
            int thin = (xf < 0 || s->flags[xf] == FL_SOLID);
            double ha_f = thin ? 0.0 : s->hs[(size_t)i * N + xf];
            double heq = Lh->w[i] * s->Twall[wall];
            double hin = (s->p.wall_bc == 1)
                             ? heq
                             : iabb(q_eff(s, q), s->hs[(size_t)i * N + n], s->hs[(size_t)ib * N + n], ha_f, thin, heq);
            flux += hin - s->hs[(size_t)i * N + n];
        }
    }
    return flux;
}

/* Force on wall `wall` by momentum exchange (reading R21; not in the paper:
 * Ladd 1994, Mei et al. 2002) over the transition from the post-collision
 * state in s->fs: every link (x_b, a) of the wall carries e_a f*_a(x_b) into
 * the wall and takes back e_a f_abar(x_b, t+1) from Eq. IBB, so
 *     F = sum over the links of e_a (f*_a(x_b) + f_abar(x_b, t+1)). */
static void wall_force_post(const orc_sim* s, int wall, double* F) {
    const int N = s->N;
    const lattice_t* L = lattice(27);
    F[0] = F[1] = F[2] = 0.0;
    for (int n = 0; n < N; ++n) {
        if (s->flags[n] != FL_FLUID) continue;
        for (int a = 1; a < 27; ++a) {
            float q = s->qtab[(size_t)n * 27 + a];
            if (q < 0.0f || s->wtab[(size_t)n * 27 + a] != wall) continue;
            int ab = L->opp[a];
            int xf = neighbour(s, n, -L->e[a][0], -L->e[a][1], -L->e[a][2]);
            int thin = (xf < 0 || s->flags[xf] == FL_SOLID);
            double fa_f = thin ? 0.0 : s->fs[(size_t)a * N + xf];
            double fin = ibb(q_eff(s, q), s->fs[(size_t)a * N + n], s->fs[(size_t)ab * N + n], fa_f, thin);
            double carried = s->fs[(size_t)a * N + n] + fin;
            for (int d = 0; d < 3; ++d) F[d] += L->e[a][d] * carried;
        }
    }
}

/* The wall force for the transition t -> t+1 from the current state:
 * collide, then wall_force_post. */
void orc_wall_force(orc_sim* s, int wall, double* F) {
    orc_collide(s);
    wall_force_post(s, wall, F);
}

/* ---- single-node entry points (used by the pin tests) ---- */
void orc_lattice(int Q, int* e, double* w, int* opp, int* mom) {
    const lattice_t* L = lattice(Q);
    for (int a = 0; a < Q; ++a) {
        for (int d = 0; d < 3; ++d) { e[3 * a + d] = L->e[a][d]; mom[3 * a + d] = L->mom[a][d]; }
        w[a] = L->w[a];
        opp[a] = L->opp[a];
    }
}
void orc_matrix_M(int Q, double* M) { build_M(lattice(Q), M); }
void orc_matrix_T(int Q, const double* u, double* T) { build_T(lattice(Q), u, T); }
void orc_equilibrium(int Q, double psi, const double* u, double* g) { equilibrium(lattice(Q), psi, u, g); }
void orc_cumulants(const double* g, double* C) { cumulants(g, C); }
void orc_cumulants_inverse(const double* C, double* g) { cumulants_inverse(C, g); }
void orc_collide_f(const orc_params* p, const double* f, double* fs, double* u) { collide_f(p, f, fs, u); }
void orc_collide_h(const orc_params* p, const double* h, const double* u, double Q, double* hs) {
    collide_h(p, h, u, Q, hs);
}
int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
/* threads of the OpenMP loops from now on (timing: single- and multi-thread) */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---- adjoint of the h evolution (Sec. 2.1 evolution equation, Eq. H_cm_collision,
 * Eq. IABB) ----------------------------------------------------------------
 * With the velocity field fixed (one-way coupling, Sec. 2: h never feeds back
 * into f), one step maps the post-collision h state s^k to
 *     g^{k+1} = P s^k + b(T_w)          (streaming, Eq. IABB, planes)
 *     s^{k+1} = L(u^{k+1}) g^{k+1} + e(u^{k+1}) theta   (collision, App. D source)
 * Both maps are affine.  L and e are read off the forward collision itself:
 * column j of L is collide_h(unit vector j, u, Q = 0), and e is
 * collide_h(0, u, Q = 1).  The objective J is a weighted sum over a window of
 * levels of a linear flux of s^k (the surface heat flux of one wall, or the
 * x-flux sum e_x h through one plane).  The reverse sweep applies the
 * transposes: lambda^k = P^T mu^{k+1} + dJ/ds^k, mu^k = L(u^k)^T lambda^k,
 * dJ/dtheta += e(u^k)^T lambda^k, dJ/dT_w += (dg^{k+1}/dT_w)^T mu^{k+1}.
 * The state s^0 is the given initial condition. */

/* partial derivatives of one Eq. IABB arrival with respect to its inputs
 * (EQ, wall_bc 1: the arrival is w_i T_w, only d_T = 1) */
static void iabb_partials(const orc_sim* s, float qf, int thin, double* d_ab, double* d_abb, double* d_af,
                          double* d_T) {
    if (s->p.wall_bc == 1) {
        *d_ab = 0.0; *d_abb = 0.0; *d_af = 0.0; *d_T = 1.0;
        return;
    }
    const double q = q_eff(s, qf);
    if (q <= 0.5 && !thin) {
        *d_ab = -2.0 * q; *d_af = -(1.0 - 2.0 * q); *d_abb = 0.0; *d_T = 2.0;
    } else {
        double qq = q <= 0.5 ? 0.5 : q;
        *d_ab = -1.0 / (2.0 * qq); *d_abb = (2.0 * qq - 1.0) / (2.0 * qq); *d_af = 0.0; *d_T = 2.0 / (2.0 * qq);
    }
}

/* Jacobian of the Cumulants-1st collision (Eq. H_cu_collision with the App. D
 * source) at the pre-collision h of one node.  With every cumulant of order
 * >= 2 at its equilibrium the result is h* = (H + Q) M(v): M(v) is the
 * lattice equilibrium of unit zeroth moment at v = (1 - s) m + s u, with
 * H = sum h and m = sum e h / H (the first cumulants).  Hence
 *     dh*_a/dh_b = M_a(v) + (H + Q) sum_d dM_a/dv_d (1 - s) (e_bd - m_d) / H,
 *     dh*_a/dQ   = M_a(v).
 * M is a polynomial of degree two in each v_d, so a central difference of the
 * equilibrium in v_d is its derivative up to rounding.  Jm[a * Q_h + b]. */
static void cum_jacobian(const orc_params* p, const double* h, const double u[3], double Q, double* Jm,
                         double* dQ) {
    const lattice_t* L = lattice(p->qh);
    const int n = L->Q;
    const double s = 1.0 / (p->k / CS2 + 0.5);
    double H = 0.0, m[3] = {0.0, 0.0, 0.0}, v[3];
    for (int a = 0; a < n; ++a) {
        H += h[a];
        for (int d = 0; d < 3; ++d) m[d] += L->e[a][d] * h[a];
    }
    for (int d = 0; d < 3; ++d) {
        m[d] /= H;
        v[d] = m[d] + s * (u[d] - m[d]);
    }
    equilibrium(L, 1.0, v, dQ);
    double dM[3][27];
    const double eps = 1e-3;
    for (int d = 0; d < 3; ++d) {
        double vp[3] = {v[0], v[1], v[2]}, vm[3] = {v[0], v[1], v[2]}, Mp[27], Mm[27];
        vp[d] += eps;
        vm[d] -= eps;
        equilibrium(L, 1.0, vp, Mp);
        equilibrium(L, 1.0, vm, Mm);
        for (int a = 0; a < n; ++a) dM[d][a] = (Mp[a] - Mm[a]) / (2.0 * eps);
    }
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            double acc = 0.0;
            for (int d = 0; d < 3; ++d) acc += dM[d][a] * (1.0 - s) * (L->e[b][d] - m[d]);
            Jm[a * n + b] = dQ[a] + (H + Q) * acc / H;
        }
}


/* whether node t keeps what streaming delivers to it: not outside the box,
 * not solid (symmetry nodes included), not an equilibrium inlet node (which
 * overwrites its arrivals; a Zou-He inlet node keeps the known ones) */
static int receives(const orc_sim* s, int t) {
    if (t < 0 || s->flags[t] == FL_SOLID) return 0;
    if (s->flags[t] == FL_INLET && !s->p.inlet_bc) return 0;
    return 1;
}

static double cd4(double fp1, double fm1, double fp2, double fm2, double e);

/* Adjoint of the Zou-He rule (zou_he_local, reading R20) at every inlet
 * node, in place: mu (the adjoint of the state after the rule) becomes the
 * adjoint of the arrivals, mu_arr = A^T mu with A = d out / d in.  The rule
 * is affine in the arrivals for fixed u_in, so A's columns are the images of
 * unit arrivals minus the image of zero.  muf NULL: the h-only adjoint (f is
 * fixed there, so only the h block of A enters).  With duin non-NULL also
 * duin += (d out / d u_in)^T mu, by 4-point differences at the level's
 * arrivals (frec, hrec: the level's state after the rule, whose known
 * entries are the arrivals). */
static void zou_he_transpose(const orc_sim* s, double* muf, double* muh, const double* frec, const double* hrec,
                             double* duin) {
    const int N = s->N, qh = s->p.qh, M = 27 + qh;
    double* A = (double*)malloc((size_t)M * M * sizeof(double));
    double z_f[27] = {0}, z_h[27] = {0}, c[54];
    zou_he_local(&s->p, s->p.u_in, z_f, z_h);
    for (int i = 0; i < 27; ++i) c[i] = z_f[i];
    for (int i = 0; i < qh; ++i) c[27 + i] = z_h[i];
    for (int j = 0; j < M; ++j) {
        double f[27] = {0}, h[27] = {0};
        if (j < 27) f[j] = 1.0; else h[j - 27] = 1.0;
        zou_he_local(&s->p, s->p.u_in, f, h);
        for (int i = 0; i < 27; ++i) A[(size_t)i * M + j] = f[i] - c[i];
        for (int i = 0; i < qh; ++i) A[(size_t)(27 + i) * M + j] = h[i] - c[27 + i];
    }
    for (int n = 0; n < N; ++n) {
        if (s->flags[n] != FL_INLET) continue;
        double m[54], out[54];
        for (int i = 0; i < 27; ++i) m[i] = muf ? muf[(size_t)i * N + n] : 0.0;
        for (int i = 0; i < qh; ++i) m[27 + i] = muh[(size_t)i * N + n];
        if (duin) {
            const double e = 1e-3;
            const double off[4] = {e, -e, 2 * e, -2 * e};
            for (int d = 0; d < 3; ++d) {
                double v[4];
                for (int k = 0; k < 4; ++k) {
                    double u[3] = {s->p.u_in[0], s->p.u_in[1], s->p.u_in[2]}, f[27], h[27];
                    u[d] += off[k];
                    for (int i = 0; i < 27; ++i) f[i] = frec[(size_t)i * N + n];
                    for (int i = 0; i < qh; ++i) h[i] = hrec[(size_t)i * N + n];
                    zou_he_local(&s->p, u, f, h);
                    double dot = 0.0;
                    for (int i = 0; i < 27; ++i) dot += f[i] * m[i];
                    for (int i = 0; i < qh; ++i) dot += h[i] * m[27 + i];
                    v[k] = dot;
                }
                duin[d] += cd4(v[0], v[1], v[2], v[3], e);
            }
        }
        const int j0 = muf ? 0 : 27;
        for (int j = j0; j < M; ++j) {
            double acc = 0.0;
            for (int i = (muf ? 0 : 27); i < M; ++i) acc += A[(size_t)i * M + j] * m[i];
            out[j] = acc;
        }
        if (muf)
            for (int i = 0; i < 27; ++i) muf[(size_t)i * N + n] = out[i];
        for (int i = 0; i < qh; ++i) muh[(size_t)i * N + n] = out[27 + i];
    }
    free(A);
}

/* lam += P^T mu (transpose of the h part of orc_stream), dTw += (db/dT_w)^T mu.
 * mu is zero at solid and inlet nodes. */
static void stream_transpose_h(const orc_sim* s, const double* mu, double* lam, double* dTw) {
    const int N = s->N, qh = s->p.qh, nx = s->p.nx;
    const lattice_t* L = lattice(27);
    const lattice_t* Lh = lattice(qh);
    for (int n = 0; n < N; ++n) {
        if (s->flags[n] == FL_SOLID && s->mirror[n] < 0) continue;
        for (int a = 0; a < qh; ++a) {
            int t = neighbour(s, n, Lh->e[a][0], Lh->e[a][1], Lh->e[a][2]);
            if (!receives(s, t)) continue;
            /* a symmetry node pushes the mirrored node's population with e_y reversed */
            int src = n, b = a;
            if (s->mirror[n] >= 0) { src = s->mirror[n]; b = flip_y(Lh, a); }
            lam[(size_t)b * N + src] += mu[(size_t)a * N + t];
        }
    }
    for (int n = 0; n < N; ++n) {
        if (s->flags[n] != FL_FLUID) continue;
        for (int i = 0; i < qh; ++i) {
            int a = Lh->dir27[i];
            if (a == 0) continue;
            float q = s->qtab[(size_t)n * 27 + a];
            if (q < 0.0f) continue;
            int ib = Lh->opp[i];
            int xf = neighbour(s, n, -L->e[a][0], -L->e[a][1], -L->e[a][2]);
            int thin = (xf < 0 || s->flags[xf] == FL_SOLID);
            double d_ab, d_abb, d_af, d_T;
            iabb_partials(s, q, thin, &d_ab, &d_abb, &d_af, &d_T);
            double m = mu[(size_t)ib * N + n];
            lam[(size_t)i * N + n] += d_ab * m;
            lam[(size_t)ib * N + n] += d_abb * m;
            if (!thin) lam[(size_t)i * N + xf] += d_af * m;
            if (dTw) dTw[s->wtab[(size_t)n * 27 + a]] += d_T * Lh->w[i] * m;
        }
    }
    if (!s->p.periodic_x) {
        for (int n = 0; n < N; ++n) {
            if (s->flags[n] != FL_OUTLET || n % nx != nx - 1) continue;
            for (int a = 0; a < qh; ++a) {
                if (Lh->e[a][0] >= 0) continue;
                int src = neighbour(s, n, 0, -Lh->e[a][1], -Lh->e[a][2]);
                int b = a;
                if (s->mirror[src] >= 0) { b = flip_y(Lh, a); src = s->mirror[src]; } /* a symmetry node's copy */
                lam[(size_t)b * N + src] += mu[(size_t)a * N + n];
            }
        }
    }
}

/* lam += weight * dF/ds_h, lamf += weight * dF/ds_f and dTw += weight *
 * dF/dT_w for the objective F.  Kinds: 0 surface heat flux of `wall`, 1
 * section flux through x = plane, 2 component comp of the force on `wall`
 * (wall_force_post; lamf must be given). */
static void objective_gradient(const orc_sim* s, int kind, int wall, int plane, int comp, double weight,
                               double* lamf, double* lam, double* dTw) {
    const int N = s->N, qh = s->p.qh, nx = s->p.nx;
    const lattice_t* L = lattice(27);
    const lattice_t* Lh = lattice(qh);
    if (kind == 2) { /* F = sum e_a,comp (f*_a(x_b) + ibb(...)), ibb affine in fs */
        for (int n = 0; n < N; ++n) {
            if (s->flags[n] != FL_FLUID) continue;
            for (int a = 1; a < 27; ++a) {
                float qf = s->qtab[(size_t)n * 27 + a];
                if (qf < 0.0f || s->wtab[(size_t)n * 27 + a] != wall) continue;
                const double c = weight * L->e[a][comp];
                if (c == 0.0) continue;
                int ab = L->opp[a];
                int xf = neighbour(s, n, -L->e[a][0], -L->e[a][1], -L->e[a][2]);
                int thin = (xf < 0 || s->flags[xf] == FL_SOLID);
                const double q = q_eff(s, qf);
                lamf[(size_t)a * N + n] += c;
                if (q <= 0.5 && !thin) {
                    lamf[(size_t)a * N + n] += c * 2.0 * q;
                    lamf[(size_t)a * N + xf] += c * (1.0 - 2.0 * q);
                } else {
                    const double qq = q <= 0.5 ? 0.5 : q;
                    lamf[(size_t)a * N + n] += c / (2.0 * qq);
                    lamf[(size_t)ab * N + n] += c * (2.0 * qq - 1.0) / (2.0 * qq);
                }
            }
        }
        return;
    }
    if (kind == 1) { /* section flux sum e_x h over the plane x = plane */
        for (int n = 0; n < N; ++n) {
            if (n % nx != plane || s->flags[n] == FL_SOLID) continue;
            for (int i = 0; i < qh; ++i) lam[(size_t)i * N + n] += weight * Lh->e[i][0];
        }
        return;
    }
    for (int n = 0; n < N; ++n) { /* surface flux of wall (reading R8) */
        if (s->flags[n] != FL_FLUID) continue;
        for (int i = 0; i < qh; ++i) {
            int a = Lh->dir27[i];
            if (a == 0) continue;
            float q = s->qtab[(size_t)n * 27 + a];
            if (q < 0.0f || s->wtab[(size_t)n * 27 + a] != wall) continue;
            int ib = Lh->opp[i];
            int xf = neighbour(s, n, -L->e[a][0], -L->e[a][1], -L->e[a][2]);
            int thin = (xf < 0 || s->flags[xf] == FL_SOLID);
            double d_ab, d_abb, d_af, d_T;
            iabb_partials(s, q, thin, &d_ab, &d_abb, &d_af, &d_T);
            lam[(size_t)i * N + n] += weight * (d_ab - 1.0);
            lam[(size_t)ib * N + n] += weight * d_abb;
            if (!thin) lam[(size_t)i * N + xf] += weight * d_af;
            if (dTw) dTw[wall] += weight * d_T * Lh->w[i];
        }
    }
}

/* the objective F(s) of the post-collision state in s->fs, s->hs */
static double objective_value(orc_sim* s, int kind, int wall, int plane, int comp) {
    const int N = s->N, qh = s->p.qh, nx = s->p.nx;
    const lattice_t* L = lattice(27);
    const lattice_t* Lh = lattice(qh);
    double F = 0.0;
    if (kind == 2) {
        double Fw[3];
        wall_force_post(s, wall, Fw);
        return Fw[comp];
    }
    if (kind == 1) {
        for (int n = 0; n < N; ++n) {
            if (n % nx != plane || s->flags[n] == FL_SOLID) continue;
            for (int i = 0; i < qh; ++i) F += Lh->e[i][0] * s->hs[(size_t)i * N + n];
        }
        return F;
    }
    for (int n = 0; n < N; ++n) {
        if (s->flags[n] != FL_FLUID) continue;
        for (int i = 0; i < qh; ++i) {
            int a = Lh->dir27[i];
            if (a == 0) continue;
            float q = s->qtab[(size_t)n * 27 + a];
            if (q < 0.0f || s->wtab[(size_t)n * 27 + a] != wall) continue;
            int ib = Lh->opp[i];
            int xf = neighbour(s, n, -L->e[a][0], -L->e[a][1], -L->e[a][2]);
            int thin = (xf < 0 || s->flags[xf] == FL_SOLID);
            double ha_f = thin ? 0.0 : s->hs[(size_t)i * N + xf];
            double hin = (s->p.wall_bc == 1) ? Lh->w[i] * s->Twall[wall]
                                             : iabb(q_eff(s, q), s->hs[(size_t)i * N + n], s->hs[(size_t)ib * N + n],
                                                    ha_f, thin, Lh->w[i] * s->Twall[wall]);
            F += hin - s->hs[(size_t)i * N + n];
        }
    }
    return F;
}

/* Forward run from the post-collision state (f_post, h_post) = s^0 over
 * nsteps steps; returns J = weight * sum_{k=t0..t1} F(s^k).  With dtheta /
 * dTw non-NULL it also runs the reverse sweep and adds dJ/dtheta[N] and
 * dJ/dT_w[nwalls] to them.  Returns 0, -1 on a streaming error, or -4 for
 * gradients of a force objective (kind 2; orc_adjoint_flow carries the f part
 * they need).  Symmetry rows enter through the streaming transpose (a
 * symmetry node pushes its mirrored node's populations with e_y reversed); a
 * Zou-He inlet through zou_he_transpose (h block: f, hence rho, is fixed
 * here) after each level's collision transposes, its nodes colliding like
 * fluid nodes.
 * The Cumulants-1st collision is not affine in h: for that kind the forward
 * keeps the pre-collision h of every level and the reverse sweep applies the
 * transpose of the collision's Jacobian there (cum_jacobian); streaming and
 * the walls stay affine. */
int orc_adjoint(orc_sim* s, const double* f_post, const double* h_post, int nsteps, int t0, int t1, int kind,
                int wall, int plane, int comp, double weight, double* J, double* dtheta, double* dTw) {
    const int N = s->N, qh = s->p.qh;
    const size_t HN = (size_t)qh * N;
    const int cum = s->p.hkind == KIND_CUM1;
    const int zou_he = s->p.inlet_bc && !s->p.periodic_x;
    /* a force objective depends on f: only the coupled adjoint carries it */
    if (dtheta && kind == 2) return -4;
    double* urec = dtheta ? (double*)malloc((size_t)(nsteps + 1) * 3 * N * sizeof(double)) : NULL;
    double* hrec = (dtheta && cum) ? (double*)malloc((size_t)(nsteps + 1) * HN * sizeof(double)) : NULL;
    orc_set_post(s, f_post, h_post);
    double Jv = 0.0;
    for (int k = 0; k <= nsteps; ++k) {
        if (k >= t0 && k <= t1) Jv += weight * objective_value(s, kind, wall, plane, comp);
        if (k == nsteps) break;
        if (orc_stream(s) != 0) { free(urec); free(hrec); return -1; }
        if (hrec) memcpy(hrec + (size_t)(k + 1) * HN, s->h, HN * sizeof(double));
        g_record_u = urec ? urec + (size_t)(k + 1) * 3 * N : NULL;
        orc_collide(s);
        g_record_u = NULL;
    }
    *J = Jv;
    if (!dtheta) return 0;
    double* mu = (double*)calloc(HN, sizeof(double));
    double* lam = (double*)calloc(HN, sizeof(double));
    for (int k = nsteps; k >= 0; --k) {
        for (size_t i = 0; i < HN; ++i) lam[i] = 0.0;
        if (k < nsteps) stream_transpose_h(s, mu, lam, dTw);
        if (k >= t0 && k <= t1) objective_gradient(s, kind, wall, plane, comp, weight, NULL, lam, dTw);
        for (size_t i = 0; i < HN; ++i) mu[i] = 0.0;
        if (k == 0) break;
#pragma omp parallel for schedule(dynamic, 16)
        for (int n = 0; n < N; ++n) {
            if (s->flags[n] == FL_SOLID || (s->flags[n] == FL_INLET && !zou_he)) continue;
            double u[3], Lm[27 * 27], col[27], unit[27], e[27], zero[27];
            for (int d = 0; d < 3; ++d) u[d] = urec[(size_t)k * 3 * N + (size_t)d * N + n];
            if (cum) {
                double g[27];
                for (int i = 0; i < qh; ++i) g[i] = hrec[(size_t)k * HN + (size_t)i * N + n];
                cum_jacobian(&s->p, g, u, theta_at(s, n), Lm, e);
            } else {
                for (int j = 0; j < qh; ++j) {
                    for (int i = 0; i < qh; ++i) unit[i] = (i == j) ? 1.0 : 0.0;
                    collide_h(&s->p, unit, u, 0.0, col);
                    for (int i = 0; i < qh; ++i) Lm[i * qh + j] = col[i];
                }
                for (int i = 0; i < qh; ++i) zero[i] = 0.0;
                collide_h(&s->p, zero, u, 1.0, e);
            }
            double dth = 0.0;
            for (int i = 0; i < qh; ++i) dth += e[i] * lam[(size_t)i * N + n];
            dtheta[n] += dth;
            for (int j = 0; j < qh; ++j) {
                double v = 0.0;
                for (int i = 0; i < qh; ++i) v += Lm[i * qh + j] * lam[(size_t)i * N + n];
                mu[(size_t)j * N + n] = v;
            }
        }
        /* the Zou-He inlet built the inlet nodes' state of level k from their arrivals */
        if (zou_he) zou_he_transpose(s, NULL, mu, NULL, NULL, NULL);
    }
    free(mu);
    free(lam);
    free(urec);
    free(hrec);
    return 0;
}

/* ---- adjoint of the coupled f + h evolution --------------------------------
 * Gradients of the same objectives with respect to parameters of the flow:
 * the body force F (reading R2) and the inlet velocity u_in (reading R6).
 * The h step depends on the flow through u, so the adjoint carries an f
 * part: with the pre-collision arrivals g_f, g_h of level k,
 *     s_f = C_f(g_f; F),  u = U(g_f; F),  s_h = C_h(g_h, u; Q)
 * (Eq. hydro_cu_collision, Eq. H_cm_collision / H_cu_collision), and the
 * reverse sweep applies, per node,
 *     w   = (dC_h/du)^T lambda_h
 *     mu_f = (dC_f/dg_f)^T lambda_f + (dU/dg_f)^T w
 *     mu_h = (dC_h/dg_h)^T lambda_h
 *     dJ/dF += (dC_f/dF)^T lambda_f + (dU/dF)^T w,   dJ/dQ += (dC_h/dQ)^T lambda_h,
 * with lambda = P^T mu^{k+1} + dJ/ds^k as before (streaming, Eq. IBB for f,
 * Eq. IABB for h, the planes).  The inlet plane holds the equilibria at u_in
 * at every level k >= 1, so dJ/du_in += (d f^eq_in/du_in)^T lambda_f +
 * (d h^eq_in/du_in)^T lambda_h there.  Every Jacobian is read off the
 * forward functions themselves by 4-point central differences,
 * D = [8 (F(x+e) - F(x-e)) - (F(x+2e) - F(x-2e))] / (12 e), whose error is
 * O(e^4): exact for the polynomial dependence on u and F, and at the level
 * of rounding for the rational dependence on the density. */
static double cd4(double fp1, double fm1, double fp2, double fm2, double e) {
    return (8.0 * (fp1 - fm1) - (fp2 - fm2)) / (12.0 * e);
}

/* lam += P_f^T mu (transpose of the f part of orc_stream). */
static void stream_transpose_f(const orc_sim* s, const double* mu, double* lam) {
    const int N = s->N, nx = s->p.nx;
    const lattice_t* L = lattice(27);
    for (int n = 0; n < N; ++n) {
        if (s->flags[n] == FL_SOLID && s->mirror[n] < 0) continue;
        for (int a = 0; a < 27; ++a) {
            int t = neighbour(s, n, L->e[a][0], L->e[a][1], L->e[a][2]);
            if (!receives(s, t)) continue;
            int src = n, b = a;
            if (s->mirror[n] >= 0) { src = s->mirror[n]; b = flip_y(L, a); }
            lam[(size_t)b * N + src] += mu[(size_t)a * N + t];
        }
    }
    for (int n = 0; n < N; ++n) { /* Eq. IBB: the arrival ab at n from the link (n, a) */
        if (s->flags[n] != FL_FLUID) continue;
        for (int a = 1; a < 27; ++a) {
            float qf = s->qtab[(size_t)n * 27 + a];
            if (qf < 0.0f) continue;
            int ab = L->opp[a];
            int xf = neighbour(s, n, -L->e[a][0], -L->e[a][1], -L->e[a][2]);
            int thin = (xf < 0 || s->flags[xf] == FL_SOLID);
            const double q = q_eff(s, qf);
            const double m = mu[(size_t)ab * N + n];
            if (q <= 0.5 && !thin) {
                lam[(size_t)a * N + n] += 2.0 * q * m;
                lam[(size_t)a * N + xf] += (1.0 - 2.0 * q) * m;
            } else {
                const double qq = q <= 0.5 ? 0.5 : q;
                lam[(size_t)a * N + n] += m / (2.0 * qq);
                lam[(size_t)ab * N + n] += (2.0 * qq - 1.0) / (2.0 * qq) * m;
            }
        }
    }
    if (!s->p.periodic_x) {
        for (int n = 0; n < N; ++n) {
            if (s->flags[n] != FL_OUTLET || n % nx != nx - 1) continue;
            for (int a = 0; a < 27; ++a) {
                if (L->e[a][0] >= 0) continue;
                int src = neighbour(s, n, 0, -L->e[a][1], -L->e[a][2]);
                int b = a;
                if (s->mirror[src] >= 0) { b = flip_y(L, a); src = s->mirror[src]; } /* a symmetry node's copy */
                lam[(size_t)b * N + src] += mu[(size_t)a * N + n];
            }
        }
    }
}

/* Returns 0 or -1 on a streaming error.  dF[3] and duin[3] (and dtheta[N],
 * dTw[nwalls]) are added to.  Symmetry rows enter through the streaming
 * transposes; a Zou-He inlet through zou_he_transpose after each level's
 * collision transposes (its nodes collide like fluid nodes). */
int orc_adjoint_flow(orc_sim* s, const double* f_post, const double* h_post, int nsteps, int t0, int t1, int kind,
                     int wall, int plane, int comp, double weight, double* J, double* dtheta, double* dTw,
                     double* dF, double* duin) {
    const int N = s->N, qh = s->p.qh;
    const size_t FN = (size_t)27 * N, HN = (size_t)qh * N;
    const int zou_he = s->p.inlet_bc && !s->p.periodic_x;
    double* frec = (double*)malloc((size_t)(nsteps + 1) * FN * sizeof(double));
    double* hrec = (double*)malloc((size_t)(nsteps + 1) * HN * sizeof(double));
    orc_set_post(s, f_post, h_post);
    double Jv = 0.0;
    for (int k = 0; k <= nsteps; ++k) {
        if (k >= t0 && k <= t1) Jv += weight * objective_value(s, kind, wall, plane, comp);
        if (k == nsteps) break;
        if (orc_stream(s) != 0) { free(frec); free(hrec); return -1; }
        memcpy(frec + (size_t)(k + 1) * FN, s->f, FN * sizeof(double));
        memcpy(hrec + (size_t)(k + 1) * HN, s->h, HN * sizeof(double));
        orc_collide(s);
    }
    *J = Jv;
    const lattice_t* L = lattice(27);
    const lattice_t* Lh = lattice(qh);
    /* derivatives of the inlet equilibria with respect to u_in */
    double dfin[3][27], dhin[3][27];
    {
        const double e = 1e-3;
        for (int d = 0; d < 3; ++d) {
            double fv[4][27], hv[4][27];
            const double off[4] = {e, -e, 2 * e, -2 * e};
            for (int j = 0; j < 4; ++j) {
                double u[3] = {s->p.u_in[0], s->p.u_in[1], s->p.u_in[2]};
                u[d] += off[j];
                equilibrium(L, 1.0, u, fv[j]);
                equilibrium(Lh, s->p.T_in, u, hv[j]);
            }
            for (int a = 0; a < 27; ++a) dfin[d][a] = cd4(fv[0][a], fv[1][a], fv[2][a], fv[3][a], e);
            for (int a = 0; a < qh; ++a) dhin[d][a] = cd4(hv[0][a], hv[1][a], hv[2][a], hv[3][a], e);
        }
    }
    double* muf = (double*)calloc(FN, sizeof(double));
    double* muh = (double*)calloc(HN, sizeof(double));
    double* lamf = (double*)calloc(FN, sizeof(double));
    double* lamh = (double*)calloc(HN, sizeof(double));
    double* gF = (double*)calloc((size_t)3 * N, sizeof(double));
    for (int k = nsteps; k >= 0; --k) {
        for (size_t i = 0; i < FN; ++i) lamf[i] = 0.0;
        for (size_t i = 0; i < HN; ++i) lamh[i] = 0.0;
        if (k < nsteps) {
            stream_transpose_f(s, muf, lamf);
            stream_transpose_h(s, muh, lamh, dTw);
        }
        if (k >= t0 && k <= t1) objective_gradient(s, kind, wall, plane, comp, weight, lamf, lamh, dTw);
        for (size_t i = 0; i < FN; ++i) muf[i] = 0.0;
        for (size_t i = 0; i < HN; ++i) muh[i] = 0.0;
        if (k == 0) break;
        /* equilibrium inlet: its nodes hold the equilibria at u_in */
        if (!s->p.periodic_x && !zou_he && duin) {
            for (int n = 0; n < N; ++n) {
                if (s->flags[n] != FL_INLET) continue;
                for (int d = 0; d < 3; ++d) {
                    double acc = 0.0;
                    for (int a = 0; a < 27; ++a) acc += dfin[d][a] * lamf[(size_t)a * N + n];
                    for (int a = 0; a < qh; ++a) acc += dhin[d][a] * lamh[(size_t)a * N + n];
                    duin[d] += acc;
                }
            }
        }
#pragma omp parallel for schedule(dynamic, 8)
        for (int n = 0; n < N; ++n) {
            if (s->flags[n] == FL_SOLID || (s->flags[n] == FL_INLET && !zou_he)) continue;
            double g[27], gh[27], u[3], fs0[27], hs0[27];
            for (int a = 0; a < 27; ++a) g[a] = frec[(size_t)k * FN + (size_t)a * N + n];
            for (int a = 0; a < qh; ++a) gh[a] = hrec[(size_t)k * HN + (size_t)a * N + n];
            const double Q = theta_at(s, n);
            collide_f(&s->p, g, fs0, u);
            double lf[27], lh[27];
            for (int a = 0; a < 27; ++a) lf[a] = lamf[(size_t)a * N + n];
            for (int a = 0; a < qh; ++a) lh[a] = lamh[(size_t)a * N + n];
            /* w = (dC_h/du)^T lambda_h and (dC_h/dg_h)^T lambda_h, dC_h/dQ */
            double w[3];
            {
                const double e = 1e-3;
                const double off[4] = {e, -e, 2 * e, -2 * e};
                for (int d = 0; d < 3; ++d) {
                    double v[4];
                    for (int j = 0; j < 4; ++j) {
                        double uu[3] = {u[0], u[1], u[2]}, hs[27];
                        uu[d] += off[j];
                        collide_h(&s->p, gh, uu, Q, hs);
                        double dot = 0.0;
                        for (int a = 0; a < qh; ++a) dot += lh[a] * hs[a];
                        v[j] = dot;
                    }
                    w[d] = cd4(v[0], v[1], v[2], v[3], e);
                }
                const double eh = 1e-4;
                const double offh[4] = {eh, -eh, 2 * eh, -2 * eh};
                for (int b = 0; b < qh; ++b) {
                    double v[4];
                    for (int j = 0; j < 4; ++j) {
                        double gg[27], hs[27];
                        for (int a = 0; a < qh; ++a) gg[a] = gh[a];
                        gg[b] += offh[j];
                        collide_h(&s->p, gg, u, Q, hs);
                        double dot = 0.0;
                        for (int a = 0; a < qh; ++a) dot += lh[a] * hs[a];
                        v[j] = dot;
                    }
                    muh[(size_t)b * N + n] = cd4(v[0], v[1], v[2], v[3], eh);
                }
                if (dtheta) {
                    double v[4];
                    for (int j = 0; j < 4; ++j) {
                        double hs[27];
                        collide_h(&s->p, gh, u, Q + offh[j], hs);
                        double dot = 0.0;
                        for (int a = 0; a < qh; ++a) dot += lh[a] * hs[a];
                        v[j] = dot;
                    }
                    dtheta[n] += cd4(v[0], v[1], v[2], v[3], eh);
                }
            }
            /* mu_f = (dC_f/dg)^T lambda_f + (dU/dg)^T w */
            {
                const double e = 1e-4;
                const double off[4] = {e, -e, 2 * e, -2 * e};
                for (int b = 0; b < 27; ++b) {
                    double v[4];
                    for (int j = 0; j < 4; ++j) {
                        double gg[27], fs[27], uu[3];
                        for (int a = 0; a < 27; ++a) gg[a] = g[a];
                        gg[b] += off[j];
                        collide_f(&s->p, gg, fs, uu);
                        double dot = 0.0;
                        for (int a = 0; a < 27; ++a) dot += lf[a] * fs[a];
                        for (int d = 0; d < 3; ++d) dot += w[d] * uu[d];
                        v[j] = dot;
                    }
                    muf[(size_t)b * N + n] = cd4(v[0], v[1], v[2], v[3], e);
                }
                /* dJ/dF: F enters the collision and the velocity of h */
                for (int d = 0; d < 3; ++d) {
                    double v[4];
                    for (int j = 0; j < 4; ++j) {
                        orc_params pp = s->p;
                        pp.F[d] += off[j];
                        double fs[27], uu[3];
                        collide_f(&pp, g, fs, uu);
                        double dot = 0.0;
                        for (int a = 0; a < 27; ++a) dot += lf[a] * fs[a];
                        for (int dd = 0; dd < 3; ++dd) dot += w[dd] * uu[dd];
                        v[j] = dot;
                    }
                    gF[(size_t)d * N + n] += cd4(v[0], v[1], v[2], v[3], e);
                }
            }
        }
        if (zou_he)
            zou_he_transpose(s, muf, muh, frec + (size_t)k * FN, hrec + (size_t)k * HN, duin);
    }
    if (dF)
        for (int d = 0; d < 3; ++d) {
            double acc = 0.0;
            for (int n = 0; n < N; ++n) acc += gF[(size_t)d * N + n];
            dF[d] += acc;
        }
    free(muf); free(muh); free(lamf); free(lamh); free(gF); free(frec); free(hrec);
    return 0;
}

/* ---- geometry of spheres in a channel (Sec. 3: q along the link) ---------
 * The definition, node by node: a node is solid when it lies in a closed
 * ball |x - c|^2 <= R^2, periodic images in y and z included (shifts of -1,
 * 0, +1 periods, enough for 2R below ny and nz), not in x; with periodic_x =
 * 0 the planes x = 0 and x = nx-1 are inlet (2) and outlet (3).  A fluid
 * node's link a (target inside 0 <= x < nx, y and z wrapped) is a wall link
 * when the target lies in a ball; q is the smaller root t of
 * |d + t e_a|^2 = R^2 with d the node's offset from that ball's centre in the
 * same image frame, clipped to (0, 1] and rounded to float.  Links come out
 * sorted by (node, direction).  Returns the number of links; writes at most
 * cap of them. */
static int ball_image(double x, double y, double z, int ns, const double* c, const double* r, int ny, int nz,
                      int* ky, int* kz) {
    for (int i = 0; i < ns; ++i) {
        const double RR = r[i] * r[i];
        for (int a = -1; a <= 1; ++a)
            for (int b = -1; b <= 1; ++b) {
                const double dx = x - c[3 * i], dy = (y + a * ny) - c[3 * i + 1], dz = (z + b * nz) - c[3 * i + 2];
                const double d2 = dx * dx + dy * dy + dz * dz;
                if (d2 <= RR) {
                    *ky = a;
                    *kz = b;
                    return i;
                }
            }
    }
    return -1;
}

int64_t orc_build_spheres(int nx, int ny, int nz, int periodic_x, int ns, const double* centres,
                          const double* radii, const int* wall_ids, uint8_t* flags, int64_t cap, int* lnode,
                          int* ldir, float* lq, int* lwall) {
    const lattice_t* L = lattice(27);
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t n = 0; n < N; ++n) {
        const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
        int ky, kz;
        uint8_t f = 0;
        if (!periodic_x) f = (x == 0) ? 2 : (x == nx - 1 ? 3 : 0);
        if (ball_image(x, y, z, ns, centres, radii, ny, nz, &ky, &kz) >= 0) f = 1;
        flags[n] = f;
    }
    int64_t k = 0;
    for (int64_t n = 0; n < N; ++n) {
        if (flags[n] != 0) continue;
        const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
        for (int a = 1; a < 27; ++a) {
            const int ex = L->e[a][0], ey = L->e[a][1], ez = L->e[a][2];
            if (x + ex < 0 || x + ex >= nx) continue;
            int ky, kz;
            const int i = ball_image(x + ex, y + ey, z + ez, ns, centres, radii, ny, nz, &ky, &kz);
            if (i < 0) continue;
            if (k < cap) {
                const double dx = x - centres[3 * i];
                const double dy = (double)(y + ky * ny) - centres[3 * i + 1];
                const double dz = (double)(z + kz * nz) - centres[3 * i + 2];
                const double ee = (double)(ex * ex + ey * ey + ez * ez);
                const double de = dx * ex + dy * ey + dz * ez;
                const double dd = dx * dx + dy * dy + dz * dz;
                double disc = de * de - ee * (dd - radii[i] * radii[i]);
                if (disc < 0.0) disc = 0.0;
                double t = (-de - sqrt(disc)) / ee;
                const double tmin = nextafter(0.0, 1.0);
                if (t < tmin) t = tmin;
                if (t > 1.0) t = 1.0;
                float q = (float)t;
                if (q <= 0.0f) q = 1.17549435e-38f; /* FLT_MIN */
                lnode[k] = (int)n;
                ldir[k] = a;
                lq[k] = q;
                lwall[k] = wall_ids ? wall_ids[i] : 0;
            }
            ++k;
        }
    }
    return k;
}
