/*
 * lbm.h - C ABI of the GB300 (sm_103a) thermal lattice Boltzmann library.
 *
 * The library advances the double-distribution thermal LBM of
 * Gruszczynski & Laniewski-Wollk (arXiv 2203.01316) on one GPU: flow
 * populations f (D3Q27, cumulant collision, Sec. 2.1.1 Eq. hydro_cu_collision)
 * and internal-energy populations h (D3Q27 or D3Q7, central-moment collision,
 * Eq. H_cm_collision, kinds CM-TRT / CM-SRT / CM-1st), streamed with
 * interpolated bounce-back for f (Sec. 3, Eq. IBB) and interpolated
 * anti-bounce-back Dirichlet walls for h (Sec. 3, Eq. IABB) on every wall link
 * with its wall-distance fraction q.
 *
 * Conventions used by every call:
 *  - Grid nx x ny x nz, node index n = x + nx*(y + ny*z).  y and z are
 *    periodic.  x is periodic, or bounded by an inlet plane (x = 0) and an
 *    outlet plane (x = nx-1).
 *  - Velocity a is the a-th vector of the paper's D3Q27 list (Sec. 2.1); D3Q7
 *    uses the vectors {0,+x,+y,+z,-x,-y,-z} = D3Q27 indices {0,1,2,3,7,8,9}.
 *  - Population arrays are structure-of-arrays [Q][N] (all N values of
 *    velocity 0, then velocity 1, ...).
 *  - `is_device` = 1 means the pointer is CUDA device memory (for example a
 *    torch tensor's data_ptr()), 0 means host memory.  The library copies what
 *    it needs; the caller keeps ownership of every buffer it passes.
 *  - The library owns all the device memory of a context.  Calls are
 *    asynchronous on the context's stream unless stated otherwise.
 *  - Every call returns an lbm_status; none aborts or prints.  On failure
 *    lbm_last_error() gives a message.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID = 1,  /* bad argument or geometry; nothing changed */
    LBM_ERR_NOMEM = 2,    /* device or host allocation failed */
    LBM_ERR_CUDA = 3,     /* a CUDA call failed; message holds its text */
    LBM_ERR_DIVERGED = 4, /* a non-finite population was found */
    LBM_ERR_STATE = 5     /* call out of order (e.g. step before geometry) */
} lbm_status;

typedef enum { LBM_D3Q27 = 27, LBM_D3Q7 = 7 } lbm_lattice;

/* Sec. 2.1.1: rates of the h collision (s^H = 1/(3k + 1/2)).  Central-moment
 * kinds (Eq. H_cm_collision): TRT: odd orders s^H, even orders 1.  SRT: all
 * s^H.  1ST: order 1 s^H, higher orders 1.  CUM_1ST (Eq. H_cu_collision,
 * "Cumulants-1st"): first-order cumulants s^H, higher orders set to their
 * equilibrium; needs a positive zeroth moment sum(h) everywhere, and has no
 * adjoint here (its step is not affine in h). */
typedef enum { LBM_H_CM_TRT = 0, LBM_H_CM_SRT = 1, LBM_H_CM_1ST = 2, LBM_H_CUM_1ST = 3 } lbm_hkind;

/* Storage of populations in HBM.  Every type stores the shifted values
 * f - w*rho0 and h - w*T_ref; arithmetic is FP32 (FP64 for LBM_F64).  The
 * 16-bit types round stochastically by default (lbm_params.round_nearest). */
typedef enum { LBM_F32 = 0, LBM_F64 = 1, LBM_F16_SHIFTED = 2, LBM_BF16_SHIFTED = 3 } lbm_storage;

typedef struct {
    int nx, ny, nz;      /* grid; nx*ny*nz*27 must stay below 2^31 */
    int lat_h;           /* lbm_lattice of h */
    int hkind;           /* lbm_hkind */
    int storage;         /* lbm_storage */
    int periodic_x;      /* 1: periodic x; 0: inlet plane x=0, outlet x=nx-1 */
    double nu;           /* kinematic viscosity (lattice units), > 0 */
    double k;            /* thermal diffusivity k (rho c_v = 1), > 0, or 0 to derive from Pr */
    double Pr;           /* Prandtl number nu/k, or 0 to derive from k; if both are
                            given they must agree to 1e-12 relative */
    double omega_bulk;   /* relaxation rate of the trace of the second-order
                            cumulants (0 < omega_bulk < 2); 1 sets it to equilibrium */
    double rho0, T_ref;  /* shift references of the stored populations */
    void* cuda_stream;   /* cudaStream_t to run on; NULL = the library creates one */
    int round_nearest;   /* 16-bit storage: 0 = stochastic rounding (unbiased, reproducible:
                            random bits hashed from node, population and time level),
                            1 = round to nearest even */
    int step_kernel;     /* lbm_step_kernel: implementation of lbm_step (same results) */
    int wall_bc;         /* lbm_wall_bc: wall rules */
    int inlet_bc;        /* lbm_inlet_bc: inlet plane rule (periodic_x = 0) */
} lbm_params;

/* Inlet plane rules (Sec. 4.4).  EQUILIBRIUM: the inlet nodes hold the
 * equilibria at (rho = 1, u_in) and (T_in, u_in) as their post-collision
 * state.  ZOU_HE: the inlet nodes stream and collide like fluid nodes; the
 * populations entering from outside (e_x = +1) are set by non-equilibrium
 * bounce-back at u_in for f (density from mass and x-momentum, transverse
 * momentum corrected to rho u_in exactly) and, for h, take the equilibrium
 * shape at u_in with the amplitude that makes the zeroth moment rho T_in.
 * With ZOU_HE the plane x = 1 holds no solid node. */
typedef enum { LBM_INLET_EQUILIBRIUM = 0, LBM_INLET_ZOU_HE = 1 } lbm_inlet_bc;

/* Wall rules (Sec. 3).  IBB_IABB: Eq. IBB for f, Eq. IABB for h, with each
 * link's q (second order).  BB_EQ: bounce-back for f (Eq. IBB at q = 1/2) and
 * EQ for h: the population arriving from the wall is the wall equilibrium
 * w_i T_w (first order).  BB_ABB: bounce-back and anti-bounce-back (Eq. IABB
 * at q = 1/2). */
typedef enum { LBM_WALL_IBB_IABB = 0, LBM_WALL_BB_EQ = 1, LBM_WALL_BB_ABB = 2 } lbm_wall_bc;

/* Implementation of lbm_step.  Both run the fused one-node-per-thread
 * kernel (f and h of a node in one thread; the fastest measured on GB300).
 * LBM_STEP_AUTO replays a CUDA graph of two steps for calls of 4 or more
 * steps (captured on the context's stream at first use and again whenever
 * the buffers or parameters it captured change; with 16-bit storage the
 * graph advances a device copy of the time level that seeds the stochastic
 * rounding), which removes the launch gaps that dominate small grids;
 * results are bit-identical to LBM_STEP_CLASSIC, which launches every step.
 * While the caller is capturing the context's stream, lbm_step launches
 * every step. */
typedef enum { LBM_STEP_AUTO = 0, LBM_STEP_CLASSIC = 1 } lbm_step_kernel;

/* Create a context and allocate its device state.  The populations are zero
 * until lbm_init_fields.  Errors: LBM_ERR_INVALID (parameters), NOMEM, CUDA. */
lbm_status lbm_create(const lbm_params* params, lbm_ctx** out);

/* Free every resource of the context (synchronises its stream). */
lbm_status lbm_destroy(lbm_ctx* ctx);

/* Geometry (Sec. 3).  flags: uint8[N], 0 fluid, 1 solid, 2 inlet, 3 outlet,
 * 4 symmetry row.
 * Wall links: n_links entries (link_node[l], link_dir[l]) meaning node
 * link_node is fluid and link_node + e_{link_dir} is solid; link_q in (0,1]
 * is the fraction of the link at which the wall lies (Eq. IBB's q);
 * link_wall in [0, n_walls) names the wall, whose temperature lbm_set_bc
 * sets.  Symmetry rows model the symmetry planes of Sec. 4.4: the whole row
 * y = 0 and / or y = ny-1 (every x and z) may be flagged 4; the plane lies
 * halfway between that row and its neighbour row, where populations reflect
 * specularly (e_y reversed).  Symmetry nodes hold no state of their own
 * (macros, balances and fluxes skip them, and populations read zero there).
 * Rules checked (LBM_ERR_INVALID otherwise): with periodic_x = 0 the
 * x = 0 plane is all inlet, x = nx-1 all outlet (symmetry rows excepted),
 * and x = nx-2 holds no solid; inlet/outlet flags appear nowhere else; every
 * fluid->solid link is listed exactly once; symmetry rows are whole, their
 * neighbour rows hold no solid node and no wall link.  Links may come in any
 * order.  Replaces any earlier geometry; the populations must be
 * (re)initialised afterwards. */
lbm_status lbm_set_geometry(lbm_ctx* ctx, const uint8_t* flags, int64_t n_links,
                            const int32_t* link_node, const int32_t* link_dir,
                            const float* link_q, const int32_t* link_wall, int n_walls,
                            int is_device);

/* Geometry of a channel with spherical obstacles, built on the device and
 * installed as by lbm_set_geometry (Sec. 3; the workloads of Sec. 4 are
 * spheres and cylinders in channels).  centres: host double[3*n_spheres]
 * (x, y, z), radii: host double[n_spheres], wall_ids: host int32[n_spheres]
 * in [0, n_walls) or NULL (all 0).  A node is solid when it lies in a closed
 * ball |x - c|^2 <= R^2, periodic images in y and z included (not in x);
 * with periodic_x = 0 the planes x = 0 and x = nx-1 are inlet and outlet.  A
 * fluid node's link a is a wall link when its target x + e_a (inside
 * 0 <= x < nx) lies in a ball; q is the smallest t in (0, 1] with
 * |x + t e_a - c| = R, from the node's coordinates in the image frame of
 * that ball, computed in FP64 with one rounding per operation in the order
 * d = x - c, e.d = (d_x e_x + d_y e_y) + d_z e_z, d.d likewise,
 * disc = max((e.d)^2 - |e|^2 (d.d - R^2), 0), t = (-e.d - sqrt(disc)) / |e|^2,
 * clipped to [smallest positive double, 1] and rounded to float (a float 0
 * becomes the smallest normal float).  Spheres must not touch one another and
 * must satisfy lbm_set_geometry's rules.  flags_out: host uint8[N] receiving
 * the flags (0 fluid, 1 solid, 2 inlet, 3 outlet), or NULL; the links can be
 * read with lbm_get_links.  Errors: LBM_ERR_INVALID (radius not in
 * (0, min(ny, nz)/2), wall id out of range, or a rule of lbm_set_geometry),
 * NOMEM, CUDA. */
lbm_status lbm_build_spheres(lbm_ctx* ctx, int n_spheres, const double* centres, const double* radii,
                             const int32_t* wall_ids, int n_walls, uint8_t* flags_out);

/* Dirichlet temperature of wall `wall_id` for Eq. IABB (h^eq_i(x_w) = w_i T_w,
 * wall velocity zero).  Takes effect at the next step. */
lbm_status lbm_set_bc(lbm_ctx* ctx, int wall_id, double T_wall);

/* Inlet plane state: post-collision populations there are the equilibria at
 * (rho = 1, u_in) and (T_in, u_in). */
lbm_status lbm_set_inlet(lbm_ctx* ctx, double ux, double uy, double uz, double T_in);

/* Uniform body force on f: collision adds F to the momentum, and
 * u = (sum e f + F/2)/rho is the velocity used for h. */
lbm_status lbm_set_force(lbm_ctx* ctx, double Fx, double Fy, double Fz);

/* Per-node heat source Q (float[N]) of Appendix D; NULL clears it.  The
 * library keeps the App. D shifted variable h - q/2 internally. */
lbm_status lbm_set_source(lbm_ctx* ctx, const float* theta, int is_device);

/* Initialise every node at equilibrium: f^eq(rho, u), h^eq(rho*T, u) (then
 * the App. D shift), and apply one collision so the stored state is
 * post-collision.  rho[N], u[3*N] (all x, then all y, then all z), T[N],
 * double.  Solid nodes are ignored; inlet nodes take the inlet state. */
lbm_status lbm_init_fields(lbm_ctx* ctx, const double* rho, const double* u, const double* T,
                           int is_device);

/* Advance n time steps (pull streaming + walls + planes + collision of f
 * and h), asynchronously on the context's stream.  n >= 0. */
lbm_status lbm_step(lbm_ctx* ctx, int n);

/* Macroscopic fields of the current time level (Sec. 2.1): rho, u (3*N,
 * SoA), T = H/rho with H = sum h + Q/2; double.  Solid nodes give 0, inlet
 * nodes the inlet state.  Synchronises; LBM_ERR_DIVERGED if a value is
 * non-finite. */
lbm_status lbm_macros(lbm_ctx* ctx, double* rho, double* u, double* T, int is_device);

/* Post-collision populations of the current time level, unshifted, double:
 * f[27*N], h[Q_h*N].  Either pointer may be NULL.  Synchronises. */
lbm_status lbm_get_populations(lbm_ctx* ctx, double* f, double* h, int is_device);

/* FP64 totals over non-solid nodes of rho and H.  Synchronises;
 * LBM_ERR_DIVERGED if any population is non-finite. */
lbm_status lbm_balances(lbm_ctx* ctx, double* mass, double* energy);

/* Surface heat flux of wall `wall_id` for the transition from the current
 * time level to the next (Sec. 4.4): the sum over that wall's IABB links of
 * h_ibar(x_b, t+1) - h*_i(x_b, t), FP64.  Synchronises. */
lbm_status lbm_surface_flux(lbm_ctx* ctx, int wall_id, double* flux);

/* Nusselt number Nu = flux * length / (k * area * dT) (Sec. 4.4), with the
 * flux of lbm_surface_flux.  Synchronises. */
lbm_status lbm_nusselt(lbm_ctx* ctx, int wall_id, double length, double area, double dT,
                       double* nu_out);

/* Section heat flux (Sec. 4.4, Eq. heat_flux_section): sum of e_x h over the
 * non-solid nodes of the plane x = plane_x, from the current post-collision
 * state, FP64.  Synchronises. */
lbm_status lbm_section_flux(lbm_ctx* ctx, int plane_x, double* flux);

/* Force on wall wall_id by momentum exchange (not in the paper: Ladd 1994,
 * Mei et al. 2002), for the transition from the current post-collision state
 * to the next step: force[d] = sum over the wall's links (x_b, a) of
 * e_a,d (f*_a(x_b) + f_abar(x_b, t+1)), with f_abar from Eq. IBB exactly as
 * lbm_step applies it and full populations (the storage shift included).
 * force: host double[3].  In a periodic box the forces on all walls add up to
 * N_fluid F minus the change of the fluid's momentum over the step.
 * LBM_ERR_INVALID for a wall id out of range.  Synchronises. */
lbm_status lbm_wall_force(lbm_ctx* ctx, int wall_id, double* force);

/* Bytes needed by lbm_save_state. */
lbm_status lbm_state_size(lbm_ctx* ctx, size_t* bytes);

/* Copy the stored populations (with a header naming the grid, lattice and
 * storage) to a buffer of *bytes bytes, host memory or (is_device = 1) device
 * memory; *bytes is set to the size used.  Synchronises. */
lbm_status lbm_save_state(lbm_ctx* ctx, void* buf, size_t* bytes, int is_device);

/* Restore a state written by lbm_save_state of a context with the same grid,
 * lattice and storage (LBM_ERR_INVALID otherwise); buf in host or
 * (is_device = 1) device memory. */
lbm_status lbm_load_state(lbm_ctx* ctx, const void* buf, size_t bytes, int is_device);

/* ---- adjoint of the h evolution -------------------------------------------
 * One-way coupling (Sec. 2: h does not act on f) fixes the velocity field of
 * the h evolution.  For the central-moment kinds the h step is then affine in
 * the h state, the per-node source Q (App. D) and the wall temperatures
 * (Eq. IABB):
 *     g^{k+1} = P s^k + b(T_w),   s^{k+1} = L(u^{k+1}) g^{k+1} + e(u^{k+1}) Q
 * (s^k: post-collision h of level k, g: arrivals after streaming and walls,
 * L, e from Eq. H_cm_collision).  The Cumulants-1st collision is nonlinear in
 * g; its adjoint uses the Jacobian at recorded states (lbm_step_record_h,
 * lbm_adjoint_step_h).  An objective is a linear function F of s^k (a heat
 * flux of h; for the coupled adjoint below also a wall force of f) summed
 * with a weight over a window of levels; the adjoint runs the transposed steps
 * backwards.  Velocity records, adjoint arrays: element type
 * float, or double for LBM_F64 contexts; SoA [3][N] and [Q_h][N]. */
typedef enum { LBM_OBJ_SURFACE_FLUX = 0, LBM_OBJ_SECTION_FLUX = 1, LBM_OBJ_WALL_FORCE = 2 } lbm_objective_kind;
typedef struct {
    int kind;       /* lbm_objective_kind */
    int wall_id;    /* SURFACE_FLUX, WALL_FORCE: the wall */
    int plane_x;    /* SECTION_FLUX: the plane (lbm_section_flux's flux) */
    int component;  /* WALL_FORCE: 0, 1, 2 for the x, y, z component of lbm_wall_force */
    double weight;  /* J += weight * F(level) */
} lbm_objective;

/* *J_device (device double) += weight * F(current level); asynchronous. */
lbm_status lbm_objective_accumulate(lbm_ctx* ctx, const lbm_objective* obj, double* J_device);

/* Advance n steps like lbm_step and record, for each step k = 1..n, the
 * velocity u used by every node's collision at u_rec + (k-1)*3*N (device).
 * advance_h = 0 advances f only and leaves h untouched (the velocity
 * recomputation of the adjoint needs no h). */
lbm_status lbm_step_record(lbm_ctx* ctx, int n, void* u_rec, int advance_h);

/* lbm_step_record with advance_h = 1 that also copies, for each step
 * k = 1..n, the post-collision h of every node as deviations h* - w T_ref to
 * h_rec + (k-1)*Q_h*N (device, SoA [Q_h][N], element type as for u_rec).
 * The Cumulants-1st collision (Eq. H_cu_collision) is not linear in h, so its
 * adjoint needs these records (lbm_adjoint_step_h); solid nodes hold zeros. */
lbm_status lbm_step_record_h(lbm_ctx* ctx, int n, void* u_rec, void* h_rec);

/* One level of the adjoint sweep.  mu_next: adjoint of the arrivals of level
 * k+1 (zeros at the last level).  Computes lambda^k = P^T mu_next + dJ/ds^k
 * (obj: the objective term of level k, NULL when level k is outside the
 * window); then, if u_level (the velocity of level k's collision, from
 * lbm_step_record) is given, writes mu^k = L(u^k)^T lambda^k to out and adds
 * e(u^k)^T lambda^k to dJ_dtheta[N] (device double, may be NULL); with
 * u_level NULL (the initial level) it writes lambda^0 to out.  The dJ/dT_w
 * terms are accumulated inside the context (lbm_adjoint_wall_gradient).
 * mu_next must be zero at solid nodes and, with the equilibrium inlet, at
 * inlet nodes (true of zero-filled arrays and of every out this call
 * writes); mu_next and out must not alias.  Symmetry rows and the Zou-He
 * inlet are covered: a symmetry row passes the adjoint back to the row
 * beside it with e_y reversed, and a Zou-He inlet node collides like a fluid
 * node whose unknown h arrivals (e_x = +1) depend on its known ones through
 * the rule sum h = rho T_in, rho held fixed.  Asynchronous. */
lbm_status lbm_adjoint_step(lbm_ctx* ctx, const void* u_level, const void* mu_next, void* out,
                            const lbm_objective* obj, double* dJ_dtheta);
/* (A WALL_FORCE objective depends on f: lbm_adjoint_step and
 * lbm_adjoint_step_h return LBM_ERR_INVALID for it; lbm_adjoint_flow_step
 * takes it.) */

/* lbm_adjoint_step for every h kind, given also h_level, the level's
 * post-collision h record from lbm_step_record_h (ignored by the
 * central-moment kinds, may be NULL there and at the initial level).  For
 * Cumulants-1st the level's collision is h* = (H + Q) M(v), M the unit
 * equilibrium at v = (1 - s^H) m + s^H u, m = sum e h / H (Eq. H_cu_collision
 * with every cumulant of order >= 2 at equilibrium, App. D source), and the
 * call applies the transpose of its Jacobian at the recorded state.
 * lbm_adjoint_step itself returns LBM_ERR_INVALID for that kind. */
lbm_status lbm_adjoint_step_h(lbm_ctx* ctx, const void* u_level, const void* h_level, const void* mu_next, void* out,
                              const lbm_objective* obj, double* dJ_dtheta);

/* ---- adjoint of the coupled f + h evolution ---------------------------------
 * Gradients of the same objectives with respect to parameters of the flow,
 * the body force F (lbm_set_force) and the inlet velocity u_in (the
 * equilibrium inlet plane of lbm_set_inlet): the h step depends on the flow
 * through u, so this sweep carries the adjoint of f as well (Eq.
 * hydro_cu_collision, Eq. IBB) next to that of h (Eq. H_cm_collision or
 * H_cu_collision, Eq. IABB).  FP32 or FP64 storage only (LBM_ERR_INVALID
 * otherwise); symmetry rows and the Zou-He inlet are covered as in
 * lbm_adjoint_step (with the Zou-He inlet, dJ/du_in differentiates the rule
 * that builds the inlet's unknown arrivals).  Adjoint arrays:
 * element type float (FP32) or double (FP64), SoA [27][N] for f and [Q_h][N]
 * for h. */

/* lbm_step_record with advance_h = 1 that records, for each step k = 1..n,
 * what the coupled adjoint needs of the pre-collision arrivals (deviations,
 * after streaming, the walls and the planes) of every node that collides
 * (fluid and outlet nodes, and inlet nodes with the Zou-He inlet, whose
 * unknown arrivals the rule has filled).  Level k's f record starts at
 * f_rec + (k-1)*F and holds the ten raw moments of the f arrivals as
 * [10][N] (sum f, sum e_x f, sum e_y f, sum e_z f, sum e_x^2 f, sum e_y^2 f,
 * sum e_z^2 f, sum e_x e_y f, sum e_x e_z f, sum e_y e_z f: the f collision
 * reads f only through them), followed, with the Zou-He inlet, by the inlet
 * nodes' 27 arrivals as [27][ny*nz] (row y + ny*z); F = 10*N, plus 27*ny*nz
 * with the Zou-He inlet (inlet_bc = LBM_INLET_ZOU_HE and periodic_x = 0).  Level k's h record holds the h arrivals [Q_h][N]
 * at h_rec + (k-1)*Q_h*N.  Element type as the storage (float or double),
 * device memory; lbm_flow_record_size gives F and Q_h*N.  Other nodes'
 * entries are left as they are. */
lbm_status lbm_step_record_pre(lbm_ctx* ctx, int n, void* f_rec, void* h_rec);

/* Elements of one level's f and h records of lbm_step_record_pre (see there).
 * Errors: LBM_ERR_INVALID for null arguments. */
lbm_status lbm_flow_record_size(lbm_ctx* ctx, int64_t* f_elems, int64_t* h_elems);

/* One level k of the coupled adjoint sweep: from the adjoints of the next
 * level's arrivals (muf_next, muh_next; zeros at the last level) and the
 * level's records (f_level, h_level from lbm_step_record_pre; both NULL at
 * the initial level, whose state is given), writes mu^k to muf_out, muh_out,
 * adds dJ/dtheta to dJ_dtheta[N] (device double, may be NULL), and
 * accumulates dJ/dF, dJ/du_in (lbm_adjoint_flow_gradient) and dJ/dT_w
 * (lbm_adjoint_wall_gradient) inside the context.  obj: the objective term of
 * level k or NULL.  The *_next arrays must be zero at solid and inlet nodes
 * (true of zero-filled arrays and of every out this call writes); inputs and
 * outputs must not alias.  Asynchronous. */
lbm_status lbm_adjoint_flow_step(lbm_ctx* ctx, const void* f_level, const void* h_level, const void* muf_next,
                                 const void* muh_next, void* muf_out, void* muh_out, const lbm_objective* obj,
                                 double* dJ_dtheta);

/* dJ/dF[3] and dJ/du_in[3] (host double) accumulated by lbm_adjoint_flow_step
 * since the last reset; reset = 1 clears the accumulators.  Synchronises. */
lbm_status lbm_adjoint_flow_gradient(lbm_ctx* ctx, double* dJ_dF, double* dJ_duin, int reset);

/* dJ/dT_w accumulated by lbm_adjoint_step since the last reset, per wall
 * (host double[n_walls]); reset = 1 clears the accumulators.  Synchronises. */
lbm_status lbm_adjoint_wall_gradient(lbm_ctx* ctx, double* dJ_dTwall, int reset);

/* Streaming map used by the step: src[a*N + n] = node whose post-collision
 * population a arrives at node n, -1 where a wall link replaces it, -2 for
 * nodes that do not pull (solid, inlet).  int32[27*N]; is_device as above.
 * Synchronises. */
lbm_status lbm_stream_map(lbm_ctx* ctx, int32_t* src, int is_device);

/* The wall links as stored by the library, sorted by (node, dir): up to
 * *n_links entries are written; *n_links is set to the total.  Host memory.
 * Synchronises. */
lbm_status lbm_get_links(lbm_ctx* ctx, int64_t* n_links, int32_t* node, int32_t* dir,
                         float* q, int32_t* wall);

/* FP64 totals of caller-owned FP32 population arrays, computed without
 * allocating device memory.  The paper has no counterpart: this is a library
 * service for callers that cannot call cudaMalloc, such as code running
 * inside a host framework that owns every device buffer and passes them in
 * (a plugin or custom-call interface with no allocator), or an application
 * whose device memory budget is fixed at start-up.
 * f: device float[27 * n_nodes], h: device float[q_h * n_nodes], each SoA
 * [Q][n_nodes] (all values of velocity 0, then velocity 1, ...), holding a
 * post-collision state as deviations from w*rho0 and w*T_ref (pass
 * rho0 = T_ref = 0 for plain populations).
 * flags: device uint8[n_nodes] with the flag values of lbm_set_geometry, or
 * NULL for all nodes; solid (1) and symmetry-row (4) nodes are skipped, as
 * lbm_balances skips them.  theta: device float[n_nodes], the App. D source
 * of lbm_set_source, or NULL; each counted node's energy is then
 * sum(h) - theta/2 (the energy lbm_balances and lbm_macros report).
 * totals: device double[3] written with (sum rho, sum H, number of counted
 * nodes holding a non-finite value).  Runs asynchronously on cuda_stream
 * (NULL = default stream) of the calling thread's current device; all
 * pointers must belong to that device.
 * Scratch lives in a fixed 64 KiB device array inside the library, so
 * n_nodes is limited to 33,554,432 (LBM_ERR_INVALID beyond).  Each call whose
 * stream is not being captured looks up that array's address in the current
 * CUDA context; a call made during stream capture reuses the address the
 * last uncaptured call on that device found (LBM_ERR_STATE if there was
 * none), so make the first call on a device before any capture, and note
 * that a context reset after that call invalidates the address a later
 * capture would record.  Calls whose kernels overlap on the GPU share the
 * array and race; serialise them.  Errors: LBM_ERR_INVALID, LBM_ERR_STATE,
 * LBM_ERR_CUDA, message in lbm_last_error(NULL). */
lbm_status lbm_balances_noalloc(const float* f, const float* h, int q_h, int64_t n_nodes,
                                const uint8_t* flags, const float* theta, double rho0, double T_ref,
                                double* totals, void* cuda_stream);

/* Wait for the context's stream; reports an asynchronous CUDA error. */
lbm_status lbm_sync(lbm_ctx* ctx);

/* Message of the last failed call on this context (or of lbm_create when
 * ctx is NULL).  Valid until the next call. */
const char* lbm_last_error(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
